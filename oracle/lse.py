"""Smooth (logsumexp) segment statistic and its adjoint, FP64 (test infrastructure).

The paper's search keeps, per chunk and searched width, the maximum boxcar
power (Algorithm 4).  The differentiable extension replaces that maximum by
its logsumexp relaxation at temperature tau,

    Y[s, w] = tau * log sum_{k in seg s, k <= M - w} exp(S_w[k] / tau),

which tends to the maximum as tau -> 0.  The adjoint runs the forward chain
backwards: softmax weights -> boxcar scatter (the adjoint of S_w[k] =
sum_{j<w} P[k+j] adds each weight to every bin of its window) -> P = (a^2 +
b^2)/2 -> the per-block median/MAD normalisation of Eq. 8 (including the
almost-everywhere derivatives of the selected order statistics) -> the real
FFT (DC bin zeroed, so it passes no gradient) -> the time series -> the
amplitude A of an injected template (x = noise + A * template).
"""
import numpy as np

from . import boxcar, fft, normalise


def _order_stat_weights(v):
    """d median(v) / d v as a dense weight vector (one or two entries)."""
    n = v.shape[0]
    order = np.argsort(v, kind="stable")
    wts = np.zeros(n)
    if n % 2 == 1:
        wts[order[n // 2]] = 1.0
    else:
        wts[order[n // 2 - 1]] += 0.5
        wts[order[n // 2]] += 0.5
    return wts


def _lse(v, tau, axis=-1):
    """tau * log sum exp(v / tau) along axis, shifted by the maximum."""
    mv = np.max(v, axis=axis, keepdims=True)
    return np.squeeze(mv, axis=axis) + tau * np.log(np.sum(np.exp((v - mv) / tau), axis=axis))


def forward_power(p, w_max, seg_len, tau):
    """Y[s, w - 1] for normalised power p (FP64)."""
    m = p.shape[0]
    bounds = normalise.block_bounds(m, seg_len)
    n_seg = len(bounds)
    y = np.full((n_seg, w_max), -np.inf)
    for w, s in boxcar.boxcar_widths(p, w_max):
        n_valid = m - w + 1
        # segments 0..f-1: full L-bin segments with every start bin valid
        f = 0
        while f < n_seg - 1 and bounds[f][1] <= n_valid:
            f += 1
        if f > 0:
            y[:f, w - 1] = _lse(s[: f * seg_len].reshape(f, seg_len), tau)
        for si in range(f, n_seg):
            lo, hi = bounds[si]
            hi = min(hi, n_valid)
            if lo < hi:
                y[si, w - 1] = _lse(s[lo:hi], tau)
    return y


def backward_power(p, y, g, w_max, seg_len, tau):
    """dL/dP from dL/dY = g: softmax weights, then the boxcar scatter."""
    m = p.shape[0]
    bounds = normalise.block_bounds(m, seg_len)
    seg_of = np.empty(m, dtype=np.int64)
    for si, (lo, hi) in enumerate(bounds):
        seg_of[lo:hi] = si
    dp = np.zeros(m)
    for w, s in boxcar.boxcar_widths(p, w_max):
        n_valid = m - w + 1
        sg = seg_of[:n_valid]
        gs = g[sg, w - 1] * np.exp((s - y[sg, w - 1]) / tau)     # dL/dS_w[k]
        # dP[j] += sum_{k = j-w+1}^{j} gs[k]  (window sums by prefix sums)
        c = np.concatenate([[0.0], np.cumsum(gs)])
        j = np.arange(m)
        hi = np.minimum(j, n_valid - 1) + 1
        lo = np.maximum(j - w + 1, 0)
        dp += np.where(hi > lo, c[hi] - c[np.minimum(lo, n_valid)], 0.0)
    return dp


def forward(x, w_max, seg_len, tau):
    """Y and the saved forward state for the full chain from a time series."""
    spec = fft.rfft(x)
    p, stats, flags = normalise.normalise_power(spec, seg_len)
    if flags.any():
        raise ValueError("zero-MAD block: statistic not differentiable")
    return forward_power(p, w_max, seg_len, tau), dict(spec=spec, p=p, stats=stats)


def backward(x, state, y, g, w_max, seg_len, tau):
    """dL/dx for L with dL/dY = g."""
    n = x.shape[0]
    spec, p, stats = state["spec"], state["p"], state["stats"]
    dp = backward_power(p, y, g, w_max, seg_len, tau)
    xs = np.array(spec, dtype=np.complex128)
    xs[0] = 0.0
    g_re = np.zeros(xs.shape[0])
    g_im = np.zeros(xs.shape[0])
    for si, (lo, hi) in enumerate(normalise.block_bounds(xs.shape[0], seg_len)):
        for comp, out, col in ((xs.real, g_re, 0), (xs.imag, g_im, 2)):
            v = comp[lo:hi]
            med, mad = stats[si, col], stats[si, col + 1]
            scale = normalise.KAPPA * mad
            a = (v - med) / scale
            g_a = dp[lo:hi] * a                       # P = (a^2 + b^2) / 2
            dmed = _order_stat_weights(v)             # d med / d v_i
            dev = np.abs(v - med)
            sel = _order_stat_weights(dev)            # which deviations set the MAD
            sgn = np.sign(v - med)
            # d MAD / d v_i = sum_m sel_m sgn_m (delta_mi - dmed_i)
            dmad = sel * sgn - np.sum(sel * sgn) * dmed
            out[lo:hi] = (g_a / scale
                          - np.sum(g_a) / scale * dmed
                          - np.sum(g_a * (v - med)) / (scale * mad) * dmad)
    g_re[0] = 0.0       # X_0 := 0 is a constant
    g_im[0] = 0.0
    return fft.rfft_adjoint(g_re, g_im, n)


def amplitude_grad(g_x, template):
    """dL/dA for x = noise + A * template."""
    return float(np.dot(np.asarray(g_x, dtype=np.float64), np.asarray(template, dtype=np.float64)))
