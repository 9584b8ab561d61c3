"""The paper's GPU approximations ("paper-GPU fidelity" mode), FP64 (test infrastructure).

Two steps of Pulscan's GPU-native version are approximations of the CPU
version's exact ones:

* Median and MAD by median of medians (§2.5 and the appendix's "Median of
  Medians Normalisation" listing): over a chunk of 4^k values, each level
  with stride s replaces element t < s by local_median(v[t], v[t+s], v[t+2s],
  v[t+3s]), s = 4^(k-1), ..., 1, where local_median(a, b, c, d) is the mean of
  the two middle values, (a + b + c + d - min - max) / 2.  The MAD is the
  same reduction over the deviations from that median, and the scale factor
  is 1.4826.
* Significance by a fitted polynomial (§2.6, Eqs. 10-12, "Power to Log
  Probability Calculation"): log p = pow f(x) / A1 with x = A1 dof / pow,
  A1 = 1500 and f the degree-16 polynomial below; log p = 0 when
  dof >= 1.05 pow.  pow is a chi-square value with dof degrees of freedom
  (in this code's convention pow = 2 S and dof = 2 a, a the gamma shape of S).
"""
import numpy as np

from . import boxcar, normalise, significance

MOM_SCALE = 1.4826
A1 = 1500.0
CUTOFF = 1.05
# A2 .. A18: coefficients of f from x^16 down to the constant term (§2.6 appendix listing)
POLY = (-4.4604059e-46, 9.4927863e-42, -9.1470451e-38, 5.2810851e-34, -2.0376166e-30, 5.5480334e-27,
        -1.0973877e-23, 1.5991804e-20, -1.7231488e-17, 1.3660070e-14, -7.8617952e-12, 3.2136336e-09,
        -9.0466418e-07, 0.00016945948, -0.021494231, 2.9515954, -755.24091)


def local_median(a, b, c, d):
    """Mean of the two middle values of four (elementwise)."""
    mn = np.minimum(np.minimum(np.minimum(a, b), c), d)
    mx = np.maximum(np.maximum(np.maximum(a, b), c), d)
    return (a + b + c + d - mn - mx) / 2.0


def median_of_medians(v):
    """The stride-4 reduction of the listing over 4^k values."""
    s = np.asarray(v, dtype=np.float64)
    n = s.shape[0]
    if n < 1 or (n & (n - 1)) or (n.bit_length() - 1) % 2:
        raise ValueError("median of medians needs 4^k values")
    while s.shape[0] > 1:
        q = s.shape[0] // 4
        s = local_median(s[:q], s[q:2 * q], s[2 * q:3 * q], s[3 * q:4 * q])
    return float(s[0])


def normalise_power_mom(spec, seg_len):
    """P = (a^2 + b^2)/2 with median and MAD of each component by median of
    medians over the first seg_len bins of each block (seg_len = 4^k; the last
    block's extra bins are normalised with the same statistics), scale 1.4826.
    Returns (P, stats[med_re, mad_re, med_im, mad_im], zero-MAD flags)."""
    x = np.array(spec, dtype=np.complex128)
    x[0] = 0.0
    m = x.shape[0]
    bounds = normalise.block_bounds(m, seg_len)
    p = np.zeros(m)
    st = np.zeros((len(bounds), 4))
    flags = np.zeros(len(bounds), dtype=bool)
    for i, (lo, hi) in enumerate(bounds):
        comps = []
        for c in (x.real[lo:hi], x.imag[lo:hi]):
            med = median_of_medians(c[:seg_len])
            mad = median_of_medians(np.abs(c[:seg_len] - med))
            comps.append((c, med, mad))
        st[i] = [comps[0][1], comps[0][2], comps[1][1], comps[1][2]]
        if comps[0][2] == 0.0 or comps[1][2] == 0.0:
            flags[i] = True
            continue
        a = (comps[0][0] - comps[0][1]) / (MOM_SCALE * comps[0][2])
        b = (comps[1][0] - comps[1][1]) / (MOM_SCALE * comps[1][2])
        p[lo:hi] = 0.5 * (a * a + b * b)
    return p, st, flags


def poly_logp(pow_, dof):
    """§2.6: natural log p of a chi-square value pow with dof degrees of freedom."""
    pow_ = np.asarray(pow_, dtype=np.float64)
    dof = np.asarray(dof, dtype=np.float64)
    x = A1 * dof / np.where(pow_ > 0, pow_, 1.0)
    f = np.zeros(np.broadcast(pow_, dof).shape)
    for c in POLY:
        f = f * x + c
    return np.where(dof >= CUTOFF * pow_, 0.0, pow_ * f / A1)


def log_p_adjusted_poly(shape, s, n_trials):
    """Bonferroni-corrected ln p of a sum S of gamma shape a by the polynomial
    (pow = 2 S, dof = 2 a), capped at 0."""
    return np.minimum(0.0, poly_logp(2.0 * np.asarray(s, dtype=np.float64), 2.0 * shape) + np.log(float(n_trials)))


def search_power_poly(p, w_max, seg_len, sigma_thr, n_trials):
    """Candidates with the polynomial significance (same maxima as the exact
    search; only the emission rule and sigma change)."""
    mx, am = boxcar.segment_maxima(p, w_max, seg_len)
    target = float(significance.log_sf_normal(sigma_thr))
    out = []
    for w in range(1, w_max + 1):
        col = mx[:, w - 1]
        for s in np.nonzero(~np.isnan(col))[0]:
            lp = float(log_p_adjusted_poly(w, col[s], n_trials))
            if lp <= target:
                out.append(dict(segment=int(s), width=w, bin=int(am[s, w - 1]), power=float(col[s]),
                                sigma=float(significance.sigma_from_log_p(np.array([lp]))[0])))
    out.sort(key=lambda r: (r["segment"], r["width"]))
    return out
