"""End-to-end boxcar search in the paper's order, FP64 (test infrastructure).

FFT (own radix-2) -> per-block median/MAD normalisation and power (§2.2.3,
Eq. 8) -> boxcar bank for widths 1..W (§2.2.5) -> per-(segment, width)
maximum (Algorithm 4) -> chi-square significance with Bonferroni correction
and a sigma threshold (§2.2.3, Eq. 9) -> candidate list (r-bin, width,
power, sigma).
"""
import numpy as np

from . import boxcar, fft, normalise, significance


def n_trials_default(m, w_max):
    """Bonferroni trial count: every bin times every searched width."""
    return float(m) * float(w_max)


def candidates_from_maxima(mx, am, w_max, n_trials, sigma_thr):
    """Candidate records from per-(segment, width) maxima.

    Returns a list of dicts ordered by (segment, width), one per (s, w) whose
    maximum passes the sigma threshold.
    """
    out = []
    for w in range(1, w_max + 1):
        col = mx[:, w - 1]
        ok = ~np.isnan(col)
        if not ok.any():
            continue
        segs = np.nonzero(ok)[0]
        pw = col[segs]
        lp = significance.log_p_adjusted(w, pw, n_trials)
        keep = lp <= significance.log_sf_normal(sigma_thr)
        if not keep.any():
            continue
        sig = significance.sigma_from_log_p(lp[keep])
        for s, p, g in zip(segs[keep], pw[keep], sig):
            out.append(dict(segment=int(s), width=w, bin=int(am[s, w - 1]),
                            power=float(p), sigma=float(g)))
    out.sort(key=lambda r: (r["segment"], r["width"]))
    return out


def search_power(p, w_max, seg_len, sigma_thr, n_trials=None):
    """Boxcar search of a normalised power spectrum (FP64)."""
    m = len(p)
    if n_trials is None:
        n_trials = n_trials_default(m, w_max)
    mx, am = boxcar.segment_maxima(p, w_max, seg_len)
    return candidates_from_maxima(mx, am, w_max, n_trials, sigma_thr)


def search_series(x, w_max, seg_len, sigma_thr, n_trials=None):
    """Full search of a real time series x (length a power of two)."""
    spec = fft.rfft(x)
    p, _, _ = normalise.normalise_power(spec, seg_len)
    return search_power(p, w_max, seg_len, sigma_thr, n_trials)
