"""End-to-end boxcar search in the paper's order, FP64 (test infrastructure).

FFT (own radix-2) -> per-block median/MAD normalisation and power (§2.2.3,
Eq. 8) -> boxcar bank for widths 1..W (§2.2.5) -> per-(segment, width)
maximum (Algorithm 4) -> chi-square significance with Bonferroni correction
and a sigma threshold (§2.2.3, Eq. 9) -> candidate list (r-bin, width,
power, sigma).
"""
import numpy as np

from . import boxcar, fft, normalise, significance


def searched_widths(w_max, mode="all", step=1):
    """Widths compared with the threshold (all widths are still summed).

    §2.2.3 lets the user pick the step of the searched widths (Algorithm 4
    tests z mod z_step = 0) and §4.1.4 searches logarithmically spaced
    z = 1, 2, 4, 8, ... only; with z = w - 1: "all" -> 1..W, "step" -> w with
    (w - 1) mod step == 0, "log2" -> w with w - 1 a power of two."""
    ws = []
    for w in range(1, w_max + 1):
        z = w - 1
        if mode == "all":
            ok = True
        elif mode == "step":
            ok = z % step == 0
        elif mode == "log2":
            ok = z > 0 and (z & (z - 1)) == 0
        else:
            raise ValueError(mode)
        if ok:
            ws.append(w)
    return ws


def n_trials_default(m, w_max, widths=None):
    """Bonferroni trial count: every bin times every searched width."""
    return float(m) * float(w_max if widths is None else len(widths))


def candidates_from_maxima(mx, am, w_max, n_trials, sigma_thr, widths=None, rblock=0, shape_mult=1):
    """Candidate records from per-(segment, width) maxima.

    Returns a list of dicts ordered by (segment, width), one per (s, w) with w
    searched whose maximum passes the sigma threshold.  rblock > 0 reports the
    block index bin // rblock instead of the bin (§2.4, "R-Block").
    shape_mult: gamma shape per unit width of the searched spectrum (1 for the
    power; H(H+1)/2 for an H-harmonic sum, §2.3).
    """
    out = []
    for w in (range(1, w_max + 1) if widths is None else widths):
        col = mx[:, w - 1]
        ok = ~np.isnan(col)
        if not ok.any():
            continue
        segs = np.nonzero(ok)[0]
        pw = col[segs]
        lp = significance.log_p_adjusted(shape_mult * w, pw, n_trials)
        keep = lp <= significance.log_sf_normal(sigma_thr)
        if not keep.any():
            continue
        sig = significance.sigma_from_log_p(lp[keep])
        for s, p, g in zip(segs[keep], pw[keep], sig):
            b = int(am[s, w - 1])
            out.append(dict(segment=int(s), width=w, bin=b // rblock if rblock else b,
                            power=float(p), sigma=float(g)))
    out.sort(key=lambda r: (r["segment"], r["width"]))
    return out


def search_power(p, w_max, seg_len, sigma_thr, n_trials=None, widths=None, rblock=0):
    """Boxcar search of a normalised power spectrum (FP64)."""
    m = len(p)
    if n_trials is None:
        n_trials = n_trials_default(m, w_max, widths)
    mx, am = boxcar.segment_maxima(p, w_max, seg_len)
    return candidates_from_maxima(mx, am, w_max, n_trials, sigma_thr, widths, rblock)


def search_series(x, w_max, seg_len, sigma_thr, n_trials=None, widths=None, rblock=0):
    """Full search of a real time series x (length a power of two)."""
    spec = fft.rfft(x)
    p, _, _ = normalise.normalise_power(spec, seg_len)
    return search_power(p, w_max, seg_len, sigma_thr, n_trials, widths, rblock)
