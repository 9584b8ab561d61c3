"""Harmonic summing by decimation (§2.3), FP64 (test infrastructure).

The normalised power P (M bins, chi^2_2 / 2 per bin for noise) is decimated
by h -- adjacent non-overlapping groups of h bins summed, so the h-th
harmonic of a signal at bin r lands in bin r -- and the decimated spectra
for h = 1..H are added aligned at bin 0, keeping the overlap:

    X_H[r] = sum_{h=1}^{H} sum_{j=0}^{h-1} P[h r + j],   r = 0 .. floor(M/H) - 1.

For noise X_H is chi^2 with sum_{h<=H} 2h = H(H+1) degrees of freedom (a sum
of H(H+1)/2 unit exponentials), and a width-w boxcar of X_H has H(H+1) w;
each X_H is then searched exactly like P (§2.3: "proceed to boxcar filter
this input as previously described").
"""
import numpy as np

from . import boxcar, pipeline


def decimate(p, h):
    """Sum of adjacent non-overlapping groups of h bins (floor(M/h) outputs)."""
    p = np.asarray(p, dtype=np.float64)
    m = p.shape[0] // h
    return p[: m * h].reshape(m, h).sum(axis=1)


def harmonic_sum(p, n_harm):
    """X_H for H = n_harm: the decimated spectra for h = 1..H added, aligned at bin 0."""
    m = np.asarray(p).shape[0] // n_harm
    return sum(decimate(p, h)[:m] for h in range(1, n_harm + 1))


def shape_per_width(n_harm):
    """Gamma shape of X_H per unit boxcar width: H(H+1)/2."""
    return n_harm * (n_harm + 1) // 2


def search_harmonics(p, w_max, seg_len, sigma_thr, numharm, widths=None, n_trials=None):
    """Candidates of every stage H = 1..numharm (records carry 'harmonics').

    Each stage gets its own Bonferroni count floor(M/H) x (searched widths)
    unless n_trials is given."""
    out = []
    for h in range(1, numharm + 1):
        x = harmonic_sum(p, h)
        nt = pipeline.n_trials_default(x.shape[0], w_max, widths) if n_trials is None else n_trials
        mx, am = boxcar.segment_maxima(x, w_max, seg_len)
        recs = pipeline.candidates_from_maxima(mx, am, w_max, nt, sigma_thr, widths, shape_mult=shape_per_width(h))
        for r in recs:
            r["harmonics"] = h
        out += recs
    return out
