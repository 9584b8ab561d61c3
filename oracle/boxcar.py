"""Recursive boxcar bank and per-segment maxima, FP64 (test infrastructure).

§2.2.5 of the paper: with Y_1 = X, the width-k filtered array is
Y_k = Y_{k-1}[:end-1] + X[k:end] (1-based slicing), so Y_k has N-k+1 entries
and Y_k[i] = x_i + ... + x_{i+k-1}.  Widths 1..z_max are all computed (§2.2.3).
Algorithm 4 then takes, per chunk and per searched width, the maximum and its
index.

Readings (see the design notes): widths are w = 1..W (the paper's z + 1);
the reported bin is the window's first bin k; a window must lie inside the
spectrum (k <= M - w, no zero padding); segment s covers starting bins
[s L, (s+1) L) and the last segment absorbs the remainder; ties go to the
lowest bin.
"""
import numpy as np

from .normalise import block_bounds


def boxcar_widths(p, w_max):
    """Yield (w, S_w) for w = 1..w_max with S_w[k] = sum_{j<w} p[k+j]."""
    p = np.asarray(p, dtype=np.float64)
    s = p.copy()
    yield 1, s
    for w in range(2, w_max + 1):
        if s.shape[0] <= 1:
            return
        # Y_w = Y_{w-1}[:end-1] + X[w:end]  (1-based)  ->  0-based p[w-1:]
        s = s[:-1] + p[w - 1:]
        yield w, s


def segment_maxima(p, w_max, seg_len, seg_range=None):
    """Per-(segment, width) maximum of S_w over the segment's valid start bins.

    Returns (mx, am) of shape [n_seg, w_max]: mx is NaN and am is -1 where a
    segment has no valid start bin for that width.  ``seg_range=(a, b)``
    restricts the work to segments a..b-1 (rows outside stay NaN / -1); it
    only reads p[a*L : end_of_segment(b-1) + w_max - 1].
    """
    p = np.asarray(p, dtype=np.float64)
    m = p.shape[0]
    bounds = block_bounds(m, seg_len)
    n_seg = len(bounds)
    a, b = (0, n_seg) if seg_range is None else seg_range
    mx = np.full((n_seg, w_max), np.nan)
    am = np.full((n_seg, w_max), -1, dtype=np.int64)
    lo0 = bounds[a][0]
    hi0 = min(m, bounds[b - 1][1] + w_max - 1)
    sub = p[lo0:hi0]
    for w, s in boxcar_widths(sub, w_max):
        n_valid = m - w + 1          # global starting bins 0..m-w
        # segments a..f-1 are full L-bin segments with every start bin valid:
        # one argmax per row of a reshaped view (argmax returns the first,
        # i.e. lowest, index on ties)
        f = a
        while f < b and f < n_seg - 1 and bounds[f][1] <= n_valid:
            f += 1
        if f > a:
            v = s[: (f - a) * seg_len].reshape(f - a, seg_len)
            k = np.argmax(v, axis=1)
            mx[a:f, w - 1] = v[np.arange(f - a), k]
            am[a:f, w - 1] = lo0 + np.arange(f - a) * seg_len + k
        for seg in range(f, b):
            lo, hi = bounds[seg]
            hi = min(hi, n_valid)
            if lo >= hi:
                continue
            v = s[lo - lo0: hi - lo0]
            k = int(np.argmax(v))
            mx[seg, w - 1] = v[k]
            am[seg, w - 1] = lo + k
    return mx, am


def boxcar_direct(p, k, w):
    """S_w[k] by direct summation (the definition, for spot checks)."""
    p = np.asarray(p, dtype=np.float64)
    return float(np.sum(p[k:k + w]))
