"""Per-block median/MAD normalisation and power, FP64 (test infrastructure).

Follows §2.2.3 of the paper (Eq. 8): the spectrum is cut into blocks, and in
each block the real and the imaginary parts are normalised separately,

    a = (Re - median(Re)) / (MAD(Re) * kappa),   kappa = 1 / Phi^{-1}(3/4),

and likewise b from Im.  The power is then the squared magnitude (§2.2.3),
which under white Gaussian noise is chi-square with two degrees of freedom.

Readings taken where the paper is silent (each listed in the design notes):
* block = segment of ``L`` bins; n_blocks = max(1, M // L); the last block
  absorbs the remainder (normally the lone Nyquist bin);
* the DC bin is set to 0 + 0i before the statistics are taken;
* median of an even count = mean of the two middle order statistics;
* MAD = median(|x - median|) (the appendix listing drops the absolute value,
  which cannot be meant: a median of signed deviations is ~0);
* kappa is the exact 1/Phi^{-1}(3/4), not the rounded 1.4826 of Algorithm 1;
* P = (a^2 + b^2) / 2, so that noise power is Exp(1) (mean 1, median ln 2)
  and a width-w boxcar sum S satisfies 2 S ~ chi^2(2 w) (Eq. 9);
* a block whose MAD is 0 gets P = 0 and is flagged.
"""
import numpy as np
from scipy.special import ndtri

KAPPA = 1.0 / ndtri(0.75)


def block_bounds(m, seg_len):
    """[(lo, hi)] of the normalisation blocks / search segments over m bins."""
    if seg_len < 1:
        raise ValueError("segment length must be >= 1")
    n_seg = max(1, m // seg_len)
    bounds = [(s * seg_len, (s + 1) * seg_len) for s in range(n_seg)]
    bounds[-1] = (bounds[-1][0], m)
    return bounds


def median(v):
    """Median; for an even count the mean of the two middle order statistics."""
    v = np.sort(np.asarray(v, dtype=np.float64))
    n = v.shape[0]
    if n == 0:
        raise ValueError("median of an empty block")
    if n % 2 == 1:
        return float(v[n // 2])
    return 0.5 * (float(v[n // 2 - 1]) + float(v[n // 2]))


def mad(v, med):
    """Median absolute deviation about ``med``."""
    return median(np.abs(np.asarray(v, dtype=np.float64) - med))


def normalise_power(spec, seg_len):
    """Normalised power P (FP64), block stats and zero-MAD flags.

    spec: complex array of bins 0..M-1 (FP64 or upcast FP32).
    Returns (P, stats, flags) where stats[s] = (med_re, mad_re, med_im, mad_im).
    """
    x = np.array(spec, dtype=np.complex128)
    m = x.shape[0]
    x[0] = 0.0
    re, im = x.real.copy(), x.imag.copy()
    bounds = block_bounds(m, seg_len)
    p = np.zeros(m, dtype=np.float64)
    stats = np.zeros((len(bounds), 4), dtype=np.float64)
    flags = np.zeros(len(bounds), dtype=bool)
    for s, (lo, hi) in enumerate(bounds):
        mr = median(re[lo:hi])
        dr = mad(re[lo:hi], mr)
        mi = median(im[lo:hi])
        di = mad(im[lo:hi], mi)
        stats[s] = (mr, dr, mi, di)
        if dr == 0.0 or di == 0.0:
            flags[s] = True
            continue
        a = (re[lo:hi] - mr) / (dr * KAPPA)
        b = (im[lo:hi] - mi) / (di * KAPPA)
        p[lo:hi] = 0.5 * (a * a + b * b)
    return p, stats, flags
