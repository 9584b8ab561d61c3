"""Own radix-2 FFT in FP64 (test infrastructure; see ``oracle/__init__``).

The paper's input is the complex spectrum of a real time series, bins
0..N/2 (§2.2.2: the same `.fft` input as PRESTO's accelsearch).  The forward
transform here is the plain unnormalised DFT with the e^{-2 pi i k n / N}
sign, computed by the iterative Cooley-Tukey radix-2 scheme (bit-reversed
reordering, then log2 N butterfly stages).  ``dft_bins`` is the O(N) per-bin
definition, used for spot checks at sizes where a full FFT is too slow.
"""
import numpy as np


def _bit_reverse_indices(n):
    bits = n.bit_length() - 1
    idx = np.arange(n, dtype=np.int64)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft_radix2(z):
    """Unnormalised forward DFT X_k = sum_n z_n exp(-2 pi i k n / N), N = 2^m."""
    z = np.asarray(z, dtype=np.complex128)
    n = z.shape[0]
    if n < 1 or (n & (n - 1)) != 0:
        raise ValueError("radix-2 FFT needs a power-of-two length")
    a = z[_bit_reverse_indices(n)].copy()
    size = 2
    while size <= n:
        half = size // 2
        tw = np.exp(-2j * np.pi * np.arange(half) / size)
        a = a.reshape(n // size, size)
        even = a[:, :half]
        odd = a[:, half:] * tw
        a = np.concatenate([even + odd, even - odd], axis=1).reshape(n)
        size *= 2
    return a


def rfft(x):
    """Bins k = 0..N/2 of the DFT of a real series (the `.fft` spectrum)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    return fft_radix2(x.astype(np.complex128))[: n // 2 + 1]


def rfft_adjoint(g_re, g_im, n):
    """Adjoint of x -> (Re X_k, Im X_k), k = 0..N/2, for real x of length n.

    Re X_k = sum_n x_n cos(theta), Im X_k = -sum_n x_n sin(theta) with
    theta = 2 pi k n / N, so the adjoint is
    g_x[n] = sum_k g_re[k] cos(theta) - g_im[k] sin(theta)
           = Re( sum_k conj(c_k) e^{-i theta} ) with c_k = g_re[k] + i g_im[k],
    i.e. the real part of a forward FFT of conj(c) zero-padded to length n.
    """
    c = np.zeros(n, dtype=np.complex128)
    m = n // 2 + 1
    c[:m] = np.asarray(g_re, dtype=np.float64) - 1j * np.asarray(g_im, dtype=np.float64)
    return fft_radix2(c).real


def dft_bins(x, bins):
    """Direct O(N) evaluation of the DFT definition at the given bins."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    out = np.empty(len(bins), dtype=np.complex128)
    for j, k in enumerate(bins):
        # reduce k*n mod N exactly in integers before forming the angle
        ph = (np.int64(k) * np.arange(n, dtype=np.int64)) % n
        out[j] = np.sum(x * np.exp(-2j * np.pi * ph / n))
    return out
