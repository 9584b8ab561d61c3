"""Pins for the oracle's own radix-2 FFT (not the GPU path)."""
import numpy as np
import pytest

from oracle import fft


def _dft_matrix(n):
    # X_k = sum_n x_n exp(-2 pi i k n / N); k*n reduced mod N in integers
    kn = np.outer(np.arange(n), np.arange(n)) % n
    return np.exp(-2j * np.pi * kn / n)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64, 256, 1024])
def test_fft_equals_direct_dft(n):
    rng = np.random.default_rng(n)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = _dft_matrix(n) @ z
    got = fft.fft_radix2(z)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [2, 8, 1024, 1 << 14])
def test_rfft_parseval(n):
    x = np.random.default_rng(7 + n).standard_normal(n)
    X = fft.rfft(x)
    assert X.shape == (n // 2 + 1,)
    e_spec = (abs(X[0]) ** 2 + 2 * np.sum(abs(X[1:n // 2]) ** 2) + abs(X[n // 2]) ** 2) / n
    assert e_spec == pytest.approx(np.sum(x * x), rel=1e-12)


def test_integer_bin_tone_and_delta():
    n, r, a = 4096, 317, 0.25
    x = a * np.cos(2 * np.pi * r * np.arange(n) / n)
    X = fft.rfft(x)
    assert abs(X[r]) == pytest.approx(a * n / 2, rel=1e-12)
    others = np.delete(np.abs(X), r)
    assert others.max() < 1e-9
    d = np.zeros(n)
    d[0] = 1.0
    assert np.allclose(fft.rfft(d), 1.0, atol=1e-14)


def test_matches_library_fft():
    x = np.random.default_rng(3).standard_normal(1 << 16)
    assert np.max(np.abs(fft.rfft(x) - np.fft.rfft(x))) < 1e-9


def test_dft_bins_matches_fft():
    x = np.random.default_rng(5).standard_normal(2048)
    bins = [0, 1, 17, 1023, 1024]
    assert np.max(np.abs(fft.dft_bins(x, bins) - fft.rfft(x)[bins])) < 1e-9


@pytest.mark.parametrize("n", [8, 64, 4096])
def test_rfft_adjoint_dot_product(n):
    # <rfft(x), g> = <x, rfft_adjoint(g)> with the real inner product
    rng = np.random.default_rng(11 + n)
    x = rng.standard_normal(n)
    gr, gi = rng.standard_normal(n // 2 + 1), rng.standard_normal(n // 2 + 1)
    X = fft.rfft(x)
    lhs = np.sum(gr * X.real + gi * X.imag)
    rhs = np.sum(x * fft.rfft_adjoint(gr, gi, n))
    assert lhs == pytest.approx(rhs, rel=1e-11, abs=1e-9)


def test_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        fft.fft_radix2(np.zeros(12))
