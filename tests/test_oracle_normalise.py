"""Pins for the oracle's median/MAD normalisation (paper §2.2.3, Eq. 8)."""
import math

import numpy as np
import pytest
from scipy import stats as sps

from oracle import normalise


def _golden(golden_dir, name):
    vals = {}
    for line in open(f"{golden_dir}/{name}"):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


def test_median_and_mad_hand_arrays():
    assert normalise.median([3.0, 1.0, 2.0]) == 2.0
    assert normalise.median([4.0, 1.0, 3.0, 2.0]) == 2.5
    assert normalise.median([5.0]) == 5.0
    # |x - 3| = [2, 1, 0, 1, 97] -> median 1
    assert normalise.mad([1.0, 2.0, 3.0, 4.0, 100.0], 3.0) == 1.0
    # even count: |x - 2.5| = [1.5, .5, .5, 1.5] -> (0.5 + 1.5) / 2
    assert normalise.mad([1.0, 2.0, 3.0, 4.0], 2.5) == 1.0


def test_kappa_against_paper(golden_dir):
    g = _golden(golden_dir, "kappa.txt")
    assert normalise.KAPPA == pytest.approx(g["exact"], rel=1e-15)
    assert abs(normalise.KAPPA - g["paper_rounded"]) < 5e-5
    # Phi(1/kappa) = 3/4 by the error function
    assert 0.5 * (1 + math.erf(1 / normalise.KAPPA / math.sqrt(2))) == pytest.approx(0.75, abs=1e-15)


def test_block_bounds_last_block_absorbs_remainder():
    assert normalise.block_bounds(10, 4) == [(0, 4), (4, 10)]
    assert normalise.block_bounds(8, 4) == [(0, 4), (4, 8)]
    assert normalise.block_bounds(3, 4) == [(0, 3)]
    assert normalise.block_bounds(524289, 1024)[-1] == (523264, 524289)


def test_normalised_block_is_standardised():
    # a block of values whose median and MAD are known in closed form
    re = np.array([0.0, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0, 8.0])      # med 4, MAD 2
    im = np.array([10.0, 12.0, 14.0, 16.0, 18.0, 20.0, 22.0, 24.0, 26.0])  # med 18, MAD 4
    spec = np.concatenate([[123.0 + 45.0j], re + 1j * im])   # DC is zeroed
    p, st, fl = normalise.normalise_power(spec, 10)
    assert not fl.any()
    # block = [0+0i (zeroed DC), re + i im]
    allre = np.concatenate([[0.0], re])
    allim = np.concatenate([[0.0], im])
    mr, mi = np.median(allre), np.median(allim)
    dr, di = np.median(np.abs(allre - mr)), np.median(np.abs(allim - mi))
    assert tuple(st[0]) == pytest.approx((mr, dr, mi, di))
    a = (allre - mr) / (dr * normalise.KAPPA)
    b = (allim - mi) / (di * normalise.KAPPA)
    assert np.allclose(p, 0.5 * (a * a + b * b), rtol=1e-14)


def test_scale_and_shift_invariance():
    rng = np.random.default_rng(1)
    spec = rng.standard_normal(4097) + 1j * rng.standard_normal(4097)
    p1, _, _ = normalise.normalise_power(spec, 512)
    p2, _, _ = normalise.normalise_power(3.5 * spec, 512)
    assert np.allclose(p1, p2, rtol=1e-10)
    # a shift moves every bin but the zeroed DC one, so only blocks > 0 are invariant
    p3, _, _ = normalise.normalise_power(3.5 * spec + (2.0 - 7.0j), 512)
    assert np.allclose(p1[512:], p3[512:], rtol=1e-10)


def test_zero_mad_block_flagged():
    spec = np.ones(64, dtype=complex)
    rng = np.random.default_rng(0)
    spec[40:] = rng.standard_normal(24) + 1j * rng.standard_normal(24)
    p, _, fl = normalise.normalise_power(spec, 32)
    assert fl[0] and not fl[1]
    assert np.all(p[:32] == 0.0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_noise_power_is_exponential(seed):
    # Gaussian noise spectrum: P ~ Exp(1) (mean 1, median ln 2) up to the
    # small-sample bias of the median/MAD estimates
    rng = np.random.default_rng(seed)
    m = 1 << 18
    spec = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    p, _, _ = normalise.normalise_power(spec, 8192)
    assert np.mean(p) == pytest.approx(1.0, rel=0.01)
    assert np.median(p) == pytest.approx(math.log(2.0), rel=0.01)
    assert sps.kstest(p[1:], "expon").pvalue > 1e-4
