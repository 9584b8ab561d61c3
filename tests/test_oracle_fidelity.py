"""Pins of the paper-GPU fidelity oracle: median of medians (§2.5, appendix
listing) and the polynomial log p (§2.6, Eqs. 10-12)."""
import os

import numpy as np
import pytest

from oracle import fidelity, significance

HERE = os.path.dirname(os.path.abspath(__file__))


def test_local_median_is_the_mean_of_the_two_middle_values():
    rng = np.random.default_rng(0)
    q = rng.standard_normal((1000, 4))
    s = np.sort(q, axis=1)
    assert np.allclose(fidelity.local_median(q[:, 0], q[:, 1], q[:, 2], q[:, 3]), 0.5 * (s[:, 1] + s[:, 2]),
                       rtol=0, atol=1e-15)


def test_median_of_medians_examples():
    # four values: the local median
    assert fidelity.median_of_medians([4.0, 1.0, 3.0, 2.0]) == 2.5
    # 0..15 in order: level 1 gives lm(0,4,8,12)=6, 7, 8, 9; level 2 gives 7.5
    assert fidelity.median_of_medians(np.arange(16.0)) == 7.5
    # groups are strided: (v[t], v[t+4], v[t+8], v[t+12]) = (x, x, -5, 9) gives
    # x for t = 0..3, then lm(1, 2, 3, 4) = 2.5
    v = np.array([1.0, 2.0, 3.0, 4.0, 1.0, 2.0, 3.0, 4.0, -5.0, -5.0, -5.0, -5.0, 9.0, 9.0, 9.0, 9.0])
    assert fidelity.median_of_medians(v) == pytest.approx(0.5 * (2.0 + 3.0))
    # and the estimate differs from the exact median (2.5) when the groups are
    # unbalanced: groups (0, 0, k, k), k = 5..8, give 2.5, 3, 3.5, 4, then 3.25
    u = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 5.0, 6.0, 7.0, 8.0, 5.0, 6.0, 7.0, 8.0])
    assert fidelity.median_of_medians(u) == 3.25 and np.median(u) == 2.5
    assert fidelity.median_of_medians(np.full(64, 3.25)) == 3.25
    with pytest.raises(ValueError):
        fidelity.median_of_medians(np.zeros(32))


def test_mom_of_gaussian_noise_is_close_to_the_median():
    """An estimator of the median: on 4^6 N(0,1) samples the MoM median is
    within 0.1 of 0 and 1.4826 x MoM(|x - med|) within 10 % of 1."""
    rng = np.random.default_rng(5)
    for _ in range(5):
        x = rng.standard_normal(4096)
        med = fidelity.median_of_medians(x)
        mad = fidelity.median_of_medians(np.abs(x - med))
        assert abs(med) < 0.1
        assert abs(fidelity.MOM_SCALE * mad - 1.0) < 0.1


def test_polynomial_constants_match_the_paper():
    vals = {}
    for ln in open(os.path.join(HERE, "golden", "logp_polynomial.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        k, v = ln.split()
        vals[k] = float(v)
    assert vals["A1"] == fidelity.A1 and vals["cutoff"] == fidelity.CUTOFF
    assert tuple(vals[f"c{i}"] for i in range(16, -1, -1)) == fidelity.POLY


def test_polynomial_tracks_the_exact_log_p_where_it_was_fitted():
    """For strong candidates of many degrees of freedom (pow >= 2 dof,
    dof >= 256) the polynomial is within 5 % of the exact ln Q; below the
    1.05 cutoff it is 0."""
    for w in (128, 256, 512, 1024):
        for r in (2.0, 3.0, 5.0, 10.0):
            s = r * w
            exact = float(significance.log_q(w, s)[0])
            poly = float(fidelity.poly_logp(2 * s, 2 * w))
            assert abs(poly - exact) <= 0.05 * abs(exact), (w, r, poly, exact)
    assert float(fidelity.poly_logp(100.0, 106.0)) == 0.0


def test_polynomial_search_on_a_strong_tone():
    rng = np.random.default_rng(6)
    p = rng.exponential(1.0, 1 << 12)
    p[1000:1008] += 40.0
    recs = fidelity.search_power_poly(p, 8, 256, 6.0, n_trials=float(p.size * 8))
    assert any(r["bin"] <= 1000 <= r["bin"] + r["width"] for r in recs)
    for r in recs:
        lp = float(fidelity.log_p_adjusted_poly(r["width"], r["power"], p.size * 8))
        assert lp <= float(significance.log_sf_normal(6.0))


def test_mom_normalisation_of_noise():
    rng = np.random.default_rng(7)
    spec = rng.standard_normal(1 << 14) + 1j * rng.standard_normal(1 << 14)
    p, st, flags = fidelity.normalise_power_mom(spec, 1024)
    assert not flags.any()
    assert abs(p.mean() - 1.0) < 0.1
    assert np.all(np.abs(st[:, [1, 3]] * fidelity.MOM_SCALE - 1.0) < 0.15)


def test_mom_last_block_uses_the_statistics_of_its_first_4k_bins():
    """Hand case of the reading taken for §2.5's median of medians: blocks of
    4 bins (4^1), M = 9, so the last block holds bins 4..8 and its fifth bin
    is normalised with the statistics of bins 4..7.  Re(4..7) = 1, 2, 3, 4:
    median lm(1, 2, 3, 4) = 2.5, deviations 1.5, 0.5, 0.5, 1.5, MAD 1.  Im(4..7)
    = 1, -1, 2, -2: median (1 + -1) / 2 = 0, deviations 1, 1, 2, 2, MAD 1.5.
    Bin 8 = 10 + 5i: a = 7.5 / 1.4826, b = 5 / (1.4826 * 1.5)."""
    spec = np.zeros(9, dtype=complex)
    spec[0:4] = [7.0 + 7.0j, 1.0 - 2.0j, -3.0 + 0.5j, 2.0 + 1.0j]
    spec[4:9] = [1.0 + 1.0j, 2.0 - 1.0j, 3.0 + 2.0j, 4.0 - 2.0j, 10.0 + 5.0j]
    p, st, flags = fidelity.normalise_power_mom(spec, 4)
    assert not flags.any() and st.shape == (2, 4)
    assert tuple(st[1]) == (2.5, 1.0, 0.0, 1.5)
    a, b = 7.5 / 1.4826, 5.0 / (1.4826 * 1.5)
    assert p[8] == pytest.approx(0.5 * (a * a + b * b), rel=1e-15)
    # bins 4..7 with the same statistics
    re, im = np.array([1.0, 2.0, 3.0, 4.0]), np.array([1.0, -1.0, 2.0, -2.0])
    want = 0.5 * (((re - 2.5) / 1.4826) ** 2 + (im / (1.4826 * 1.5)) ** 2)
    assert np.allclose(p[4:8], want, rtol=1e-15, atol=0)
    # the first block: DC taken as 0, so Re = 0, 1, -3, 2 -> lm = (0 + 1) / 2
    assert st[0, 0] == 0.5
    # had bin 8 entered the statistics, the median of Re would differ
    assert np.median(np.array([1.0, 2.0, 3.0, 4.0, 10.0])) != st[1, 0]


def test_polynomial_log_p_equals_eqs_10_to_12_by_polyval():
    """Eqs. 10-12 evaluated independently: numpy.polyval on the golden
    coefficients, x = A1 dof / pow, log p = pow f(x) / A1; zero from the
    1.05 cutoff on."""
    vals = {}
    for ln in open(os.path.join(HERE, "golden", "logp_polynomial.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        k, v = ln.split()
        vals[k] = float(v)
    coeffs = [vals[f"c{i}"] for i in range(16, -1, -1)]
    for pow_, dof in ((2048.0, 512.0), (1200.0, 200.0), (4096.0, 2048.0), (300.0, 64.0), (150.0, 140.0)):
        x = vals["A1"] * dof / pow_
        want = pow_ * np.polyval(coeffs, x) / vals["A1"]
        assert float(fidelity.poly_logp(pow_, dof)) == pytest.approx(want, rel=1e-12, abs=1e-12)
    assert float(fidelity.poly_logp(100.0, 105.0)) == 0.0           # dof = 1.05 pow: cut off
    assert float(fidelity.poly_logp(100.0, 104.9)) != 0.0
