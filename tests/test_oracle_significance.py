"""Pins for the oracle's chi-square significance and sigma (paper §2.2.3, Eq. 9)."""
import math

import numpy as np
import pytest
from scipy import special

from oracle import significance as sig


def test_width_one_is_exponential_tail():
    s = np.array([0.0, 0.1, 1.0, 10.0, 700.0, 5000.0])
    assert np.allclose(sig.log_q(1, s), -s, rtol=1e-14, atol=1e-300)


@pytest.mark.parametrize("w", [1, 2, 5, 64, 256, 1024])
def test_matches_library_incomplete_gamma(w):
    s = np.linspace(0.05, 3.0, 11) * w
    ref = special.gammaincc(w, s)
    ok = ref > 1e-300
    assert np.allclose(np.exp(sig.log_q(w, s[ok])), ref[ok], rtol=1e-10)


def test_log_q_is_monotone_and_zero_at_origin():
    assert sig.log_q(7, 0.0)[0] == 0.0
    v = sig.log_q(33, np.linspace(0, 400, 200))
    assert np.all(np.diff(v) <= 0)
    assert np.all(np.diff(v[v < -1e-3]) < 0)


def test_chi_square_reading_by_monte_carlo():
    # 2 S ~ chi^2(2w) for S a sum of w Exp(1): empirical survival vs Q(w, s)
    rng = np.random.default_rng(0)
    w = 16
    s = rng.exponential(size=(200000, w)).sum(axis=1)
    for q in (20.0, 25.0, 30.0):
        emp = np.mean(s >= q)
        assert emp == pytest.approx(math.exp(sig.log_q(w, q)[0]), rel=0.05)


def test_sigma_against_normal_table(golden_dir):
    for line in open(f"{golden_dir}/gaussian_tail.txt"):
        if line.startswith("#") or not line.strip():
            continue
        s, p = (float(t) for t in line.split())
        assert sig.sigma_from_log_p(math.log(p))[0] == pytest.approx(s, abs=1e-9)
        assert float(sig.log_sf_normal(s)) == pytest.approx(math.log(p), rel=1e-12)


def test_sigma_deep_tail():
    # far below FP64 underflow the inversion still satisfies ln Phi_c(sigma) = lp
    for lp in (-800.0, -5000.0, -1.0e5):
        s = sig.sigma_from_log_p(lp)[0]
        assert float(sig.log_sf_normal(s)) == pytest.approx(lp, rel=1e-10)
        # Mills-ratio asymptote: ln Phi_c(s) ~ -s^2/2 - ln(s sqrt(2 pi))
        assert -s * s / 2 - math.log(s * math.sqrt(2 * math.pi)) == pytest.approx(lp, rel=1e-3)


def test_bonferroni_and_threshold():
    w, n_trials = 10, 4.0e9
    t = sig.threshold_power(w, 6.0, n_trials)
    assert sig.passes(w, t * (1 + 1e-9), n_trials, 6.0)[0]
    assert not sig.passes(w, t * (1 - 1e-9), n_trials, 6.0)[0]
    assert sig.sigma_of(w, t, n_trials)[0] == pytest.approx(6.0, abs=1e-6)
    # one trial: no correction
    assert sig.log_p_adjusted(w, 30.0, 1.0)[0] == pytest.approx(sig.log_q(w, 30.0)[0])
    # the correction saturates at p = 1
    assert sig.log_p_adjusted(w, 1.0, n_trials)[0] == 0.0


def test_width_one_threshold_closed_form():
    # Q(1, T) = exp(-T) = Phi_c(sigma) / n_trials  ->  T = ln(n_trials / Phi_c(sigma))
    n_trials = 524289.0 * 256
    t = sig.threshold_power(1, 6.0, n_trials)
    assert t == pytest.approx(math.log(n_trials / 9.865876450376946e-10), rel=1e-12)
