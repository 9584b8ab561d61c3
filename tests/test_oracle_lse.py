"""Pins for the oracle's logsumexp statistic and its hand-written adjoint."""
import numpy as np
import pytest

from oracle import boxcar, lse


def _loss(x, g, w_max, seg_len, tau):
    y, _ = lse.forward(x, w_max, seg_len, tau)
    return float(np.sum(g * y))


def test_tends_to_the_segment_maximum():
    p = np.random.default_rng(0).exponential(size=300)
    mx, _ = boxcar.segment_maxima(p, 6, 50)
    y = lse.forward_power(p, 6, 50, 1e-4)
    assert np.allclose(y, mx, atol=1e-3)
    # logsumexp is never below the max and at most tau*ln(count) above it
    y1 = lse.forward_power(p, 6, 50, 0.1)
    assert np.all(y1 >= mx - 1e-12) and np.all(y1 <= mx + 0.1 * np.log(50) + 1e-12)


def test_power_adjoint_against_finite_differences():
    rng = np.random.default_rng(1)
    p = rng.exponential(size=120)
    w_max, seg_len, tau = 5, 30, 0.5
    g = rng.standard_normal((4, w_max))
    y = lse.forward_power(p, w_max, seg_len, tau)
    dp = lse.backward_power(p, y, g, w_max, seg_len, tau)
    h = 1e-6
    for j in (0, 7, 29, 30, 64, 119):
        e = np.zeros_like(p)
        e[j] = h
        fd = (np.sum(g * lse.forward_power(p + e, w_max, seg_len, tau))
              - np.sum(g * lse.forward_power(p - e, w_max, seg_len, tau))) / (2 * h)
        assert dp[j] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_hard_max_limit_of_the_adjoint():
    # tau -> 0: the weight of (s, w) moves onto the bins of the argmax window
    p = np.random.default_rng(2).exponential(size=64)
    w_max, seg_len = 3, 32
    g = np.zeros((2, w_max))
    g[1, 2] = 1.0
    y = lse.forward_power(p, w_max, seg_len, 1e-4)
    dp = lse.backward_power(p, y, g, w_max, seg_len, 1e-4)
    _, am = boxcar.segment_maxima(p, w_max, seg_len)
    k = am[1, 2]
    ref = np.zeros_like(p)
    ref[k:k + 3] = 1.0
    assert np.allclose(dp, ref, atol=1e-6)


@pytest.mark.parametrize("seed", [3, 4])
def test_full_chain_against_finite_differences(seed):
    rng = np.random.default_rng(seed)
    n, w_max, seg_len, tau = 1 << 10, 8, 64, 0.1
    t = np.arange(n) / n
    template = np.cos(2 * np.pi * (60 * t + 0.5 * 12 * t * t))
    noise = rng.standard_normal(n)
    amp = 0.3
    x = noise + amp * template
    g = rng.standard_normal((n // 2 // seg_len, w_max))
    y, st = lse.forward(x, w_max, seg_len, tau)
    gx = lse.backward(x, st, y, g, w_max, seg_len, tau)
    h = 1e-6
    for j in rng.choice(n, size=6, replace=False):
        e = np.zeros(n)
        e[j] = h
        fd = (_loss(x + e, g, w_max, seg_len, tau) - _loss(x - e, g, w_max, seg_len, tau)) / (2 * h)
        assert gx[j] == pytest.approx(fd, rel=1e-4, abs=1e-6)
    # amplitude gradient
    ga = lse.amplitude_grad(gx, template)
    fd = (_loss(noise + (amp + h) * template, g, w_max, seg_len, tau)
          - _loss(noise + (amp - h) * template, g, w_max, seg_len, tau)) / (2 * h)
    assert ga == pytest.approx(fd, rel=1e-4, abs=1e-6)
