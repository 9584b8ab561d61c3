"""The library's host-side threshold (pulscan_threshold_power: bisection on
its own FP64 ln Q, rounded up to FP32) against the oracle's threshold
(oracle/significance.py, written independently), on the CPU: no plan and no
CUDA call are involved.  T_w is the smallest float whose Bonferroni-corrected
significance reaches sigma_thr (Eq. 9), so it must be the FP32 round-up of
the oracle's FP64 threshold."""
import numpy as np
import pytest

from oracle import significance as osig


@pytest.fixture(scope="module")
def pkg():
    from paper_2406_15186_gb300 import build
    build.build()
    import paper_2406_15186_gb300 as p
    p.load()
    return p


@pytest.mark.parametrize("sigma", [0.5, 2.0, 6.0, 7.0])
@pytest.mark.parametrize("n_trials", [1.0, 1.0e6, 524289.0 * 256, 4194305.0 * 1024, 67108865.0 * 4096])
def test_threshold_is_the_fp32_round_up_of_the_oracle(pkg, sigma, n_trials):
    for shape in (1, 2, 3, 7, 33, 100, 256, 1000, 1024, 3 * 512, 4096, 10 * 1024):
        t = pkg.threshold_power(shape, n_trials, sigma)
        ref = osig.threshold_power(shape, sigma, n_trials)
        below = float(np.nextafter(np.float32(t), np.float32(0.0)))
        assert t >= ref * (1.0 - 1e-10), (shape, t, ref)
        assert below < ref * (1.0 + 1e-10), (shape, t, ref)


def test_threshold_grows_with_width_sigma_and_trials(pkg):
    ts = [pkg.threshold_power(w, 1e9, 6.0) for w in (1, 2, 4, 64, 512)]
    assert all(a < b for a, b in zip(ts, ts[1:]))
    assert pkg.threshold_power(64, 1e9, 5.0) < pkg.threshold_power(64, 1e9, 6.0)
    assert pkg.threshold_power(64, 1e6, 6.0) < pkg.threshold_power(64, 1e9, 6.0)


def test_invalid_arguments(pkg):
    for args in ((0.0, 1e6, 6.0), (-1.0, 1e6, 6.0), (5.0, 0.5, 6.0), (5.0, 1e6, -1.0),
                 (5.0, 1e6, float("nan")), (float("inf"), 1e6, 6.0)):
        with pytest.raises(pkg.PulscanError):
            pkg.threshold_power(*args)
