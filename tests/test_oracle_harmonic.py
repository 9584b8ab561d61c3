"""Pins of the harmonic-sum oracle (§2.3 and its GPU decimation listing)."""
import numpy as np
import pytest
from scipy import stats

from oracle import harmonic, pipeline


def test_brute_force_double_loop():
    rng = np.random.default_rng(1)
    p = rng.random(103)
    for H in range(1, 6):
        m = 103 // H
        ref = np.zeros(m)
        for r in range(m):
            for h in range(1, H + 1):
                for j in range(h):
                    ref[r] += p[h * r + j]
        assert np.allclose(harmonic.harmonic_sum(p, H), ref, rtol=1e-14, atol=0)


def test_listing_terms_on_a_ramp():
    """P[i] = i: X_H[r] = r sum_h h^2 + sum_h h(h-1)/2 (each h-group at h r adds
    h^2 r + h(h-1)/2), e.g. X_2[t] = t + 2t + 2t + 1 as in the listing."""
    p = np.arange(1000, dtype=np.float64)
    for H in (1, 2, 3, 4, 8):
        r = np.arange(1000 // H)
        sh2 = sum(h * h for h in range(1, H + 1))
        c = sum(h * (h - 1) // 2 for h in range(1, H + 1))
        assert np.array_equal(harmonic.harmonic_sum(p, H), r * sh2 + c)
    t = np.arange(500)
    assert np.array_equal(harmonic.harmonic_sum(p, 2), t + 2 * t + (2 * t + 1))


def test_noise_is_chi2_with_H_H_plus_1_dof():
    """§2.3: X_H ~ chi^2(H(H+1)) for Gaussian input, i.e. 2 X_H with P ~ Exp(1)."""
    rng = np.random.default_rng(2)
    p = rng.exponential(1.0, 1 << 18)
    for H in (2, 3, 4):
        x = harmonic.harmonic_sum(p, H)
        k = H * (H + 1)
        assert abs(x.mean() - k / 2) < 5 * np.sqrt(k / 2 / x.size)
        assert stats.kstest(2 * x, stats.chi2(k).cdf).pvalue > 1e-3
        assert harmonic.shape_per_width(H) * 2 == k


def test_harmonics_of_a_pulse_train_add_up():
    """Power A at bins h f (h = 1..4) -- the first bin of each h-group at r = f --
    all lands in X_4[f]."""
    p = np.zeros(4096)
    f = 300
    for h in range(1, 5):
        p[h * f] = 10.0
    assert harmonic.harmonic_sum(p, 4)[f] == 40.0
    assert harmonic.harmonic_sum(p, 2)[f] == 20.0
    assert harmonic.harmonic_sum(p, 4)[f + 1] == 0.0


def test_stage_one_is_the_plain_search():
    rng = np.random.default_rng(3)
    p = rng.exponential(1.0, 1 << 13)
    p[2000:2030] += 1.5
    a = pipeline.search_power(p, 32, 256, 2.0)
    b = harmonic.search_harmonics(p, 32, 256, 2.0, numharm=1)
    assert [dict(r, harmonics=1) for r in a] == b


def test_stage_thresholds_use_the_stage_shape():
    """A stage-H width-w sum has gamma shape H(H+1)/2 w: with a constant
    spectrum every stage maximum is exactly its expectation."""
    p = np.ones(1 << 12)
    recs = harmonic.search_harmonics(p, 8, 256, 0.0, numharm=3, n_trials=1.0)
    for r in recs:
        assert r["power"] == pytest.approx(harmonic.shape_per_width(r["harmonics"]) * r["width"])
