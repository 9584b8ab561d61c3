"""The seeded input generator (CPU): noise statistics and reproducibility,
and the chirp convention -- the instantaneous frequency starts at Fourier
bin r0 and drifts by z bins over the observation (plus w/2 from the jerk
term) -- checked through where the signal's power lands in the spectrum."""
import numpy as np
import pytest

from paper_2406_15186_gb300 import synth


def test_noise_is_seeded_unit_gaussian_float32():
    a, b, c = synth.noise(1 << 16, 7), synth.noise(1 << 16, 7), synth.noise(1 << 16, 8)
    assert a.dtype == np.float32 and np.array_equal(a, b) and not np.array_equal(a, c)
    assert abs(float(a.mean())) < 0.02 and abs(float(a.std()) - 1.0) < 0.02


def test_pure_tone_lands_in_its_bin():
    n, r0 = 1 << 14, 1234
    x = synth.chirp(n, r0, 0.0)
    spec = np.abs(np.fft.rfft(x))
    assert int(np.argmax(spec)) == r0
    assert spec[r0] == pytest.approx(n / 2, rel=1e-9)


@pytest.mark.parametrize("z,w", [(40.0, 0.0), (200.0, 0.0), (60.0, 80.0)])
def test_drift_spreads_power_from_r0_over_z_bins(z, w):
    n, r0 = 1 << 16, 5000
    x = synth.chirp(n, r0, z, w)
    p = np.abs(np.fft.rfft(x)) ** 2
    f_end = r0 + z + w / 2.0                 # instantaneous frequency at the end
    k = np.arange(p.shape[0])
    band = (k >= r0 - 3) & (k <= f_end + 3)
    assert p[band].sum() >= 0.95 * p.sum()
    # the mean frequency over the observation: r0 + z/2 + w/6
    centroid = float((k * p).sum() / p.sum())
    assert centroid == pytest.approx(r0 + z / 2.0 + w / 6.0, abs=1.0)


def test_inject_keeps_float32_and_zero_amplitude_is_identity():
    x = synth.noise(4096, 3)
    y = synth.inject(x, [dict(amp=0.0, r0=100.0, z=5.0)])
    assert y.dtype == np.float32 and np.array_equal(x, y)
    y2 = synth.inject(x, [dict(amp=0.5, r0=100.0, z=0.0)])
    assert y2.dtype == np.float32 and not np.array_equal(x, y2)


def test_workload_sizes():
    w = synth.WORKLOADS
    assert (w["single_2p20"]["n"], w["single_2p20"]["z_max"], w["single_2p20"]["segment_len"]) == (1 << 20, 256, 1024)
    assert (w["single_2p23"]["n"], w["single_2p23"]["z_max"], w["single_2p23"]["segment_len"]) == (1 << 23, 1024, 4096)
    assert (w["batch_512"]["n_series"], w["batch_512"]["z_max"], w["batch_512"]["segment_len"]) == (512, 512, 2048)
    assert (w["diff_4096"]["n_series"], w["diff_4096"]["n"], w["diff_4096"]["tau"]) == (4096, 1 << 20, 0.1)
    assert (w["single_2p27"]["n"], w["single_2p27"]["z_max"], w["single_2p27"]["sigma"]) == (1 << 27, 4096, 7.0)


def test_prefix_draw_is_the_prefix_of_the_whole_series():
    x, _ = synth.single_series("single_2p20")
    assert np.array_equal(synth.single_series_prefix("single_2p20", 1 << 12), x[: 1 << 12])
