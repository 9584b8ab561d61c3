"""End-to-end sanity of the oracle search on the 2^20-sample workload recipe."""
import numpy as np
import pytest

from oracle import pipeline
from paper_2406_15186_gb300 import synth


def test_injected_tone_is_found():
    x, tones = synth.single_series("single_2p20")
    t = tones[0]
    cands = pipeline.search_series(x, 256, 1024, 6.0)
    best = max(cands, key=lambda r: r["sigma"])
    # the drifting tone occupies bins r0..r0+z; a window of width w covering it
    # starts between r0 - w and r0 + z
    assert t["r0"] - 256 <= best["bin"] <= t["r0"] + t["z"]
    assert best["sigma"] > 20.0
    # widths near the drift (z = 50) are the most significant ones
    assert 30 <= best["width"] <= 80


def test_pure_noise_gives_no_candidates_at_six_sigma():
    x = synth.noise(1 << 16, 12345)
    assert pipeline.search_series(x, 64, 1024, 6.0) == []


def test_low_threshold_emits_every_segment_width():
    x = synth.noise(1 << 12, 7)
    c = pipeline.search_series(x, 8, 256, 0.0, n_trials=1.0)
    # with sigma_thr = 0 and no trial correction, every max with p <= 1/2 passes
    assert len(c) > 0
    assert all(r["sigma"] >= 0.0 for r in c)
    keys = [(r["segment"], r["width"]) for r in c]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)


def test_searched_widths_examples():
    """§2.2.3 / Algorithm 4 (z mod z_step = 0) and §4.1.4 (z = 1, 2, 4, ...), z = w - 1."""
    assert pipeline.searched_widths(10, "all") == list(range(1, 11))
    assert pipeline.searched_widths(10, "step", 3) == [1, 4, 7, 10]
    assert pipeline.searched_widths(10, "step", 1) == list(range(1, 11))
    assert pipeline.searched_widths(10, "log2") == [2, 3, 5, 9]
    assert pipeline.searched_widths(1025, "log2") == [2, 3, 5, 9, 17, 33, 65, 129, 257, 513, 1025]
    assert pipeline.n_trials_default(1000, 10, [2, 3, 5, 9]) == 4000.0


def test_width_subset_is_a_filter_of_the_full_search():
    """With the trial count held fixed, searching a subset of widths reports
    exactly the full search's records at those widths."""
    rng = np.random.default_rng(3)
    p = rng.exponential(1.0, 1 << 13)
    p[3000:3040] += 2.0
    full = pipeline.search_power(p, 40, 256, 1.0, n_trials=1.0)
    for ws in (pipeline.searched_widths(40, "step", 4), pipeline.searched_widths(40, "log2")):
        sub = pipeline.search_power(p, 40, 256, 1.0, n_trials=1.0, widths=ws)
        assert sub == [r for r in full if r["width"] in ws]
        assert len(sub) > 0


def test_rblock_reports_block_indices():
    """§2.4: R-Block keeps the block index of each candidate, not its bin."""
    rng = np.random.default_rng(4)
    p = rng.exponential(1.0, 1 << 12)
    exact = pipeline.search_power(p, 16, 128, 1.0, n_trials=1.0)
    block = pipeline.search_power(p, 16, 128, 1.0, n_trials=1.0, rblock=100)
    assert len(exact) == len(block) > 0
    for a, b in zip(exact, block):
        assert b["bin"] == a["bin"] // 100
        assert {k: v for k, v in a.items() if k != "bin"} == {k: v for k, v in b.items() if k != "bin"}


def test_smoke_case_gives_candidates_clear_of_the_threshold():
    """The smoke run compares GPU candidates with the oracle's: its input must
    give candidates, most of them far above the threshold (CPU, FP64 FFT)."""
    import __graft_entry__ as ge
    from oracle import fft as offt
    from oracle import normalise as onorm
    x, n, w_max, seg_len, sigma = ge.smoke_input()
    p, _, flags = onorm.normalise_power(offt.rfft(np.asarray(x, dtype=np.float64)), seg_len)
    assert not flags.any()
    ref = pipeline.search_power(p, w_max, seg_len, sigma)
    assert len(ref) >= 20
    assert max(r["sigma"] for r in ref) > 2 * sigma
