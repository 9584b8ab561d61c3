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
