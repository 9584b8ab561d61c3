"""Pins for the oracle's boxcar bank and segment search (paper §2.2.5, Algorithm 4)."""
import numpy as np
import pytest

from oracle import boxcar, normalise


def _read_example(golden_dir):
    rows = {}
    for line in open(f"{golden_dir}/boxcar_recursion_example.txt"):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        rows[k] = np.array([float(t) for t in v])
    return rows


def test_paper_worked_example(golden_dir):
    g = _read_example(golden_dir)
    x = g["X"]
    got = dict(boxcar.boxcar_widths(x, 3))
    n = len(x)
    for w in (1, 2, 3):
        assert got[w].shape == (n - w + 1,)          # lengths N, N-1, N-2
        assert np.array_equal(got[w], g[f"Y{w}"])
    # Y_3 = Y_2[:end-1] + X[3:end] (1-based)
    assert np.array_equal(got[3], got[2][:-1] + x[2:])


def test_matches_direct_double_loop():
    rng = np.random.default_rng(4)
    p = rng.exponential(size=37)
    for w, s in boxcar.boxcar_widths(p, 12):
        ref = np.array([sum(p[k + j] for j in range(w)) for k in range(len(p) - w + 1)])
        assert np.allclose(s, ref, rtol=1e-13)


def test_closed_forms():
    c = 2.5
    for w, s in boxcar.boxcar_widths(np.full(50, c), 20):
        assert np.allclose(s, w * c)
    k = np.arange(60, dtype=float)
    for w, s in boxcar.boxcar_widths(k, 25):
        kk = np.arange(len(s))
        assert np.array_equal(s, w * kk + w * (w - 1) / 2)


def _brute_force(p, w_max, seg_len):
    m = len(p)
    bounds = normalise.block_bounds(m, seg_len)
    mx = np.full((len(bounds), w_max), np.nan)
    am = np.full((len(bounds), w_max), -1)
    for si, (lo, hi) in enumerate(bounds):
        for w in range(1, w_max + 1):
            best, arg = None, -1
            for k in range(lo, hi):
                if k + w > m:
                    continue
                v = sum(p[k:k + w])
                if best is None or v > best:
                    best, arg = v, k
            if best is not None:
                mx[si, w - 1], am[si, w - 1] = best, arg
    return mx, am


@pytest.mark.parametrize("m,w_max,seg_len", [(16, 4, 4), (33, 8, 8), (64, 8, 10), (20, 7, 7), (9, 3, 9)])
def test_segment_maxima_brute_force(m, w_max, seg_len):
    rng = np.random.default_rng(m * 100 + w_max)
    p = rng.exponential(size=m)
    mx, am = boxcar.segment_maxima(p, w_max, seg_len)
    rmx, ram = _brute_force(p, w_max, seg_len)
    assert np.array_equal(np.isnan(mx), np.isnan(rmx))
    ok = ~np.isnan(rmx)
    assert np.allclose(mx[ok], rmx[ok], rtol=1e-13)
    assert np.array_equal(am, ram)


def test_ties_go_to_lowest_bin_and_segment_range():
    p = np.zeros(40)
    p[5] = p[9] = 3.0
    mx, am = boxcar.segment_maxima(p, 2, 20)
    assert am[0, 0] == 5 and mx[0, 0] == 3.0
    full_mx, full_am = boxcar.segment_maxima(np.random.default_rng(2).exponential(size=200), 6, 30)
    part_mx, part_am = boxcar.segment_maxima(np.random.default_rng(2).exponential(size=200), 6, 30, seg_range=(2, 5))
    assert np.array_equal(part_am[2:5], full_am[2:5])
    assert np.all(part_am[:2] == -1) and np.all(part_am[5:] == -1)
    assert np.allclose(part_mx[2:5], full_mx[2:5], rtol=1e-13)


def test_window_never_runs_past_the_end():
    # the last segment's late start bins are invalid for wide windows
    p = np.arange(12, dtype=float)
    mx, am = boxcar.segment_maxima(p, 5, 4)
    for w in range(1, 5):
        assert am[2, w - 1] == 12 - w          # rightmost valid start wins (increasing p)
        assert mx[2, w - 1] == sum(range(12 - w, 12))
    # width 5: segment 2 = [8, 12) has no valid start (k <= 7); segment 1 ends at 7
    assert am[2, 4] == -1 and np.isnan(mx[2, 4])
    assert am[1, 4] == 7
