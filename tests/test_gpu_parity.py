"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Stage A: normalisation of the GPU spectrum.  Stage B: all (segment, width)
maxima of the GPU power.  Candidates: thresholded search against the oracle's
decisions.  Stage C: end-to-end from the raw series with the oracle's own FFT.
"""
import math

import numpy as np
import pytest

from oracle import boxcar as obox
from oracle import fft as offt
from oracle import pipeline as opipe
from oracle import significance as osig
from paper_2406_15186_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2406_15186_gb300 as p
    from paper_2406_15186_gb300 import build
    build.build()
    p.load()
    return p


# (n, z_max, segment_len, sigma): several tiles, ragged tails, odd segment
# lengths (unaligned TMA sources fall back to plain loads), widths that are
# not multiples of 33, widths < 33, segment_len < 66 (lane bins span three
# segments), a single segment, a non-power-of-two length
SHAPES = [
    (1 << 16, 64, 1024, 6.0),
    (1 << 16, 100, 777, 4.0),
    (1 << 14, 5, 16, 3.0),
    (1 << 13, 40, 48, 3.0),
    (1 << 12, 33, 2049, 3.0),
    (3 * (1 << 12) + 10, 130, 1000, 3.0),
    (1 << 17, 300, 4096, 5.0),
]


def _series(n, seed=11):
    x = synth.noise(n, seed)
    tones = [dict(amp=0.2, r0=0.31 * n / 2, z=min(40.0, n / 400), w=0.0, phi0=0.3),
             dict(amp=0.1, r0=0.77 * n / 2, z=3.0, w=0.0, phi0=1.1)]
    return synth.inject(x, tones)


@pytest.mark.parametrize("packed", [0, 1])
@pytest.mark.parametrize("n,w_max,seg_len,sigma", SHAPES)
def test_stage_a_b_and_candidates(pkg, n, w_max, seg_len, sigma, packed):
    """Every shape with the scalar bank and with the packed one (two 1056-bin
    slices per warp, add.f32x2), whose dump mode then runs the slices of a
    packed tile one after the other."""
    x = _series(n)
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    if packed:
        plan.set_tiling(2, -1, 1)
    out = parity.run_gpu(plan, x, stats=True)
    m = n // 2 + 1
    spec = parity.spectrum_complex(out["spec"], 0, m)
    parity.check_normalise(spec, out["power"][:m], out["stats"], seg_len)
    p64 = out["power"][:m].astype(np.float64)
    mx_ref, am_ref = parity.check_maxima(p64, out["mx"], out["am"], w_max, seg_len)
    parity.check_candidates(out["cands"], p64, mx_ref, am_ref, w_max, seg_len, sigma,
                            parity.n_trials_of(m, w_max))


@pytest.mark.parametrize("sigma", [0.0, 2.0])
def test_low_thresholds_exercise_many_candidates(pkg, sigma):
    n, w_max, seg_len = 1 << 16, 70, 512
    x = _series(n, seed=5)
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    plan.set_trials(1.0)
    out = parity.run_gpu(plan, x)
    m = n // 2 + 1
    p64 = out["power"][:m].astype(np.float64)
    mx_ref, am_ref = parity.check_maxima(p64, out["mx"], out["am"], w_max, seg_len)
    k = parity.check_candidates(out["cands"], p64, mx_ref, am_ref, w_max, seg_len, sigma, 1.0)
    assert k > 100


def test_thresholds_match_oracle(pkg):
    n, w_max, seg_len = 1 << 20, 256, 1024
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=6.0)
    t = plan.thresholds()
    nt = parity.n_trials_of(n // 2 + 1, w_max)
    for w in (1, 2, 7, 33, 100, 255, 256):
        ref = osig.threshold_power(w, 6.0, nt)
        assert t[w - 1] >= ref * (1 - 1e-7) and t[w - 1] <= ref * (1 + 2 ** -22), (w, t[w - 1], ref)
    assert np.all(np.diff(t) > 0)
    # width 1: exp(-T) = Phi_c(6) / n_trials
    assert t[0] == pytest.approx(math.log(nt / 9.865876450376946e-10), rel=1e-6)


def test_full_single_2p20_end_to_end(pkg):
    """Stage C on the full 2^20-sample workload: oracle from the raw series."""
    cfg = synth.WORKLOADS["single_2p20"]
    n, w_max, seg_len, sigma = cfg["n"], cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    x, tones = synth.single_series("single_2p20")
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    out = parity.run_gpu(plan, x, stats=True)
    m = n // 2 + 1
    # FFT stage: relative L2 error of the FP32 cuFFT spectrum vs the FP64 radix-2 oracle
    ref_spec = offt.rfft(x.astype(np.float64))
    gspec = parity.spectrum_complex(out["spec"], 0, m)
    rel = np.linalg.norm(gspec - ref_spec) / np.linalg.norm(ref_spec)
    assert rel <= 1e-6 * math.log2(n), rel
    # stages A and B on the GPU's own intermediates
    parity.check_normalise(gspec, out["power"][:m], out["stats"], seg_len)
    p64 = out["power"][:m].astype(np.float64)
    parity.check_maxima(p64, out["mx"], out["am"], w_max, seg_len)
    # stage C: the oracle's full FP64 path from x
    from oracle import boxcar as obox
    from oracle import normalise as onorm
    p_ref, _, _ = onorm.normalise_power(ref_spec, seg_len)
    mx_ref, am_ref = obox.segment_maxima(p_ref, w_max, seg_len)
    parity.check_candidates(out["cands"], p_ref, mx_ref, am_ref, w_max, seg_len, sigma,
                            parity.n_trials_of(m, w_max))
    best = out["cands"][np.argmax(out["cands"]["sigma"])]
    assert tones[0]["r0"] - w_max <= best["bin"] <= tones[0]["r0"] + tones[0]["z"]
    ref_c = opipe.candidates_from_maxima(mx_ref, am_ref, w_max, parity.n_trials_of(m, w_max), sigma)
    assert abs(len(ref_c) - len(out["cands"])) <= 2


def test_graph_replay_matches_eager(pkg):
    n, w_max, seg_len = 1 << 16, 64, 1024
    x = _series(n, seed=3)
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=3.0)
    eager = parity.run_gpu(plan, x, maxima=False)
    graph = parity.run_gpu(plan, x, maxima=False, use_graph=True)
    assert np.array_equal(eager["power"], graph["power"])
    a = np.sort(eager["cands"], order=["series", "bin", "width"])
    b = np.sort(graph["cands"], order=["series", "bin", "width"])
    assert np.array_equal(a, b)


def test_batch_uneven_lengths(pkg):
    lengths = [1 << 13, 1 << 15, 1 << 12, 1 << 14, 1 << 13, 6000]
    w_max, seg_len, sigma = 48, 256, 3.0
    xs = [_series(n, seed=100 + i) for i, n in enumerate(lengths)]
    plan = pkg.Plan(lengths=lengths, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    xo, so, po, go = plan.offsets()
    x_all = np.zeros(plan.x_floats, dtype=np.float32)
    for i, x in enumerate(xs):
        x_all[xo[i]: xo[i] + len(x)] = x
    out = parity.run_gpu(plan, x_all, stats=True)
    for i, n in enumerate(lengths):
        m = n // 2 + 1
        spec = parity.spectrum_complex(out["spec"], so[i], m)
        p = out["power"][po[i]: po[i] + m]
        st = out["stats"][go[i]: go[i] + max(1, m // seg_len)]
        parity.check_normalise(spec, p, st, seg_len)
        p64 = p.astype(np.float64)
        rows = slice(go[i], go[i] + max(1, m // seg_len))
        mx_ref, am_ref = parity.check_maxima(p64, out["mx"][rows], out["am"][rows], w_max, seg_len)
        parity.check_candidates(out["cands"], p64, mx_ref, am_ref, w_max, seg_len, sigma,
                                parity.n_trials_of(m, w_max), series=i)


def test_batch_pipelined_graph_matches_oracle_and_sequential(pkg):
    """The captured batch search, pipelined over parts of a few series (each
    part's transform and normalisation on the side stream, its bank after
    them), gives the oracle's maxima and candidates and exactly the records of
    the stages run one after another."""
    lengths = [1 << 13, 1 << 15, 1 << 12, 1 << 14, 1 << 13, 6000, 1 << 15, 1 << 14, 1 << 12]
    w_max, seg_len, sigma = 40, 512, 3.0
    xs = [_series(n, seed=300 + i) for i, n in enumerate(lengths)]
    plan = pkg.Plan(lengths=lengths, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    plan.set_pipeline(10000)
    assert plan.pipeline_parts() >= 6
    xo, so, po, go = plan.offsets()
    x_all = np.zeros(plan.x_floats, dtype=np.float32)
    for i, x in enumerate(xs):
        x_all[xo[i]: xo[i] + len(x)] = x
    piped = parity.run_gpu(plan, x_all, stats=True, use_graph=True)
    seq = parity.run_gpu(plan, x_all, stats=True, use_graph=False)
    # a part's transform may round differently from the whole length class's
    for i, n in enumerate(lengths):
        m = n // 2 + 1
        a = parity.spectrum_complex(piped["spec"], so[i], m)
        b = parity.spectrum_complex(seq["spec"], so[i], m)
        assert np.linalg.norm(a - b) <= 1e-6 * np.log2(n) * np.linalg.norm(b)
    # on the same spectrum, the stages in turn give the pipelined power and records exactly
    d_spec = torch.from_numpy(piped["spec"]).cuda()
    d_power = torch.zeros(plan.power_floats, device="cuda")
    plan.power_normalise(d_spec, d_power)
    plan.boxcar_search(d_power)
    again = plan.candidates()
    assert np.array_equal(d_power.cpu().numpy(), piped["power"])
    key = ["series", "bin", "width"]
    assert np.array_equal(np.sort(piped["cands"], order=key), np.sort(again, order=key))
    for i, n in enumerate(lengths):
        m = n // 2 + 1
        p = piped["power"][po[i]: po[i] + m].astype(np.float64)
        rows = slice(go[i], go[i] + max(1, m // seg_len))
        parity.check_normalise(parity.spectrum_complex(piped["spec"], so[i], m), piped["power"][po[i]: po[i] + m],
                               piped["stats"][rows], seg_len)
        mx_ref, am_ref = parity.check_maxima(p, piped["mx"][rows], piped["am"][rows], w_max, seg_len)
        parity.check_candidates(piped["cands"], p, mx_ref, am_ref, w_max, seg_len, sigma,
                                parity.n_trials_of(m, w_max), series=i)
    plan.set_pipeline(0)
    assert plan.pipeline_parts() == 0


@pytest.mark.parametrize("lengths,w_max,seg_len,sigma,tiling", [
    ([1 << 17], 300, 4096, 3.0, (4, 0, 0)),
    ([1 << 17], 300, 4096, 3.0, (4, 0, 1)),
    ([1 << 16], 100, 777, 2.0, (2, 1, 0)),
    ([1 << 13, 1 << 15, 6000, 1 << 14], 48, 256, 3.0, (1, 0, 1)),
    ([1 << 14], 40, 50, 3.0, (1, 0, 0)),
])
def test_fused_search_matches_separate_stages(pkg, lengths, w_max, seg_len, sigma, tiling):
    """The fused search (block statistics, then P formed from the spectrum in
    the bank and the deferred blocks) gives exactly the records of the
    separate stages, with and without a graph; those records match the
    oracle on the separate stages' power, with either form of the deferred
    blocks.  Shapes: scalar and packed banks,
    persistent tiles, an odd segment length, a batch of uneven lengths and
    segments shorter than a deferred block's reach (the small deferred kernel)."""
    xs = [_series(n, seed=400 + i) for i, n in enumerate(lengths)]
    plan = pkg.Plan(lengths=lengths, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    plan.set_tiling(*tiling)
    xo, so, po, go = plan.offsets()
    x_all = np.zeros(plan.x_floats, dtype=np.float32)
    for i, x in enumerate(xs):
        x_all[xo[i]: xo[i] + len(x)] = x
    sep = parity.run_gpu(plan, x_all, maxima=True)
    key = ["series", "bin", "width"]
    plan.set_fused(1)
    for form in (0, 1):   # both forms of the deferred blocks form P themselves
        plan.set_defer_form(form)
        for use_graph in (False, True):
            d_x, d_spec, d_power = plan.buffers("cuda")
            d_x.copy_(torch.from_numpy(x_all))
            d_power.fill_(-1.0)
            plan.search(d_x, d_spec, d_power, use_graph=use_graph)
            fused = plan.candidates()
            assert float(d_power.max()) == -1.0   # P never written
            assert len(fused) == len(sep["cands"]) and len(fused) > 0
            assert np.array_equal(np.sort(fused, order=key), np.sort(sep["cands"], order=key))
    plan.set_fused(0)
    for i, n in enumerate(lengths):
        m = n // 2 + 1
        p = sep["power"][po[i]: po[i] + m].astype(np.float64)
        rows = slice(go[i], go[i] + max(1, m // seg_len))
        mx_ref, am_ref = parity.check_maxima(p, sep["mx"][rows], sep["am"][rows], w_max, seg_len)
        parity.check_candidates(sep["cands"], p, mx_ref, am_ref, w_max, seg_len, sigma,
                                parity.n_trials_of(m, w_max), series=i)


@pytest.mark.parametrize("n,w_max,seg_len,sigma", [
    (1 << 16, 100, 1024, 3.0),
    (3 * (1 << 12) + 10, 130, 1000, 3.0),
    (1 << 17, 300, 4096, 3.0),
])
@pytest.mark.parametrize("tiling", [(2, 0, 0), (4, 0, 1)])
def test_deferred_forms_and_inline_exact_agree(pkg, n, w_max, seg_len, sigma, tiling):
    """The deferred blocks inspected by three warps per block, by one warp per
    block (through a captured graph too), and with no room for deferred
    blocks (every flagged block inspected inline by its own warp): the same
    records bit for bit, and the oracle's."""
    x = _series(n, seed=9)
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    plan.set_tiling(*tiling)
    outs = []
    for form in (0, 1):
        plan.set_defer_form(form)
        assert plan.defer_form() == form
        outs.append(parity.run_gpu(plan, x, maxima=(form == 0)))
        deferred = plan.counters()[0]
        assert deferred > 0
        outs.append(parity.run_gpu(plan, x, maxima=False, use_graph=True))
    plan.set_defer_capacity(0)
    outs.append(parity.run_gpu(plan, x, maxima=False))
    assert plan.counters()[0] >= deferred
    keys = [np.sort(o["cands"], order=["series", "bin", "width"]) for o in outs]
    for k in keys[1:]:
        assert np.array_equal(keys[0], k)
    m = n // 2 + 1
    p64 = outs[0]["power"][:m].astype(np.float64)
    mx_ref, am_ref = parity.check_maxima(p64, outs[0]["mx"], outs[0]["am"], w_max, seg_len)
    parity.check_candidates(outs[0]["cands"], p64, mx_ref, am_ref, w_max, seg_len, sigma,
                            parity.n_trials_of(m, w_max))


def test_plans_of_different_sizes_coexist(pkg):
    """A smaller plan created later must not break the launches of a larger one."""
    n = 1 << 15
    x = _series(n, seed=21)
    big = pkg.Plan(n=n, z_max=400, segment_len=2048, threshold_sigma=4.0)
    first = parity.run_gpu(big, x, maxima=False)
    small = pkg.Plan(n=n, z_max=5, segment_len=16, threshold_sigma=4.0)
    parity.run_gpu(small, x, maxima=False)
    again = parity.run_gpu(big, x, maxima=False)
    a = np.sort(first["cands"], order=["series", "bin", "width"])
    b = np.sort(again["cands"], order=["series", "bin", "width"])
    assert np.array_equal(a, b)


@pytest.mark.parametrize("mode,step", [(1, 3), (1, 7), (2, 1)])
def test_searched_width_subsets(pkg, mode, step):
    """Width sampling: only the searched widths are compared and reported, with
    the Bonferroni count over the searched widths (all widths still summed)."""
    n, w_max, seg_len, sigma = 1 << 16, 70, 512, 2.0
    x = _series(n, seed=9)
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    plan.set_widths(mode, step)
    out = parity.run_gpu(plan, x)
    m = n // 2 + 1
    ws = opipe.searched_widths(w_max, {1: "step", 2: "log2"}[mode], step)
    t = plan.thresholds()
    assert np.all(np.isinf(np.delete(t, np.array(ws) - 1))) and np.all(np.isfinite(t[np.array(ws) - 1]))
    p64 = out["power"][:m].astype(np.float64)
    mx_ref, am_ref = parity.check_maxima(p64, out["mx"], out["am"], w_max, seg_len)
    k = parity.check_candidates(out["cands"], p64, mx_ref, am_ref, w_max, seg_len, sigma,
                                opipe.n_trials_default(m, w_max, ws), widths=ws)
    assert k >= 10
    assert set(int(w) for w in out["cands"]["width"]) <= set(ws)


def test_rblock_reports_block_index(pkg):
    n, w_max, seg_len, sigma = 1 << 16, 48, 512, 2.0
    x = _series(n, seed=10)
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    plan.set_trials(1.0)
    exact = parity.run_gpu(plan, x)["cands"]
    plan.set_rblock(1000)
    approx = parity.run_gpu(plan, x)["cands"]
    assert len(exact) == len(approx) > 100
    assert np.array_equal(approx["bin"], exact["bin"] // 1000)
    for f in ("series", "width", "power", "sigma"):
        assert np.array_equal(approx[f], exact[f])


@pytest.mark.parametrize("warps,persistent,packed", [(1, 1, 0), (2, 1, 0), (3, 1, 0), (4, 1, 0), (1, 0, 0), (3, 0, 0),
                                                     (4, 0, 0), (1, 1, 1), (2, 0, 1), (3, 1, 1), (4, 0, 1)])
def test_launch_shapes_give_the_same_search(pkg, warps, persistent, packed):
    """Every tile width, both launch forms (one CTA per tile; persistent
    per-SM tile ranges with stealing) and both add forms (scalar; packed
    pairs over two slices per warp) against the oracle on one input."""
    n, w_max, seg_len, sigma = 1 << 18, 48, 1024, 2.5
    x = _series(n, seed=12)
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    plan.set_tiling(warps, persistent, packed)
    assert plan.tiling() == (warps, persistent, packed)
    out = parity.run_gpu(plan, x)
    m = n // 2 + 1
    p64 = out["power"][:m].astype(np.float64)
    mx_ref, am_ref = parity.check_maxima(p64, out["mx"], out["am"], w_max, seg_len)
    parity.check_candidates(out["cands"], p64, mx_ref, am_ref, w_max, seg_len, sigma,
                            parity.n_trials_of(m, w_max))


def test_autotune_keeps_the_candidates(pkg):
    n, w_max, seg_len, sigma = 1 << 18, 64, 1024, 3.0
    x = _series(n, seed=13)
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    before = parity.run_gpu(plan, x, maxima=False)
    d_power = torch.from_numpy(before["power"]).cuda()
    warps, persistent, packed = plan.autotune(d_power)
    assert warps in (1, 2, 3, 4) and persistent in (0, 1) and packed in (0, 1)
    after = parity.run_gpu(plan, x, maxima=False)
    assert len(after["cands"]) == len(before["cands"]) > 0
    for f in ("series", "width", "bin", "power", "sigma"):
        assert np.array_equal(np.sort(after["cands"][f]), np.sort(before["cands"][f]))


def test_host_entry_points_match_the_device_path(pkg):
    """pulscan_search_host and pulscan_search_host_async (two plans in turn on
    two streams, as a pipelined stream of series) give exactly the records of
    the device-buffer path on the same series."""
    n, w_max, seg_len, sigma = 1 << 16, 64, 1024, 4.0
    xs = [synth.inject(synth.noise(n, 40 + i), [dict(amp=0.15, r0=0.2 * n / 2 + 300 * i, z=30.0, w=0.0, phi0=0.3)])
          for i in range(4)]
    ref = []
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    d_x, d_spec, d_power = plan.buffers("cuda")
    for x in xs:
        d_x.copy_(torch.from_numpy(x))
        plan.search(d_x, d_spec, d_power)
        ref.append(plan.candidates())
    assert all(len(r) > 0 for r in ref)
    for i, x in enumerate(xs):
        got = plan.search_host(torch.from_numpy(x).pin_memory(), use_graph=bool(i % 2))
        assert np.array_equal(got, ref[i])
    plans = [plan, pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pins = [torch.from_numpy(x).pin_memory() for x in xs]
    plans[0].search_host_async(pins[0], stream=streams[0])
    for i in range(len(xs)):
        if i + 1 < len(xs):
            plans[(i + 1) % 2].search_host_async(pins[i + 1], stream=streams[(i + 1) % 2])
        got = plans[i % 2].candidates(stream=streams[i % 2])
        assert np.array_equal(got, ref[i]), i


# (n, z_max, segment_len): 1024 = 31 * 33 + 1 puts a segment boundary at every
# position 1..32 of a lane and two boundaries in some 1056-bin slices; 4096
# and 1000 give one boundary per slice; 48 puts a lane across three segments
@pytest.mark.parametrize("n,w_max,seg_len", [
    (1 << 16, 100, 1024),
    (1 << 15, 70, 4096),
    (3 * (1 << 12) + 10, 130, 1000),
    (1 << 13, 40, 48),
])
@pytest.mark.parametrize("tiling", [(2, 0, 0), (4, 0, 1)])
def test_segment_maxima_exact_ties(pkg, n, w_max, seg_len, tiling):
    """Integer-valued power (sparse ones and twos, and three segments of
    zeros): every window sum is exact in FP32 and in FP64, so maxima tie
    exactly and often.  The dump mode must return the oracle's maxima and its
    lowest-bin argmax (Algorithm 4's first index) bit for bit, and so must
    the thresholded search's records."""
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=3.0)
    plan.set_tiling(*tiling)
    m = n // 2 + 1
    rng = np.random.default_rng(seg_len + w_max)
    p = rng.choice(np.array([0.0, 0.0, 0.0, 1.0, 2.0], dtype=np.float32), size=m)
    p[m // 3: m // 3 + 3 * seg_len] = 0.0
    d_power = torch.zeros(plan.power_floats, dtype=torch.float32, device="cuda")
    d_power[:m] = torch.from_numpy(p)
    nn = plan.total_segments * w_max
    mx = torch.empty(nn, dtype=torch.float32, device="cuda")
    am = torch.empty(nn, dtype=torch.int64, device="cuda")
    plan.segment_maxima(d_power, mx, am)
    torch.cuda.synchronize()
    mx_ref, am_ref = obox.segment_maxima(p.astype(np.float64), w_max, seg_len)
    mg = mx.cpu().numpy().reshape(plan.total_segments, w_max).astype(np.float64)
    ag = am.cpu().numpy().reshape(plan.total_segments, w_max)
    empty = np.isnan(mx_ref)
    assert np.array_equal(np.isnan(mg), empty)
    assert np.array_equal(mg[~empty], mx_ref[~empty])
    assert np.array_equal(ag, am_ref)
    # the thresholded search on a denser integer power (deferred blocks and
    # inline exact steps): every record's power and bin exactly the oracle's
    q = rng.choice(np.arange(6, dtype=np.float32), size=m)
    d_power[:m] = torch.from_numpy(q)
    q64 = q.astype(np.float64)
    mq, aq = obox.segment_maxima(q64, w_max, seg_len)
    for form in (0, 1):
        plan.set_defer_form(form)
        plan.boxcar_search(d_power)
        cands = plan.candidates()
        assert parity.check_candidates(cands, q64, mq, aq, w_max, seg_len, 3.0,
                                       parity.n_trials_of(m, w_max)) > 0
        seg = np.minimum(cands["bin"].astype(np.int64) // seg_len, mq.shape[0] - 1)
        wi = cands["width"].astype(np.int64) - 1
        assert np.array_equal(cands["power"].astype(np.float64), mq[seg, wi])
        assert np.array_equal(cands["bin"].astype(np.int64), aq[seg, wi])
    plan.close()


def test_packed_and_scalar_banks_give_identical_records(pkg):
    """The packed bank performs the scalar bank's FP32 adds in the same order
    (each half of add.rn.f32x2 rounds as add.rn.f32), so the records agree
    bit for bit, on a series hot enough to defer many blocks."""
    n, w_max, seg_len, sigma = 1 << 18, 200, 2048, 2.0
    x = _series(n, seed=15)
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    plan.set_trials(1.0)
    outs = []
    for packed in (0, 1):
        plan.set_tiling(4, 0, packed)
        outs.append(parity.run_gpu(plan, x, maxima=True))
        assert plan.counters()[0] > 0
    assert len(outs[0]["cands"]) > 100
    assert np.array_equal(outs[0]["cands"], outs[1]["cands"])
    assert np.array_equal(outs[0]["mx"], outs[1]["mx"]) and np.array_equal(outs[0]["am"], outs[1]["am"])


@pytest.mark.parametrize("packed", [0, 1])
def test_timeout_path_reports_and_recovers(pkg, packed):
    """The bounded-wait path without a fault: an armed search issues no copy
    and waits 20 us on the copy's barrier, so every tile gives up with
    nothing in flight; pulscan_candidates reports PULSCAN_ERR_TIMEOUT, and the
    next search (graph replay) gives the normal records."""
    n, w_max, seg_len, sigma = 1 << 16, 64, 1024, 4.0
    x = _series(n, seed=14)
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    plan.set_tiling(2, -1, packed)
    d_x, d_spec, d_power = plan.buffers("cuda")
    d_x.copy_(torch.from_numpy(x))
    plan.search(d_x, d_spec, d_power, use_graph=True)
    ref = plan.candidates()
    assert len(ref) > 0
    plan.test_wait_timeout(20)
    plan.search(d_x, d_spec, d_power, use_graph=True)
    with pytest.raises(pkg.PulscanError) as err:
        plan.candidates()
    assert err.value.code == -5
    plan.search(d_x, d_spec, d_power, use_graph=True)
    assert np.array_equal(plan.candidates(), ref)
    with pytest.raises(pkg.PulscanError):
        plan.test_wait_timeout(0)
