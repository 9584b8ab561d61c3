"""Benchmark of the GB300 boxcar search (one JSON line on stdout, rank 0).

Workload: the SPOTLIGHT-scale single series -- N = 2^23 float32 samples of
Gaussian noise with 8 injected drifting tones, boxcar widths 1..1024, segments
of 4096 bins, threshold 6 sigma (synthetic stand-in for the paper's `.fft`
inputs).  One step = the whole path: R2C FFT (cuFFT), per-segment median/MAD
normalisation, the boxcar bank over every width at every bin, and the
per-(segment, width) maximum / threshold / significance.  The metric is
boxcar bins x widths per second, M * W / step time, summed over ranks.

--impl reference times the FP64 CPU oracle instead (the repository's own
reference implementation of the method), on a bounded sample of the same
workload scaled to the same unit.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "single_2p23"
METRIC = "boxcar bins x widths per second"
UNIT = "G bin-widths/s"
L2_FLUSH_BYTES = 512 << 20      # > 129 MB of L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-series batched measurement")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiable 4096-binary measurement")
    ap.add_argument("--diff-binaries", type=int, default=None,
                    help="run the differentiable measurement on its first N binaries only (profiling)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the step's stages one by one instead of as one CUDA graph")
    ap.add_argument("--tiling", default=None, metavar="WARPS,PERSISTENT",
                    help="bank launch shape of the single-series plan instead of the autotuner (e.g. 4,0)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (x itself without a process group): every
    rank's step time is the slowest rank's, as the job ends with the last."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank, ms):
    """Whole-job throughput in G units/s: each of `world` replicas processes
    units_per_rank in the slowest rank's ms."""
    return world * units_per_rank / (ms * 1e-3) / 1e9


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def profile_traffic(kernel_src):
    """DRAM bytes per launch from the committed ncu summary, if it matches the kernel source."""
    path = os.path.join(ROOT, "profiles", "boxcar_search_single_2p23.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    want = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    src_hash = traffic = None
    for ln in text.splitlines():
        if ln.startswith("kernel_source_sha256_16:"):
            src_hash = ln.split(":", 1)[1].strip()
        if ln.startswith("dram_bytes_per_launch:"):
            traffic = float(ln.split(":", 1)[1].strip())
    return traffic if src_hash == want else None


# ------------------------------------------------------------------ oracle arm
def oracle_fft(x):
    """The oracle's FFT of the whole series, with its time (s)."""
    from oracle import fft as offt
    t0 = time.perf_counter()
    spec = offt.rfft(x.astype(np.float64))
    return spec, time.perf_counter() - t0


def oracle_sample(spec, t_fft, cfg, n_seg_sample):
    """Time the FP64 oracle on a bounded sample; returns (G bin-widths/s, seconds, description).

    The FFT is timed once on the whole series (t_fft); normalisation and the
    boxcar stage are linear in segments, so they are timed on the first
    n_seg_sample segments and scaled to the whole series.
    """
    from oracle import boxcar as obox
    from oracle import normalise as onorm
    from oracle import pipeline as opipe
    n, w_max, seg_len, sigma = cfg["n"], cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    m = n // 2 + 1
    n_seg = m // seg_len
    t1 = time.perf_counter()
    sub = n_seg_sample * seg_len + w_max
    p, _, _ = onorm.normalise_power(spec[:sub], seg_len)
    mx, am = obox.segment_maxima(p, w_max, seg_len, seg_range=(0, n_seg_sample))
    opipe.candidates_from_maxima(mx[:n_seg_sample], am[:n_seg_sample], w_max, opipe.n_trials_default(m, w_max),
                                 sigma)
    t3 = time.perf_counter()
    frac = n_seg_sample / n_seg
    t_full = t_fft + (t3 - t1) / frac
    desc = (f"oracle FFT of the full 2^{n.bit_length() - 1}-sample series ({t_fft:.1f} s, timed once) + "
            f"normalise/boxcar/search of {n_seg_sample}/{n_seg} segments, scaled linearly to all segments")
    return m * w_max / t_full / 1e9, (t3 - t1), desc


def _oracle_segments(job):
    """One worker's share of the oracle stages (normalise, maxima, candidates); seconds."""
    spec, w_max, seg_len, sigma, n_trials, n_seg = job
    from oracle import boxcar as obox
    from oracle import normalise as onorm
    from oracle import pipeline as opipe
    t0 = time.perf_counter()
    p, _, _ = onorm.normalise_power(spec, seg_len)
    mx, am = obox.segment_maxima(p, w_max, seg_len, seg_range=(0, n_seg))
    opipe.candidates_from_maxima(mx[:n_seg], am[:n_seg], w_max, n_trials, sigma)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_parallel(spec, t_fft, cfg, seg_per_proc, procs):
    """The oracle on all host cores: processes (spawned, so no CUDA state is
    inherited) each run normalise + maxima + candidates on their own run of
    seg_per_proc segments; wall time of the parallel pass, the FFT (one core,
    timed once) added, scaled linearly to all segments."""
    import multiprocessing as mp
    n, w_max, seg_len, sigma = cfg["n"], cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    m = n // 2 + 1
    n_seg = m // seg_len
    procs = max(1, min(procs, n_seg // seg_per_proc))
    nt = float(m) * w_max
    jobs = [(spec[i * seg_per_proc * seg_len: (i + 1) * seg_per_proc * seg_len + w_max], w_max, seg_len, sigma, nt,
             seg_per_proc) for i in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_segments, [(j[0][: 2 * seg_len + w_max], w_max, seg_len, sigma, nt, 1) for j in jobs])
        t0 = time.perf_counter()
        pool.map(_oracle_segments, jobs)
        t = time.perf_counter() - t0
    frac = procs * seg_per_proc / n_seg
    t_full = t_fft + t / frac
    desc = (f"oracle FFT of the full series on one core ({t_fft:.1f} s, timed once) + normalise/boxcar/search "
            f"of {procs * seg_per_proc}/{n_seg} segments on {procs} processes ({seg_per_proc} each, "
            f"{t:.1f} s wall), scaled linearly to all segments")
    return m * w_max / t_full / 1e9, t, desc, procs


def run_reference(args, rank, world):
    """The oracle on the host cores: each step is one bounded sample of the
    workload -- normalise + maxima + candidates of 2 segments per process over
    a spawned pool of all host cores -- with the FFT of the whole series
    (one core, timed once) added and the sample scaled to the series."""
    if rank != 0:
        return
    import multiprocessing as mp
    from paper_2406_15186_gb300 import synth
    cfg = synth.WORKLOADS[WORKLOAD]
    x, _ = synth.single_series(WORKLOAD)
    n, w_max, seg_len, sigma = cfg["n"], cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    m = n // 2 + 1
    n_seg = m // seg_len
    spec, t_fft = oracle_fft(x)
    procs = max(1, min(host_cores(), n_seg // 2))
    per = 2
    nt = float(m) * w_max
    jobs = [(spec[i * per * seg_len: (i + 1) * per * seg_len + w_max], w_max, seg_len, sigma, nt, per)
            for i in range(procs)]
    vals = []
    with mp.get_context("spawn").Pool(procs) as pool:
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_segments, jobs)
            t = time.perf_counter() - t0
            if i >= args.warmup:
                t_full = t_fft + t / (procs * per / n_seg)
                vals.append(m * w_max / t_full / 1e9)
    value = statistics.mean(vals)
    desc = (f"oracle FFT of the full series on one core ({t_fft:.1f} s, timed once) + normalise/boxcar/search of "
            f"{procs * per}/{n_seg} segments per step on {procs} processes, scaled linearly to all segments")
    ms = m * w_max / (value * 1e9) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: N=2^23, z_max=1024, segment_len=4096, sigma=6",
                       "sample": desc, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_batched(torch, pkg, synth, dev, stream, steps):
    """512 uneven DM-trial series: one graph replay vs per-series launches of the same kernels."""
    cfg = synth.WORKLOADS["batch_512"]
    w_max, seg_len, sigma = cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    lengths = synth.batch_lengths(cfg["n_series"], cfg["lengths"])
    mask = synth.batch_tone_mask(cfg["n_series"])
    plan = pkg.Plan(lengths=lengths, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    xo, so, po, _ = plan.offsets()
    with torch.cuda.stream(stream):
        d_x, d_spec, d_power = plan.buffers(dev)
        synth.batch_device(d_x, xo, lengths, mask)
    torch.cuda.synchronize()
    bins = sum(n // 2 + 1 for n in lengths)

    def timed(fn, reps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    plan.rfft(d_x, d_spec, stream=stream)
    plan.power_normalise(d_spec, d_power, stream=stream)
    tiling = plan.autotune(d_power, stream=stream)

    def batched():
        plan.search(d_x, d_spec, d_power, use_graph=True, stream=stream)

    plans = {n: pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma) for n in sorted(set(lengths))}
    xp, sp, pp = d_x.data_ptr(), d_spec.data_ptr(), d_power.data_ptr()

    def per_series():
        for i, n in enumerate(lengths):
            p = plans[n]
            p.rfft(xp + 4 * int(xo[i]), sp + 8 * int(so[i]), stream=stream)
            p.power_normalise(sp + 8 * int(so[i]), pp + 4 * int(po[i]), stream=stream)
            p.boxcar_search(pp + 4 * int(po[i]), stream=stream)

    batched()
    per_series()
    t_b = timed(batched, steps)
    n_cands = len(plan.candidates(stream=stream))
    t_s = timed(per_series, max(1, steps // 2))
    return {"workload": f"batch_512: 512 series, lengths U{{2^20..2^23}} (sum {sum(lengths)} samples, "
                        f"{bins} bins), 26 with a tone, z_max={w_max}, segment_len={seg_len}, sigma={sigma:g}",
            "dm_trials_per_s": len(lengths) / (t_b * 1e-3), "ms_per_batch": t_b,
            "per_series_dm_trials_per_s": len(lengths) / (t_s * 1e-3), "ms_per_series_loop": t_s,
            "ratio_batched_vs_per_series": t_s / t_b, "bin_widths_per_s": bins * w_max / (t_b * 1e-3) / 1e9,
            "bank_tiling": {"warps_per_cta": tiling[0], "persistent": tiling[1], "by": "pulscan_plan_autotune"},
            "unit": "G bin-widths/s", "candidates": n_cands, "graph": True,
            "per_series": "the same kernels launched per series on one stream (no graph), one plan per length",
            "l2": "inputs (8.2 GB) far larger than L2"}


def run_harmonic(torch, pkg, synth, dev, stream, x, cfg, steps, flush):
    """The bench series searched with harmonic summing up to 4 harmonics (§2.3;
    numharm = 4 is the paper's setting in its timing runs)."""
    n, w_max, seg_len, sigma = cfg["n"], cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    numharm = 4
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma, numharm=numharm)
    with torch.cuda.stream(stream):
        d_x, d_spec, d_power = plan.buffers(dev)
        d_x.copy_(torch.from_numpy(x))
    torch.cuda.synchronize()
    plan.enable_timing(True)

    def step():
        plan.rfft(d_x, d_spec, stream=stream)
        plan.power_normalise(d_spec, d_power, stream=stream)
        plan.boxcar_search(d_power, stream=stream)

    for _ in range(3):
        step()
    ms, th = [], []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        th.append(plan.timings()[6])
    cands = plan.candidates(stream=stream)
    m = n // 2 + 1
    bins = sum(m // h for h in range(1, numharm + 1))
    t = statistics.mean(ms)
    t_h = statistics.mean(th)
    # algorithmic bytes of the stage sums per series bin: reads 4 B x (1/2 + 3),
    # writes 4 B x (1/2 + 1/3 + 1/4)
    hbytes = 4.0 * m * (0.5 + 3.0) + 4.0 * m * (1 / 2 + 1 / 3 + 1 / 4)
    plan.close()
    return {"workload": f"single_2p23 with harmonic sums H = 1..{numharm} (stage spectra of M/H bins, "
                        f"all searched with widths 1..{w_max})",
            "ms_per_step": t, "bin_widths_per_s": bins * w_max / (t * 1e-3) / 1e9, "unit": "G bin-widths/s",
            "harmonic_sum_ms": t_h, "harmonic_sum_gbs": hbytes / (t_h * 1e-3) / 1e9,
            "harmonic_sum_bytes": hbytes,
            "candidates_by_stage": [int((cands["harmonics"] == h).sum()) for h in range(1, numharm + 1)]}


def run_fidelity(torch, pkg, plan, step, stream, steps, flush):
    """The bench step in the paper-GPU fidelity mode (median of medians, every
    (segment, width) maximum, polynomial log p)."""
    plan.set_fidelity(pkg.FIDELITY_PAPER_GPU)
    step()
    ms, kn, kb, kf = [], [], [], []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        t = plan.timings()
        kn.append(t[1])
        kb.append(t[2])
        kf.append(t[4])
    n_c = len(plan.candidates(stream=stream))
    plan.set_fidelity(pkg.FIDELITY_EXACT)
    return {"ms_per_step": statistics.mean(ms), "normalise_mom_ms": statistics.mean(kn),
            "all_maxima_ms": statistics.mean(kb), "poly_finalise_ms": statistics.mean(kf), "candidates": n_c,
            "note": "median of medians over each 4096-bin block, the unthresholded bank (every segment x width "
                    "maximum), the fitted polynomial log p per maximum"}


def run_diff(torch, pkg, synth, dev, stream, steps, n_binaries=None):
    """Differentiable batch: logsumexp forward and hand-written backward over
    4096 binaries of 2^20 samples (widths 1..512, L = 2048, tau = 0.1); the
    first n_binaries of them only when given (a reduced case for profiling)."""
    cfg = synth.WORKLOADS["diff_4096"]
    n, n_series, w_max, seg_len, tau = cfg["n"], cfg["n_series"], cfg["z_max"], cfg["segment_len"], cfg["tau"]
    if n_binaries:
        n_series = min(n_series, int(n_binaries))
    m = n // 2 + 1
    lib = pkg.load()
    plan = pkg.Plan(lengths=[n] * n_series, z_max=w_max, segment_len=seg_len, threshold_sigma=6.0)
    xo = plan.offsets()[0]
    f32 = dict(dtype=torch.float32, device=dev)
    x = torch.empty(plan.x_floats, **f32)
    tmpl = torch.empty(plan.x_floats, **f32)
    with torch.cuda.stream(stream):
        amps = torch.from_numpy(synth.diff_device(x, tmpl, xo, n, n_series)).to(dev)
    torch.cuda.synchronize()
    sp = stream.cuda_stream
    rc = lib.pulscan_inject(plan._h, x.data_ptr(), tmpl.data_ptr(), amps.data_ptr(), x.data_ptr(), sp)
    assert rc == 0
    spec = torch.empty(plan.spec_floats, **f32)
    power = torch.empty(plan.power_floats, **f32)
    stats = torch.empty(4 * plan.total_segments, **f32)
    sel = torch.empty(8 * plan.total_segments, **f32)
    y = torch.empty(plan.total_segments * w_max, **f32)
    gy = torch.ones_like(y)
    gx = torch.empty(plan.x_floats, **f32)
    gamp = torch.empty(n_series, **f32)

    def fwd():
        return lib.pulscan_lse_forward(plan._h, x.data_ptr(), spec.data_ptr(), power.data_ptr(), stats.data_ptr(),
                                       sel.data_ptr(), y.data_ptr(), tau, sp)

    def bwd():
        rc = lib.pulscan_lse_backward(plan._h, spec.data_ptr(), power.data_ptr(), stats.data_ptr(), sel.data_ptr(),
                                      y.data_ptr(), gy.data_ptr(), gx.data_ptr(), tau, sp)
        return rc or lib.pulscan_amplitude_grad(plan._h, gx.data_ptr(), tmpl.data_ptr(), gamp.data_ptr(), sp)

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            assert fn() == 0
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    assert fwd() == 0 and bwd() == 0
    t_f = timed(fwd, steps)
    t_b = timed(bwd, steps)
    ok = bool(torch.isfinite(gamp).all())
    bw = n_series * m * w_max
    plan.close()
    return {"workload": f"diff_4096: {n_series} binaries x 2^20 samples (M={m}), widths 1..{w_max}, "
                        f"segment_len={seg_len}, tau={tau}",
            "ms_forward": t_f, "ms_backward": t_b, "forward_bin_widths_per_s": bw / (t_f * 1e-3) / 1e9,
            "forward_backward_bin_widths_per_s": bw / ((t_f + t_b) * 1e-3) / 1e9, "unit": "G bin-widths/s",
            "finite_gradients": ok,
            "forward": "rfft + normalise (order statistics kept) + logsumexp of the boxcar bank",
            "backward": "softmax-weighted boxcar scatter + median/MAD adjoint + C2R + amplitude reduction",
            "l2": f"inputs ({4 * n * n_series / 1e9:.2f} GB) larger than L2"}


def run_ours(args, rank, world, local):
    import torch
    import paper_2406_15186_gb300 as pkg
    from paper_2406_15186_gb300 import build, synth

    build.build()
    pkg.load()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    cfg = synth.WORKLOADS[WORKLOAD]
    n, w_max, seg_len, sigma = cfg["n"], cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    m = n // 2 + 1
    x, _ = synth.single_series(WORKLOAD)
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        d_x, d_spec, d_power = plan.buffers(dev)
        d_x.copy_(torch.from_numpy(x))
    torch.cuda.synchronize()
    # the timed steps record only the bank kernel's event pair (the roofline's
    # live kernel time): every event between two kernels drains the pipeline
    # and adds a few microseconds; the per-stage breakdown comes from extra
    # steps with every stage's events, after the timed region
    plan.enable_timing(2)

    def step():
        if args.no_graph:
            plan.rfft(d_x, d_spec, stream=stream)
            plan.power_normalise(d_spec, d_power, stream=stream)
            plan.boxcar_search(d_power, stream=stream)
        else:
            # the whole path as one CUDA graph launch (pulscan_search), its
            # timing events captured inside the graph
            plan.search(d_x, d_spec, d_power, use_graph=True, stream=stream)

    step()
    if args.tiling:
        plan.set_tiling(*[int(v) for v in args.tiling.split(",")])
        tiling, tiling_by = plan.tiling(), "--tiling"
    else:
        tiling = plan.autotune(d_power, stream=stream)     # launch shape of the bank, timed on this input
        tiling_by = "pulscan_plan_autotune"
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        step()
    n_cands = len(plan.candidates(stream=stream))
    n_deferred = plan.counters()[0]      # blocks the bank handed to the deferred kernel
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    k_search = []
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()                       # L2 flushed between timed steps (outside the events)
            ev[i][0].record(stream)
        step()
        with torch.cuda.stream(stream):
            ev[i][1].record(stream)
        k_search.append(plan.timings()[2])     # the bank kernel's events in this step (same stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(statistics.mean(step_ms), dist, dev)
    value = job_value(world, m * w_max, ms)

    # per-stage breakdown: extra steps with every stage's events
    plan.enable_timing(True)
    step()
    n_break = max(5, args.steps // 2)
    k_fft, k_norm, k_bank, k_def, k_fin, break_ms = [], [], [], [], [], []
    for _ in range(n_break):
        with torch.cuda.stream(stream):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        step()
        with torch.cuda.stream(stream):
            e1.record(stream)
        t = plan.timings()
        k_fft.append(t[0])
        k_norm.append(t[1])
        k_bank.append(t[2])
        k_def.append(t[3])
        k_fin.append(t[4])
        torch.cuda.synchronize()
        break_ms.append(e0.elapsed_time(e1))

    # searched-width subsets (every width still summed): the same step with
    # the z mod 8 and log2 z samplings
    sampling = {}
    for name, mode, stp in (("step8", 1, 8), ("log2", 2, 1)):
        plan.set_widths(mode, stp)
        step()
        ts = []
        for _ in range(max(3, args.steps // 2)):
            with torch.cuda.stream(stream):
                flush.zero_()
            step()
            t = plan.timings()
            ts.append(t[2] + t[3] + t[4])
        sampling[name] = {"search_ms": statistics.mean(ts), "candidates": len(plan.candidates(stream=stream))}
    plan.set_widths(0, 1)
    harmonic = run_harmonic(torch, pkg, synth, dev, stream, x, cfg, max(3, args.steps // 2), flush)
    fidelity = run_fidelity(torch, pkg, plan, step, stream, max(3, args.steps // 2), flush)
    sampling["all"] = {"search_ms": statistics.mean(k_bank) + statistics.mean(k_def) + statistics.mean(k_fin),
                       "candidates": n_cands}

    # end to end through the host-buffer entry points, as a stream of series:
    # two plans in turn on two streams (double buffering), so one series'
    # copy to the device runs while the previous one's search does.  Every
    # step has its own L2 flush (on its stream, before its copy), its H2D
    # copy of the series from pinned memory and its D2H read of candidates.
    plan.enable_timing(False)
    plan_b = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    plan_b.set_tiling(*tiling)
    plans, streams = [plan, plan_b], [stream, torch.cuda.Stream(device=dev)]
    x_pin = [torch.from_numpy(x).pin_memory(), torch.from_numpy(x.copy()).pin_memory()]
    cap = min(plan.max_candidates, 1 << 16)

    def issue(i):
        k = i % 2
        with torch.cuda.stream(streams[k]):
            flush.zero_()
        plans[k].search_host_async(x_pin[k], use_graph=True, stream=streams[k])

    for i in range(2):                          # warm-up: both plans capture their graphs
        issue(i)
        plans[i].candidates(cap=cap, stream=streams[i])
    torch.cuda.synchronize()
    n_e2e = max(4, args.steps)
    nc = 0
    t0 = time.perf_counter()
    issue(0)
    for i in range(n_e2e):
        if i + 1 < n_e2e:
            issue(i + 1)
        nc = len(plans[i % 2].candidates(cap=cap, stream=streams[i % 2]))   # waits for step i
    e2e_ms_mean = max_over_ranks((time.perf_counter() - t0) * 1e3 / n_e2e, dist, dev)
    plan_b.close()

    peaks, peak_kind = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    p_add = props.multi_processor_count * 128 * sm_max * 1e6          # FP32 adds/s
    t_search = statistics.mean(k_search) * 1e-3
    adds = m * (w_max - 1)
    achieved = adds / t_search / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": p_add / 1e12, "unit": "TFLOP/s",
                "frac": achieved / (p_add / 1e12),
                "traffic": profile_traffic(os.path.join(ROOT, "paper_2406_15186_gb300", "csrc", "boxcar.cu")),
                "kernel": "boxcar_kernel<search>",
                "peak_source": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {sm_max:.0f} MHz "
                               f"({peak_kind} sm_max_mhz)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: N=2^23 samples (M=4194305 bins), 8 drifting tones, "
                                   f"z_max=1024, segment_len=4096, sigma=6",
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "bank_tiling": {"warps_per_cta": tiling[0], "persistent": tiling[1], "by": tiling_by},
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "kernels_ms": {"rfft_cufft": statistics.mean(k_fft), "normalise": statistics.mean(k_norm),
                           "boxcar_search": statistics.mean(k_bank), "deferred_blocks": statistics.mean(k_def),
                           "finalise": statistics.mean(k_fin),
                           "boxcar_search_live": statistics.mean(k_search),
                           "note": f"per-stage events from {n_break} extra steps recording every stage "
                                   f"({statistics.mean(break_ms):.4f} ms per step with those events); "
                                   "boxcar_search_live: the bank's own event pair inside the timed steps "
                                   "(the roofline's time)"},
            "candidates": n_cands, "deferred_blocks": n_deferred,
            "width_sampling": dict(sampling, note="boxcar + deferred + finalise per step; all widths summed, "
                                                  "only the sampled ones compared (z mod 8 == 0; z a power of two)"),
            "harmonics": harmonic,
            "paper_gpu_fidelity": fidelity,
            "roofline": roofline,
            "e2e": {"value": job_value(world, m * w_max, e2e_ms_mean), "unit": UNIT,
                    "ms_per_step": e2e_ms_mean, "h2d_bytes_per_step": 4 * n,
                    "d2h_bytes_per_step": 16 + 32 * nc, "steps": n_e2e,
                    "pipeline": "pulscan_search_host_async + pulscan_candidates on two plans and two "
                                "streams in turn (a series' copy overlaps the previous search); each step "
                                "flushes L2 on its stream before its copy; wall clock over all steps"},
            # this library's kernels per step: normalise, bank, deferred
            # blocks, word scan, finaliser (cuFFT's own kernels not counted)
            "gpu_launches": 5 * args.steps,
            "clocks": clocks}
    if not args.no_batched:
        plan.close()
        del d_x, d_spec, d_power
        torch.cuda.empty_cache()
        line["batched"] = run_batched(torch, pkg, synth, dev, stream, max(3, args.steps // 4))
        torch.cuda.empty_cache()
    if not args.no_diff:
        plan.close()
        d_x = d_spec = d_power = None
        torch.cuda.empty_cache()
        line["differentiable"] = run_diff(torch, pkg, synth, dev, stream, 3, args.diff_binaries)
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        spec, t_fft = oracle_fft(x)
        v1, secs, desc1 = oracle_sample(spec, t_fft, cfg, 64)
        vp, secs_p, desc_p, procs = oracle_parallel(spec, t_fft, cfg, 32, host_cores())
        line["cpu_baseline"] = {"value": vp, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": desc_p,
                                "seconds": secs_p + t_fft,
                                "single_core": {"value": v1, "cores": 1, "sample": desc1, "seconds": secs + t_fft}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
