"""Benchmark of the GB300 boxcar search (one JSON line on stdout, rank 0).

Headline workload: the large single series -- N = 2^27 float32 samples of
Gaussian noise with 32 injected drifting tones, boxcar widths 1..4096,
segments of 16384 bins, threshold 7 sigma (synthetic stand-in for the
paper's `.fft` inputs), the largest single-series workload.  One step = the
whole path: R2C FFT (cuFFT), per-segment median/MAD normalisation, the
boxcar bank over every width at every bin, and the per-(segment, width)
maximum / threshold / significance.  The metric is boxcar bins x widths per
second, M * W / step time, summed over ranks.  The other single-series
workloads (2^23 samples, widths 1..1024; 2^20 samples, widths 1..256), the
512-series batch and the differentiable batch are reported under their own
keys.

--impl reference times the FP64 CPU oracle instead (the repository's own
reference implementation of the method), on a bounded sample of the same
workload scaled to the same unit.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "single_2p27"
EXTRA_SINGLE = ("single_2p23", "single_2p20")
METRIC = "boxcar bins x widths per second"
UNIT = "G bin-widths/s"
L2_FLUSH_BYTES = 512 << 20      # > 129 MB of L2
L2_BYTES = 129 * 1000 * 1000   # GB300 L2 (inputs above it start cold)
FFT_PREFIX = 1 << 24            # oracle FFT sample of the 2^27-sample series


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD, choices=["single_2p27", "single_2p23", "single_2p20"],
                    help="headline single-series workload (profiling of a smaller case)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-series batched measurement")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiable 4096-binary measurement")
    ap.add_argument("--only-headline", action="store_true",
                    help="skip every section after the headline's timed steps (profiling)")
    ap.add_argument("--only-diff", action="store_true",
                    help="run only the differentiable measurement and print its JSON (profiling)")
    ap.add_argument("--only-fidelity", action="store_true",
                    help="run only the paper-GPU fidelity mode on --workload and print its JSON (profiling)")
    ap.add_argument("--diff-binaries", type=int, default=None,
                    help="run the differentiable measurement on its first N binaries only (profiling)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the step's stages one by one instead of as one CUDA graph")
    ap.add_argument("--tiling", default=None, metavar="WARPS,PERSISTENT,PACKED",
                    help="bank launch shape of the single-series plan instead of the autotuner (e.g. 4,0,1: 4 warps "
                         "per CTA, one CTA per tile, packed adds)")
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


def profile_traffic(kernel_src, workload):
    """DRAM bytes per launch of the bank kernel from the committed ncu summary
    of this workload, if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"boxcar_search_{workload}.md")
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
def oracle_fft_sample(name):
    """The oracle's FFT timed on a bounded sample of the workload's series: the
    whole series when it has at most FFT_PREFIX samples, else its first
    FFT_PREFIX samples, with the time scaled by N log2 N (the radix-2 FFT does
    log2 N stages of N / 2 butterflies).  Returns (spectrum of the sample, the
    scaled seconds for the whole series, description)."""
    from oracle import fft as offt
    from paper_2406_15186_gb300 import synth
    n = synth.WORKLOADS[name]["n"]
    n_p = min(n, FFT_PREFIX)
    x = synth.single_series_prefix(name, n_p)
    t0 = time.perf_counter()
    spec = offt.rfft(x.astype(np.float64))
    t = time.perf_counter() - t0
    scale = (n * math.log2(n)) / (n_p * math.log2(n_p))
    if n_p == n:
        desc = f"oracle FFT of the whole 2^{int(math.log2(n))}-sample series ({t:.1f} s, timed once, one core)"
    else:
        desc = (f"oracle FFT of the series' first 2^{int(math.log2(n_p))} samples ({t:.1f} s, one core), "
                f"scaled by N log2 N to 2^{int(math.log2(n))} ({t * scale:.1f} s)")
    return spec, t * scale, desc


def oracle_sample(spec, t_fft, fft_desc, cfg, n_seg_sample):
    """Time the FP64 oracle on a bounded sample, one core; returns (G bin-widths/s, seconds, description).

    Normalisation and the boxcar stage are linear in segments, so they are
    timed on the first n_seg_sample segments of the sampled spectrum and
    scaled to the whole series; the FFT time is added (t_fft).
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
    desc = (f"{fft_desc} + normalise/boxcar/search of {n_seg_sample} of its segments on one core, scaled "
            f"linearly to the {n_seg} segments of the series")
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


def oracle_parallel(spec, t_fft, fft_desc, cfg, seg_per_proc, procs):
    """The oracle on all host cores: processes (spawned, so no CUDA state is
    inherited) each run normalise + maxima + candidates on their own run of
    seg_per_proc segments of the sampled spectrum; wall time of the parallel
    pass, scaled linearly to all segments of the series, plus the FFT time."""
    import multiprocessing as mp
    n, w_max, seg_len, sigma = cfg["n"], cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    m = n // 2 + 1
    n_seg = m // seg_len
    avail = (len(spec) - w_max) // seg_len
    procs = max(1, min(procs, avail // seg_per_proc))
    nt = float(m) * w_max
    jobs = [(spec[i * seg_per_proc * seg_len: (i + 1) * seg_per_proc * seg_len + w_max], w_max, seg_len, sigma, nt,
             seg_per_proc) for i in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_segments, [(j[0][: seg_len + w_max], w_max, seg_len, sigma, nt, 1) for j in jobs])
        t0 = time.perf_counter()
        pool.map(_oracle_segments, jobs)
        t = time.perf_counter() - t0
    frac = procs * seg_per_proc / n_seg
    t_full = t_fft + t / frac
    desc = (f"{fft_desc} + normalise/boxcar/search of {procs * seg_per_proc} of its segments on {procs} "
            f"processes ({seg_per_proc} each, {t:.1f} s wall), scaled linearly to the {n_seg} segments of the "
            f"series")
    return m * w_max / t_full / 1e9, t, desc, procs


def run_reference(args, rank, world):
    """The oracle on the host cores: each step is one bounded sample of the
    workload -- normalise + maxima + candidates of one segment per process
    over a spawned pool of all host cores -- with the oracle FFT time (a
    sample scaled by N log2 N, timed once) added and the sample scaled to the
    series."""
    if rank != 0:
        return
    import multiprocessing as mp
    from paper_2406_15186_gb300 import synth
    name = args.workload
    cfg = synth.WORKLOADS[name]
    n, w_max, seg_len, sigma = cfg["n"], cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    m = n // 2 + 1
    n_seg = m // seg_len
    spec, t_fft, fft_desc = oracle_fft_sample(name)
    per = 1
    procs = max(1, min(host_cores(), (len(spec) - w_max) // seg_len))
    nt = float(m) * w_max
    jobs = [(spec[i * per * seg_len: (i + 1) * per * seg_len + w_max], w_max, seg_len, sigma, nt, per)
            for i in range(procs)]
    # one step = the sample: procs * per segments (their bins x widths), in
    # the wall time of the pool pass plus the same fraction of the FFT time
    frac = procs * per / n_seg
    step_s = []
    with mp.get_context("spawn").Pool(procs) as pool:
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_segments, jobs)
            t = time.perf_counter() - t0
            if i >= args.warmup:
                step_s.append(t + t_fft * frac)
    ms = statistics.mean(step_s) * 1e3
    value = frac * m * w_max / (ms * 1e-3) / 1e9
    desc = (f"{fft_desc} + normalise/boxcar/search of {procs * per} of its segments per step on {procs} "
            f"processes; a step is those segments' share ({frac:.3g}) of the series' bins x widths, in the pool "
            f"pass's wall time plus the same share of the FFT time")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_text(name), "sample": desc, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_text(name):
    from paper_2406_15186_gb300 import synth
    cfg = synth.WORKLOADS[name]
    n = cfg["n"]
    tones = {"single_2p27": "32 drifting tones", "single_2p23": "8 drifting tones",
             "single_2p20": "one drifting tone"}[name]
    return (f"{name}: N=2^{int(math.log2(n))} samples (M={n // 2 + 1} bins), {tones}, z_max={cfg['z_max']}, "
            f"segment_len={cfg['segment_len']}, sigma={cfg['sigma']:g}")


# ------------------------------------------------------------------ GPU arm
def run_batched(torch, pkg, synth, dev, stream, steps):
    """512 uneven DM-trial series: one graph replay vs per-series launches of
    the same kernels; also the graph pipelined over parts of the batch."""
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
    defer_warps = 1 if plan.defer_form() else 3

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
    # the same batch graph pipelined over parts of 2^26 bins (each part's FFT
    # and normalisation on a high-priority stream beside the previous part's bank)
    plan.set_pipeline(1 << 26)
    parts = plan.pipeline_parts()
    batched()
    t_q = timed(batched, steps)
    plan.set_pipeline(0)
    # and with normalisation and bank fused
    plan.set_fused(1)
    batched()
    t_f = timed(batched, steps)
    plan.set_fused(0)
    return {"workload": f"batch_512: 512 series, lengths U{{2^20..2^23}} (sum {sum(lengths)} samples, "
                        f"{bins} bins), 26 with a tone, z_max={w_max}, segment_len={seg_len}, sigma={sigma:g}",
            "dm_trials_per_s": len(lengths) / (t_b * 1e-3), "ms_per_batch": t_b,
            "per_series_dm_trials_per_s": len(lengths) / (t_s * 1e-3), "ms_per_series_loop": t_s,
            "ratio_batched_vs_per_series": t_s / t_b, "bin_widths_per_s": bins * w_max / (t_b * 1e-3) / 1e9,
            "ms_per_batch_pipelined": t_q, "pipeline_parts": parts, "ms_per_batch_fused": t_f,
            "bank_tiling": {"warps_per_cta": tiling[0], "persistent": tiling[1], "packed": tiling[2],
                            "by": "pulscan_plan_autotune", "deferred_warps_per_block": defer_warps},
            "unit": "G bin-widths/s", "candidates": n_cands, "graph": True,
            "per_series": "the same kernels launched per series on one stream (no graph), one plan per length",
            "l2": "inputs (8.2 GB) far larger than L2"}


def run_harmonic(torch, pkg, synth, dev, stream, x_dev, cfg, steps, flush):
    """The bench series searched with harmonic summing up to 4 harmonics (§2.3;
    numharm = 4 is the paper's setting in its timing runs)."""
    n, w_max, seg_len, sigma = cfg["n"], cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    numharm = 4
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma, numharm=numharm)
    with torch.cuda.stream(stream):
        d_x, d_spec, d_power = plan.buffers(dev)
        d_x.copy_(x_dev)
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
    ylo = torch.empty_like(y)
    gy = torch.ones_like(y)
    gx = torch.empty(plan.x_floats, **f32)
    gamp = torch.empty(n_series, **f32)

    def fwd():
        return lib.pulscan_lse_forward(plan._h, x.data_ptr(), spec.data_ptr(), power.data_ptr(), stats.data_ptr(),
                                       sel.data_ptr(), y.data_ptr(), ylo.data_ptr(), tau, sp)

    def bwd():
        rc = lib.pulscan_lse_backward(plan._h, spec.data_ptr(), power.data_ptr(), stats.data_ptr(), sel.data_ptr(),
                                      y.data_ptr(), ylo.data_ptr(), gy.data_ptr(), gx.data_ptr(), tau, sp)
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


def time_single(torch, pkg, synth, dev, stream, flush, name, args, steps, warmup, around=None):
    """One single-series workload: the whole path as one CUDA graph per step
    (or its stages one by one with --no-graph), the bank's launch shape by the
    autotuner (or --tiling), `warmup` untimed steps, then `steps` timed steps
    with the L2 flushed before each (outside the events); the bank kernel's
    own event pair is recorded inside every timed step.  around = (start,
    stop) callables bracketing the timed region (clock sampling, barriers).
    Then extra steps with every stage's events give the per-stage breakdown.
    Returns (result dict, plan, (d_x, d_spec, d_power))."""
    cfg = synth.WORKLOADS[name]
    n, w_max, seg_len, sigma = cfg["n"], cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    m = n // 2 + 1
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    with torch.cuda.stream(stream):
        d_x, d_spec, d_power = plan.buffers(dev)
        synth.single_series_device(name, d_x)
    torch.cuda.synchronize()
    # the timed steps record only the bank kernel's event pair (the roofline's
    # live kernel time): every event between two kernels drains the pipeline
    # and adds a few microseconds
    plan.enable_timing(2)

    def step():
        if args.no_graph:
            plan.rfft(d_x, d_spec, stream=stream)
            plan.power_normalise(d_spec, d_power, stream=stream)
            plan.boxcar_search(d_power, stream=stream)
        else:
            plan.search(d_x, d_spec, d_power, use_graph=True, stream=stream)

    step()
    if args.tiling:
        plan.set_tiling(*[int(v) for v in args.tiling.split(",")])
        tiling, tiling_by = plan.tiling(), "--tiling"
    else:
        tiling = plan.autotune(d_power, stream=stream)     # launch shape of the bank, timed on this input
        tiling_by = "pulscan_plan_autotune"
    for _ in range(warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        step()
    n_cands = len(plan.candidates(stream=stream))
    n_deferred = plan.counters()[0]
    extra = around[0]() if around else None
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    k_bank_live = []
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()                       # L2 flushed between timed steps (outside the events)
            ev[i][0].record(stream)
        step()
        with torch.cuda.stream(stream):
            ev[i][1].record(stream)
        k_bank_live.append(plan.timings()[2])  # the bank kernel's events in this step (same stream)
    torch.cuda.synchronize()
    clocks = around[1](extra) if around else None
    step_ms = [a.elapsed_time(b) for a, b in ev]

    plan.enable_timing(True)
    step()
    n_break = max(5, steps // 2)
    k = {key: [] for key in ("rfft_cufft", "normalise", "boxcar_search", "deferred_blocks", "finalise")}
    break_ms = []
    for _ in range(n_break):
        with torch.cuda.stream(stream):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        step()
        with torch.cuda.stream(stream):
            e1.record(stream)
        t = plan.timings()
        for key, idx in zip(k, (0, 1, 2, 3, 4)):
            k[key].append(t[idx])
        torch.cuda.synchronize()
        break_ms.append(e0.elapsed_time(e1))
    plan.enable_timing(False)
    kernels = {key: statistics.mean(v) for key, v in k.items()}
    kernels["boxcar_search_live"] = statistics.mean(k_bank_live)
    kernels["note"] = (f"per-stage events from {n_break} extra steps recording every stage "
                       f"({statistics.mean(break_ms):.4f} ms per step with those events); boxcar_search_live: "
                       "the bank's own event pair inside the timed steps (the roofline's time)")
    res = {"workload": workload_text(name), "m": m, "w_max": w_max, "step_ms": step_ms,
           "ms_per_step": statistics.mean(step_ms), "kernels_ms": kernels, "candidates": n_cands,
           "deferred_blocks": n_deferred, "clocks": clocks,
           "bank_tiling": {"warps_per_cta": tiling[0], "persistent": tiling[1], "packed": tiling[2], "by": tiling_by,
                           "deferred_warps_per_block": 1 if plan.defer_form() else 3}}
    return res, plan, (d_x, d_spec, d_power)


def time_fused(torch, plan, bufs, stream, flush, steps, sep_ms):
    """The same search step with normalisation and bank fused (pulscan_plan_set_fused:
    block statistics only, then P formed from the spectrum inside the bank and the
    deferred blocks), as one CUDA graph per step, L2 flushed before each step;
    against sep_ms, the separate stages' step."""
    plan.set_fused(1)
    step = lambda: plan.search(*bufs, use_graph=True, stream=stream)
    for _ in range(3):
        step()
    ms = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    n_cands = len(plan.candidates(stream=stream))
    plan.set_fused(0)
    t = statistics.mean(ms)
    return {"ms_per_step": t, "separate_ms_per_step": sep_ms, "ratio_separate_over_fused": sep_ms / t,
            "candidates": n_cands, "kept": t < sep_ms,
            "note": "fused normalise + boxcar (f4): statistics kernel, then the bank forms P from the spectrum; "
                    "off by default where slower"}


def rooflines(res, peak, n_sm, sm_max, name):
    """roofline (the bank kernel alone, its live events) and roofline_search
    (bank + deferred blocks + finaliser, the per-stage events) against the
    FP32 add rate measured in this run; the derived rate (SMs x 128 FP32
    lanes x the maximum SM clock) is reported beside it."""
    m, w_max = res["m"], res["w_max"]
    adds = m * (w_max - 1)                  # sum_{w=2}^{W} (M - w + 1) ~ M (W - 1): one add per bin and width
    kn = res["kernels_ms"]
    p = peak["packed_adds_per_s"] / 1e12
    derived = n_sm * 128 * sm_max * 1e6 / 1e12
    ach = adds / (kn["boxcar_search_live"] * 1e-3) / 1e12
    t_search = kn["boxcar_search"] + kn["deferred_blocks"] + kn["finalise"]
    ach_s = adds / (t_search * 1e-3) / 1e12
    src = os.path.join(ROOT, "paper_2406_15186_gb300", "csrc", "boxcar.cu")
    bank = {"bound": "alu", "achieved": ach, "peak": p, "unit": "TFLOP/s", "frac": ach / p,
            "traffic": profile_traffic(src, name), "kernel": "boxcar_kernel<search>",
            "algorithmic": f"M (W - 1) = {adds:.4g} FP32 adds per launch, 4 M = {4 * m:.4g} bytes read",
            "peak_source": (f"pulscan_measure_add_peak in this run: packed f32x2 adds at "
                            f"{peak['packed_sm_mhz']:.0f} MHz (scalar adds: "
                            f"{peak['scalar_adds_per_s'] / 1e12:.2f} T/s)"),
            "peak_derived": derived, "frac_of_derived": ach / derived,
            "peak_derived_source": f"{n_sm} SMs x 128 FP32 lanes x {sm_max:.0f} MHz (sm_max_mhz)"}
    search = {"bound": "alu", "achieved": ach_s, "peak": p, "unit": "TFLOP/s", "frac": ach_s / p,
              "kernels": "boxcar_kernel<search> + " + (
                  "deferred_warp_kernel" if res["bank_tiling"].get("deferred_warps_per_block") == 1
                  else "deferred_kernel") + " + word_scan_kernel + finalize_kernel",
              "time_ms": t_search, "time_source": "per-stage events of the breakdown steps"}
    return bank, search


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

    if args.only_diff:
        r = run_diff(torch, pkg, synth, dev, torch.cuda.Stream(device=dev), 3, args.diff_binaries)
        if rank == 0:
            print(json.dumps({"differentiable": r}), flush=True)
        return
    name = args.workload
    cfg = synth.WORKLOADS[name]
    n, w_max, seg_len, sigma = cfg["n"], cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    m = n // 2 + 1
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    if args.only_fidelity:
        plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
        with torch.cuda.stream(stream):
            bufs = plan.buffers(dev)
            synth.single_series_device(name, bufs[0])
        torch.cuda.synchronize()

        def fstep():
            plan.search(*bufs, use_graph=True, stream=stream)

        fstep()
        if args.tiling:
            plan.set_tiling(*[int(v) for v in args.tiling.split(",")])
        else:
            plan.autotune(bufs[2], stream=stream)
        plan.enable_timing(True)
        r = run_fidelity(torch, pkg, plan, fstep, stream, max(3, args.steps // 2), flush)
        if rank == 0:
            print(json.dumps({"paper_gpu_fidelity": dict(r, workload=name, bank_tiling=plan.tiling())}), flush=True)
        plan.close()
        return
    props = torch.cuda.get_device_properties(dev)
    peaks, peak_kind = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)

    # the FP32 add rate of this GPU, measured now (the bank's roofline)
    add_peak = pkg.measure_add_peak(reps=5, stream=stream)
    sampler = ClockSampler(local)

    def start():
        sampler.start()
        time.sleep(0.3)
        if dist:
            dist.barrier()

    def stop(_):
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return sampler.stop()

    head, plan, (d_x, d_spec, d_power) = time_single(torch, pkg, synth, dev, stream, flush, name, args, args.steps,
                                                     args.warmup, around=(start, stop))
    ms = max_over_ranks(head["ms_per_step"], dist, dev)
    value = job_value(world, m * w_max, ms)
    roof, roof_search = rooflines(head, add_peak, props.multi_processor_count, sm_max, name)
    tiling = (head["bank_tiling"]["warps_per_cta"], head["bank_tiling"]["persistent"], head["bank_tiling"]["packed"])

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": head["workload"],
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "bank_tiling": head["bank_tiling"],
                       "input": "noise from torch's seeded device generator plus the workload's tones (FP64 "
                                "phase), drawn on the device",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "kernels_ms": head["kernels_ms"], "candidates": head["candidates"],
            "deferred_blocks": head["deferred_blocks"],
            "roofline": roof, "roofline_search": roof_search,
            "fp32_add_peak": {"packed_T_per_s": add_peak["packed_adds_per_s"] / 1e12,
                              "scalar_T_per_s": add_peak["scalar_adds_per_s"] / 1e12,
                              "packed_sm_mhz": add_peak["packed_sm_mhz"], "scalar_sm_mhz": add_peak["scalar_sm_mhz"],
                              "derived_T_per_s": props.multi_processor_count * 128 * sm_max * 1e6 / 1e12,
                              "sm_max_mhz_source": peak_kind},
            # this library's kernels per step: normalise, bank, deferred
            # blocks, word scan, finaliser (cuFFT's own kernels not counted)
            "gpu_launches": 5 * args.steps,
            "clocks": head["clocks"]}

    if not args.only_headline:
        # end to end through the host-buffer entry points, as a stream of
        # series: two plans in turn on two streams (double buffering), so one
        # series' copy to the device runs while the previous one's search
        # does.  Every step has its H2D copy of the series from pinned memory
        # and its D2H read of candidates; a series smaller than L2 also gets
        # its own L2 flush (on its stream, before its copy), while a larger
        # one (the 2^27-sample series: 512 MiB) already starts cold.
        x_host = d_x.cpu()
        plan_b = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
        plan_b.set_tiling(*tiling)
        plans, streams = [plan, plan_b], [stream, torch.cuda.Stream(device=dev)]
        x_pin = [x_host.pin_memory(), x_host.clone().pin_memory()]
        cap = min(plan.max_candidates, 1 << 20)

        e2e_flush = 4 * n <= L2_BYTES

        def issue(i):
            k = i % 2
            if e2e_flush:
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
        e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / n_e2e, dist, dev)
        plan_b.close()
        del x_pin, x_host
        line["e2e"] = {"value": job_value(world, m * w_max, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
                       "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 16 + 32 * nc, "steps": n_e2e,
                       "pipeline": "pulscan_search_host_async + pulscan_candidates on two plans and two streams "
                                   "in turn (a series' copy overlaps the previous search); wall clock over all steps",
                       "l2": (f"flushed on each step's stream before its copy" if e2e_flush else
                              f"not flushed: each step's input ({4 * n / 2**20:.0f} MiB, copied from the host) "
                              f"is larger than L2")}
    plan.close()
    del d_x, d_spec, d_power
    torch.cuda.empty_cache()

    if not args.only_headline:
        # the other single-series workloads, each with its own roofline
        for other in EXTRA_SINGLE:
            if other == name:
                continue
            r, p2, bufs = time_single(torch, pkg, synth, dev, stream, flush, other, args, args.steps, args.warmup)
            b, sr = rooflines(r, add_peak, props.multi_processor_count, sm_max, other)
            om = r["m"] * r["w_max"]
            line[other] = {"workload": r["workload"], "value": om / (r["ms_per_step"] * 1e-3) / 1e9, "unit": UNIT,
                           "ms_per_step": r["ms_per_step"], "kernels_ms": r["kernels_ms"],
                           "candidates": r["candidates"], "deferred_blocks": r["deferred_blocks"],
                           "bank_tiling": r["bank_tiling"], "roofline": b, "roofline_search": sr}
            if other == "single_2p23":
                line[other]["fused"] = time_fused(torch, p2, bufs, stream, flush, max(5, args.steps // 2),
                                                  r["ms_per_step"])
                # f1-f3 on this series: harmonic sums, the paper-GPU fidelity
                # mode, and the searched-width subsets
                d_x2 = bufs[0]
                sub_steps = max(3, args.steps // 2)
                ocfg = synth.WORKLOADS[other]
                p2.enable_timing(True)

                def step2():
                    p2.search(*bufs, use_graph=True, stream=stream)

                sampling = {}
                for sname, mode, stp in (("step8", 1, 8), ("log2", 2, 1)):
                    p2.set_widths(mode, stp)
                    step2()
                    ts = []
                    for _ in range(sub_steps):
                        with torch.cuda.stream(stream):
                            flush.zero_()
                        step2()
                        t = p2.timings()
                        ts.append(t[2] + t[3] + t[4])
                    sampling[sname] = {"search_ms": statistics.mean(ts),
                                       "candidates": len(p2.candidates(stream=stream))}
                p2.set_widths(0, 1)
                kn = r["kernels_ms"]
                sampling["all"] = {"search_ms": kn["boxcar_search"] + kn["deferred_blocks"] + kn["finalise"],
                                   "candidates": r["candidates"]}
                line["width_sampling"] = dict(sampling, workload=other,
                                              note="boxcar + deferred + finalise per step; all widths summed, only "
                                                   "the sampled ones compared (z mod 8 == 0; z a power of two)")
                line["harmonics"] = run_harmonic(torch, pkg, synth, dev, stream, d_x2, ocfg, sub_steps, flush)
                line["paper_gpu_fidelity"] = run_fidelity(torch, pkg, p2, step2, stream, sub_steps, flush)
            p2.close()
            del bufs
            torch.cuda.empty_cache()
    if not args.no_batched and not args.only_headline:
        line["batched"] = run_batched(torch, pkg, synth, dev, stream, max(3, args.steps // 4))
        torch.cuda.empty_cache()
    if not args.no_diff and not args.only_headline:
        line["differentiable"] = run_diff(torch, pkg, synth, dev, stream, 3, args.diff_binaries)
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.only_headline:
        spec, t_fft, fft_desc = oracle_fft_sample(name)
        v1, secs, desc1 = oracle_sample(spec, t_fft, fft_desc, cfg, 4)
        vp, secs_p, desc_p, procs = oracle_parallel(spec, t_fft, fft_desc, cfg, 2, host_cores())
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
