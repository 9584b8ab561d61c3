"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: white Gaussian noise and injected drifting
(chirped, optionally jerked) sinusoids.  It holds none of the search method's
arithmetic and is the one module that both the CUDA path's tests/bench and
the FP64 oracle receive their inputs from (the oracle never imports it; the
caller passes it the same arrays).  It does not load the CUDA library.

Signal model (paper §2.1, Eq. 1, with the jerk term of §2.1 for FDJS):
x[n] += A cos(2 pi (r0 u + z u^2 / 2 + w u^3 / 6) + phi0), u = n / N, so the
instantaneous frequency starts at Fourier bin r0 and drifts by z bins over
the observation (plus a w-bin change of drift).  The phase is formed in FP64
and the sum is cast to float32.

The paper's SIGPROC/PRESTO datasets are not available; these stand in for
them (noise mean 0, sd 1, seed = 1000 * workload + series).
"""
import numpy as np

# The five workloads: sizes, widths, segment lengths, thresholds.
WORKLOADS = {
    # one series, 2^20 samples, one tone at bin 1e5 drifting 50 bins
    "single_2p20": dict(id=1, n=1 << 20, z_max=256, segment_len=1024, sigma=6.0),
    # SPOTLIGHT-scale single series, 8 tones
    "single_2p23": dict(id=2, n=1 << 23, z_max=1024, segment_len=4096, sigma=6.0),
    # 512 DM-trial series of uneven length 2^20..2^23
    "batch_512": dict(id=3, n_series=512, lengths=(1 << 20, 1 << 21, 1 << 22, 1 << 23),
                      z_max=512, segment_len=2048, sigma=6.0),
    # differentiable: 4096 binaries of 2^20 samples, logsumexp at tau 0.1
    "diff_4096": dict(id=4, n_series=4096, n=1 << 20, z_max=512, segment_len=2048, tau=0.1),
    # large single series, 2^27 samples, 32 tones
    "single_2p27": dict(id=5, n=1 << 27, z_max=4096, segment_len=16384, sigma=7.0),
}


def seed_of(workload_id, series=0):
    return 1000 * int(workload_id) + int(series)


def noise(n, seed):
    """Unit-variance white Gaussian noise, float32."""
    return np.random.default_rng(seed).standard_normal(int(n), dtype=np.float32)


def chirp(n, r0, z, w=0.0, phi0=0.0):
    """Unit-amplitude drifting sinusoid (FP64)."""
    u = np.arange(int(n), dtype=np.float64) / float(n)
    phase = r0 * u + 0.5 * z * u * u + (w / 6.0) * u * u * u
    return np.cos(2.0 * np.pi * phase + phi0)


def tone_params(rng, n, k, z_hi, a_lo=0.01, a_hi=0.1, w_lo=0.0, w_hi=0.0, r_lo=1.0e4, r_hi=None):
    """k tone parameter dicts drawn uniformly from ``rng``."""
    if r_hi is None:
        r_hi = 0.9 * (n // 2)
    out = []
    for _ in range(k):
        out.append(dict(amp=float(rng.uniform(a_lo, a_hi)), r0=float(rng.uniform(r_lo, r_hi)),
                        z=float(rng.uniform(0.0, z_hi)), w=float(rng.uniform(w_lo, w_hi)),
                        phi0=float(rng.uniform(0.0, 2.0 * np.pi))))
    return out


def inject(x, tones):
    """x + sum of tones, computed in FP64 and cast back to float32."""
    n = x.shape[0]
    acc = x.astype(np.float64)
    for t in tones:
        acc += t["amp"] * chirp(n, t["r0"], t["z"], t.get("w", 0.0), t.get("phi0", 0.0))
    return acc.astype(np.float32)


def single_tones(name, n=None):
    """The injected tones of one of the single-series workloads."""
    cfg = WORKLOADS[name]
    n = int(cfg["n"] if n is None else n)
    rng = np.random.default_rng(seed_of(cfg["id"]) + 500_000)
    if name == "single_2p20":
        return [dict(amp=0.05, r0=min(100000.0, 0.4 * n), z=50.0, w=0.0,
                     phi0=float(rng.uniform(0.0, 2.0 * np.pi)))]
    if name == "single_2p23":
        return tone_params(rng, n, 8, 800.0)
    if name == "single_2p27":
        return tone_params(rng, n, 32, 4000.0)
    raise KeyError(name)


def single_series(name, n=None):
    """(x, tones) for one of the single-series workloads.

    ``n`` overrides the length (for small test cases of the same recipe).
    """
    cfg = WORKLOADS[name]
    n = int(cfg["n"] if n is None else n)
    tones = single_tones(name, n)
    return inject(noise(n, seed_of(cfg["id"])), tones), tones


def single_series_prefix(name, n_prefix):
    """The first n_prefix samples of a single-series workload drawn on the
    host (noise of the workload's seed, tones with u = n / N of the full
    length N), for timing samples of a series too long to draw whole."""
    cfg = WORKLOADS[name]
    n = int(cfg["n"])
    u = np.arange(int(n_prefix), dtype=np.float64) / float(n)
    acc = noise(n_prefix, seed_of(cfg["id"])).astype(np.float64)
    for t in single_tones(name):
        ph = t["r0"] * u + 0.5 * t["z"] * u * u + (t.get("w", 0.0) / 6.0) * u * u * u
        acc += t["amp"] * np.cos(2.0 * np.pi * ph + t.get("phi0", 0.0))
    return acc.astype(np.float32)


def batch_lengths(n_series=512, lengths=(1 << 20, 1 << 21, 1 << 22, 1 << 23), seed=None):
    """Uneven series lengths drawn uniformly from ``lengths``."""
    rng = np.random.default_rng(seed_of(3) + 900_000 if seed is None else seed)
    return [int(lengths[i]) for i in rng.integers(0, len(lengths), size=n_series)]


def batch_series(i, n, with_tone):
    """Series i of the DM-trial batch (noise, plus one tone if ``with_tone``)."""
    seed = seed_of(3, i)
    x = noise(n, seed)
    if not with_tone:
        return x, []
    rng = np.random.default_rng(seed + 500_000)
    tones = tone_params(rng, n, 1, 500.0)
    return inject(x, tones), tones


def batch_tone_mask(n_series=512, frac=0.05):
    """Which series of the batch carry an injected tone (5% by default)."""
    rng = np.random.default_rng(seed_of(3) + 700_000)
    k = int(round(frac * n_series))
    mask = np.zeros(n_series, dtype=bool)
    mask[rng.choice(n_series, size=k, replace=False)] = True
    return mask


def binary_params(i, n=1 << 20):
    """Spin bin, drift and jerk of binary i of the differentiable workload."""
    rng = np.random.default_rng(seed_of(4, i) + 500_000)
    return dict(r0=float(rng.uniform(1.0e4, 4.0e5)), z=float(rng.uniform(0.0, 300.0)),
                w=float(rng.uniform(-600.0, 600.0)), phi0=float(rng.uniform(0.0, 2.0 * np.pi)),
                amp=float(np.exp(rng.uniform(np.log(0.01), np.log(0.1)))))


# ---------------------------------------------------------------- on the GPU
# Large workloads (the DM-trial batch, the big single series, the
# differentiable batch) are drawn directly on the device: torch's seeded
# Philox generator for the noise and FP64 chirps, cast to float32.  Tests that
# compare with the oracle copy the sampled series back to the host, so both
# sides see the same bytes.

def device_noise(total, seed, device="cuda"):
    """float32[total] standard normal noise from a seeded device generator."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return torch.randn(int(total), generator=g, device=device, dtype=torch.float32)


def device_inject(x, tones):
    """x += sum of tones in place (FP64 phase on the device, cast to float32)."""
    import torch
    n = x.shape[0]
    u = torch.arange(n, device=x.device, dtype=torch.float64) / float(n)
    acc = x.to(torch.float64)
    for t in tones:
        ph = t["r0"] * u + 0.5 * t["z"] * u * u + (t.get("w", 0.0) / 6.0) * u * u * u
        acc += t["amp"] * torch.cos(2.0 * np.pi * ph + t.get("phi0", 0.0))
    x.copy_(acc.to(torch.float32))
    return x


def single_series_device(name, x):
    """Fill x (device, float32[N]) with a single-series workload: noise from
    the device generator seeded with the workload's seed, plus the
    workload's tones (the same draws as single_series)."""
    cfg = WORKLOADS[name]
    x.copy_(device_noise(int(cfg["n"]), seed_of(cfg["id"]), device=x.device))
    return device_inject(x, single_tones(name))


def batch_device(x_all, offsets, lengths, tone_mask, workload_id=3):
    """Fill x_all (device, float32) with the DM-trial batch at the given offsets."""
    tones_of = {}
    for i, n in enumerate(lengths):
        seg = x_all[int(offsets[i]): int(offsets[i]) + int(n)]
        seg.copy_(device_noise(n, seed_of(workload_id, i), device=x_all.device))
        if tone_mask[i]:
            rng = np.random.default_rng(seed_of(workload_id, i) + 500_000)
            tones = tone_params(rng, n, 1, 500.0)
            device_inject(seg, tones)
            tones_of[i] = tones
    return tones_of


def diff_device(noise, template, offsets, n, n_series, workload_id=4):
    """Fill the differentiable workload on the device: per binary i, noise and
    its unit-amplitude template (spin bin, drift z and jerk w from
    binary_params); returns the amplitudes (float32 numpy, log-uniform
    0.01-0.1)."""
    import torch
    amps = np.zeros(n_series, dtype=np.float32)
    u = torch.arange(int(n), device=noise.device, dtype=torch.float64) / float(n)
    for i in range(n_series):
        o = int(offsets[i])
        noise[o: o + n].copy_(device_noise(n, seed_of(workload_id, i), device=noise.device))
        b = binary_params(i, n)
        ph = b["r0"] * u + 0.5 * b["z"] * u * u + (b["w"] / 6.0) * u * u * u
        template[o: o + n].copy_(torch.cos(2.0 * np.pi * ph + b["phi0"]).to(torch.float32))
        amps[i] = b["amp"]
    return amps
