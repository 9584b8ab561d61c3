"""GPU parity at the workloads' full sizes, on outputs the oracle can afford.

* single_2p23 (the bench workload, bench launch configuration): everything,
  from the raw series, with the oracle's own FFT (stage C).
* batch_512: the whole batch in one graph replay; sampled series checked
  (stage A and B on their GPU intermediates, candidates).
* single_2p27: sampled segments (stage A and B), FFT checked on sampled bins
  against the DFT definition.
* diff_4096: the whole batch forward and backward through torch.autograd;
  sampled binaries checked against the oracle's logsumexp and adjoint.
"""
import math

import numpy as np
import pytest

from oracle import boxcar as obox
from oracle import fft as offt
from oracle import normalise as onorm
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


def test_single_2p23_full(pkg):
    cfg = synth.WORKLOADS["single_2p23"]
    n, w_max, seg_len, sigma = cfg["n"], cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    x, tones = synth.single_series("single_2p23")
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    out = parity.run_gpu(plan, x, stats=True, use_graph=True)
    m = n // 2 + 1
    ref_spec = offt.rfft(x.astype(np.float64))
    gspec = parity.spectrum_complex(out["spec"], 0, m)
    assert np.linalg.norm(gspec - ref_spec) / np.linalg.norm(ref_spec) <= 1e-6 * math.log2(n)
    parity.check_normalise(gspec, out["power"][:m], out["stats"], seg_len)
    p64 = out["power"][:m].astype(np.float64)
    parity.check_maxima(p64, out["mx"], out["am"], w_max, seg_len)
    # stage C: the oracle's FP64 path from the raw series
    p_ref, _, _ = onorm.normalise_power(ref_spec, seg_len)
    mx_ref, am_ref = obox.segment_maxima(p_ref, w_max, seg_len)
    k = parity.check_candidates(out["cands"], p_ref, mx_ref, am_ref, w_max, seg_len, sigma,
                                parity.n_trials_of(m, w_max))
    assert k > 100
    # every injected tone is detected near its spin bin
    c = out["cands"]
    for t in tones:
        if t["amp"] < 0.03:
            continue
        near = c[(c["bin"] >= t["r0"] - w_max) & (c["bin"] <= t["r0"] + t["z"] + 1)]
        assert len(near) > 0, t


def _sample_rows(n_seg, rng, k, must=()):
    rows = set(int(r) for r in must if 0 <= r < n_seg)
    rows |= set(int(r) for r in rng.choice(n_seg, size=min(k, n_seg), replace=False))
    rows.add(0)
    rows.add(n_seg - 1)
    return sorted(rows)


def test_batch_512_sampled(pkg):
    cfg = synth.WORKLOADS["batch_512"]
    w_max, seg_len, sigma = cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    lengths = synth.batch_lengths(cfg["n_series"], cfg["lengths"])
    mask = synth.batch_tone_mask(cfg["n_series"])
    plan = pkg.Plan(lengths=lengths, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    xo, so, po, go = plan.offsets()
    d_x, d_spec, d_power = plan.buffers()
    tones = synth.batch_device(d_x, xo, lengths, mask)
    d_stats = torch.zeros(4 * plan.total_segments, dtype=torch.float32, device="cuda")
    plan.search(d_x, d_spec, d_power, use_graph=True)
    cands = plan.candidates()
    plan.power_normalise(d_spec, d_power, d_stats)   # statistics of the same spectra
    torch.cuda.synchronize()
    assert len(cands) > 0
    # the series with injected tones are found
    found = set(int(s) for s in np.unique(cands["series"]))
    strong = [i for i, t in tones.items() if t[0]["amp"] >= 0.05]
    assert all(i in found for i in strong)
    n_all = plan.total_segments * w_max
    mx = torch.empty(n_all, dtype=torch.float32, device="cuda")
    am = torch.empty(n_all, dtype=torch.int64, device="cuda")
    plan.segment_maxima(d_power, mx, am)
    all_mx = mx.cpu().numpy().reshape(plan.total_segments, w_max)
    all_am = am.cpu().numpy().reshape(plan.total_segments, w_max)
    del mx, am
    rng = np.random.default_rng(5)
    picks = [lengths.index(L) for L in sorted(set(lengths))] + sorted(tones)[:2]
    for i in picks:
        n = lengths[i]
        m = n // 2 + 1
        n_seg = max(1, m // seg_len)
        spec = d_spec[2 * so[i]: 2 * (so[i] + m)].cpu().numpy()
        p = d_power[po[i]: po[i] + m].cpu().numpy()
        st = d_stats[4 * go[i]: 4 * (go[i] + n_seg)].cpu().numpy().reshape(-1, 4)
        rows = _sample_rows(n_seg, rng, 6, must=[int(t["r0"]) // seg_len for t in tones.get(i, [])])
        # stage A on the sampled segments
        z = parity.spectrum_complex(spec, 0, m)
        for r in rows:
            lo_, hi_ = r * seg_len, (m if r == n_seg - 1 else (r + 1) * seg_len)
            blk = z[lo_:hi_].copy()
            if r == 0:
                blk[0] = 0.0          # the DC bin is taken as 0
            ref_stats = [onorm.median(blk.real), 0, onorm.median(blk.imag), 0]
            assert st[r, 0] == pytest.approx(ref_stats[0], rel=2 ** -22, abs=1e-6 * (1 + abs(st[r, 1])))
            assert st[r, 2] == pytest.approx(ref_stats[2], rel=2 ** -22, abs=1e-6 * (1 + abs(st[r, 3])))
            mad_re = onorm.mad(blk.real, ref_stats[0])
            assert st[r, 1] == pytest.approx(mad_re, rel=1e-6)
            a = (blk.real - ref_stats[0]) / (onorm.KAPPA * mad_re)
            mad_im = onorm.mad(blk.imag, ref_stats[2])
            b = (blk.imag - ref_stats[2]) / (onorm.KAPPA * mad_im)
            pref = 0.5 * (a * a + b * b)
            assert np.max(np.abs(p[lo_:hi_] - pref) / np.maximum(pref, 1.0)) <= parity.P_TOL
        # stage B and candidates on the sampled segments
        p64 = p.astype(np.float64)
        gmx = all_mx[go[i]: go[i] + n_seg]
        gam = all_am[go[i]: go[i] + n_seg]
        for r in rows:
            mx_ref, am_ref = parity.check_maxima(p64, gmx, gam, w_max, seg_len, seg_range=(r, r + 1))
            parity.check_candidates(cands, p64, mx_ref, am_ref, w_max, seg_len, sigma,
                                    parity.n_trials_of(m, w_max), series=i, seg_rows=(r, r + 1))


def test_single_2p27_sampled(pkg):
    cfg = synth.WORKLOADS["single_2p27"]
    n, w_max, seg_len, sigma = cfg["n"], cfg["z_max"], cfg["segment_len"], cfg["sigma"]
    m = n // 2 + 1
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    d_x, d_spec, d_power = plan.buffers()
    d_x.copy_(synth.device_noise(n, synth.seed_of(5)))
    rng = np.random.default_rng(synth.seed_of(5) + 500_000)
    tones = synth.tone_params(rng, n, 32, 4000.0)
    synth.device_inject(d_x, tones)
    d_stats = torch.zeros(4 * plan.total_segments, dtype=torch.float32, device="cuda")
    plan.rfft(d_x, d_spec)
    plan.power_normalise(d_spec, d_power, d_stats)
    plan.boxcar_search(d_power)
    cands = plan.candidates()
    n_mx = plan.total_segments * w_max
    mx = torch.empty(n_mx, dtype=torch.float32, device="cuda")
    am = torch.empty(n_mx, dtype=torch.int64, device="cuda")
    plan.segment_maxima(d_power, mx, am)
    torch.cuda.synchronize()
    x = d_x.cpu().numpy()
    spec = parity.spectrum_complex(d_spec.cpu().numpy(), 0, m)
    # FFT on sampled bins against the DFT definition
    bins = [1, int(tones[0]["r0"]), m // 3, m - 1]
    ref = offt.dft_bins(x.astype(np.float64), bins)
    rms = math.sqrt(n / 2.0)
    assert np.max(np.abs(spec[bins] - ref)) <= 1e-6 * math.log2(n) * max(rms, np.max(np.abs(ref)) * 1e-3)
    p = d_power.cpu().numpy()
    st = d_stats.cpu().numpy().reshape(-1, 4)
    gmx = mx.cpu().numpy().reshape(plan.total_segments, w_max)
    gam = am.cpu().numpy().reshape(plan.total_segments, w_max)
    n_seg = plan.total_segments
    rows = _sample_rows(n_seg, np.random.default_rng(7), 4, must=[int(t["r0"]) // seg_len for t in tones[:3]])
    p64 = p.astype(np.float64)
    for r in rows:
        lo_, hi_ = r * seg_len, (m if r == n_seg - 1 else (r + 1) * seg_len)
        blk = spec[lo_:hi_].copy()
        if r == 0:
            blk[0] = 0.0
        med_re, med_im = onorm.median(blk.real), onorm.median(blk.imag)
        mad_re, mad_im = onorm.mad(blk.real, med_re), onorm.mad(blk.imag, med_im)
        assert st[r, 1] == pytest.approx(mad_re, rel=1e-6) and st[r, 3] == pytest.approx(mad_im, rel=1e-6)
        a = (blk.real - med_re) / (onorm.KAPPA * mad_re)
        b = (blk.imag - med_im) / (onorm.KAPPA * mad_im)
        pref = 0.5 * (a * a + b * b)
        assert np.max(np.abs(p[lo_:hi_] - pref) / np.maximum(pref, 1.0)) <= parity.P_TOL
        mx_ref, am_ref = parity.check_maxima(p64, gmx, gam, w_max, seg_len, seg_range=(r, r + 1))
        parity.check_candidates(cands, p64, mx_ref, am_ref, w_max, seg_len, sigma, parity.n_trials_of(m, w_max),
                                seg_rows=(r, r + 1))



def test_diff_4096_sampled(pkg):
    """The differentiable batch at full size (4096 x 2^20, widths 1..512, L =
    2048, tau = 0.1) forward and backward through torch.autograd; binaries 0
    and 4095 against the oracle, taken from the GPU's own spectrum of the
    same float32 x (the median / MAD derivatives sit on selected order
    statistics, and an FP32 and an FP64 spectrum of the same x can select
    different elements where two deviations are within rounding of each
    other -- binary 4095 has one such block -- which would move a whole
    block's MAD term to another bin).

    Y to 1e-5 * max(|Y|, w) against the oracle's logsumexp of its power of
    that spectrum; dL/dx to rel-L2 1e-4 against the oracle's adjoint; dL/dA
    against the oracle's dL/dA (its dL/dx on the template) to
    1e-4 ||dL/dx|| ||template|| (Cauchy-Schwarz).  The FP64 chain from x
    itself (oracle FFT and medians) is checked on Y at 1e-4 * max(|Y|, w)."""
    from oracle import lse as olse
    from oracle import normalise as onorm
    from paper_2406_15186_gb300 import lse
    cfg = synth.WORKLOADS["diff_4096"]
    n, n_series, w_max, seg_len, tau = cfg["n"], cfg["n_series"], cfg["z_max"], cfg["segment_len"], cfg["tau"]
    m = n // 2 + 1
    plan = pkg.Plan(lengths=[n] * n_series, z_max=w_max, segment_len=seg_len, threshold_sigma=6.0)
    xo, so, _, go = plan.offsets()
    noise = torch.empty(plan.x_floats, device="cuda")
    tmpl = torch.empty(plan.x_floats, device="cuda")
    amps = synth.diff_device(noise, tmpl, xo, n, n_series)
    amp = torch.from_numpy(amps).cuda().requires_grad_(True)
    x = lse.inject(noise, tmpl, amp, plan)
    x.retain_grad()
    y = lse.lse_statistic(x, plan, tau)
    g = torch.Generator(device="cuda")
    g.manual_seed(4044)
    gy = torch.randn(tuple(y.shape), generator=g, device="cuda")
    (y * gy).sum().backward()
    torch.cuda.synchronize()
    assert torch.isfinite(y).all() and torch.isfinite(amp.grad).all() and torch.isfinite(x.grad).all()
    del noise
    spec = torch.empty(plan.spec_floats, device="cuda")
    plan.rfft(x.detach(), spec)
    torch.cuda.synchronize()
    n_seg = m // seg_len
    w = np.arange(1, w_max + 1)[None, :]
    ga_gpu = amp.grad.cpu().numpy().astype(np.float64)
    for i in (0, n_series - 1):
        xi = x.detach()[xo[i]: xo[i] + n].cpu().numpy().astype(np.float64)
        ti = tmpl[xo[i]: xo[i] + n].cpu().numpy().astype(np.float64)
        yi = y.detach()[go[i]: go[i] + n_seg].cpu().numpy().astype(np.float64)
        gyi = gy[go[i]: go[i] + n_seg].cpu().numpy().astype(np.float64)
        gxi = x.grad[xo[i]: xo[i] + n].cpu().numpy().astype(np.float64)
        y_x, _ = olse.forward(xi, w_max, seg_len, tau)
        assert np.all(np.abs(yi - y_x) <= 1e-4 * np.maximum(np.abs(y_x), w)), i
        z = spec[2 * so[i]: 2 * (so[i] + m)].cpu().numpy().reshape(-1, 2).astype(np.float64)
        zi = z[:, 0] + 1j * z[:, 1]
        p_ref, stats, flags = onorm.normalise_power(zi, seg_len)
        assert not flags.any()
        y_o = olse.forward_power(p_ref, w_max, seg_len, tau)
        assert np.all(np.abs(yi - y_o) <= 1e-5 * np.maximum(np.abs(y_o), w)), i
        gx_ref = olse.backward(xi, dict(spec=zi, p=p_ref, stats=stats), y_o, gyi, w_max, seg_len, tau)
        rel = np.linalg.norm(gxi - gx_ref) / np.linalg.norm(gx_ref)
        assert rel <= 1e-4, (i, rel)
        ga_ref = olse.amplitude_grad(gx_ref, ti)
        assert abs(ga_gpu[i] - ga_ref) <= 1e-4 * np.linalg.norm(gx_ref) * np.linalg.norm(ti), (i, ga_gpu[i], ga_ref)
