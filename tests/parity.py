"""Shared helpers of the GPU parity tests: run the CUDA path, compare with the oracle.

Tolerances (written here once, used by every parity test):
* normalised power: |P_gpu - P_ref| <= 1e-5 * max(P_ref, 1)
* boxcar maxima:    |S_gpu - S_ref| <= 1e-5 * max(S_ref, w)   (w = noise mean of S_w)
* argmax:           equal, or a near tie: S_ref[k_gpu] >= S_ref[k*] - 1e-5 * max(S_ref, w)
* candidate sets:   equal except (segment, width) pairs whose oracle maximum is
                    within 1e-4 of the threshold (the emission decision flips
                    between S (1 - 1e-4) and S (1 + 1e-4))
* sigma:            |sigma_gpu - sigma_ref(S_gpu)| <= 1e-5 * max(1, sigma)
"""
import numpy as np

from oracle import boxcar as obox
from oracle import normalise as onorm
from oracle import pipeline as opipe
from oracle import significance as osig

P_TOL = 1e-5
S_TOL = 1e-5
BAND = 1e-4
SIG_TOL = 1e-5


def run_gpu(plan, x, device="cuda", stats=False, maxima=True, use_graph=False):
    """Run rfft -> normalise -> search (-> segment maxima) on the GPU."""
    import torch
    d_x, d_spec, d_power = plan.buffers(device)
    d_x.copy_(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)))
    d_stats = torch.zeros(4 * plan.total_segments, dtype=torch.float32, device=device) if stats else None
    if use_graph:
        plan.search(d_x, d_spec, d_power, use_graph=True)
        if stats:
            plan.power_normalise(d_spec, d_power, d_stats)
    else:
        plan.rfft(d_x, d_spec)
        plan.power_normalise(d_spec, d_power, d_stats)
        plan.boxcar_search(d_power)
    cands = plan.candidates()
    out = dict(spec=d_spec.cpu().numpy(), power=d_power.cpu().numpy(), cands=cands)
    if stats:
        out["stats"] = d_stats.cpu().numpy().reshape(-1, 4)
    if maxima:
        n = plan.total_segments * plan.z_max
        mx = torch.empty(n, dtype=torch.float32, device=device)
        am = torch.empty(n, dtype=torch.int64, device=device)
        plan.segment_maxima(d_power, mx, am)
        out["mx"] = mx.cpu().numpy().reshape(plan.total_segments, plan.z_max)
        out["am"] = am.cpu().numpy().reshape(plan.total_segments, plan.z_max)
    torch.cuda.synchronize()
    return out


def spectrum_complex(spec_floats, off=0, m=None):
    z = spec_floats.reshape(-1, 2)
    z = z[:, 0].astype(np.float64) + 1j * z[:, 1].astype(np.float64)
    return z[off: off + m] if m is not None else z


def check_normalise(spec_c, p_gpu, stats_gpu, seg_len):
    """Stage A: oracle normalisation of the GPU spectrum vs the GPU power."""
    p_ref, st_ref, flags = onorm.normalise_power(spec_c, seg_len)
    assert not flags.any()
    # medians and MADs: the same order statistics, up to FP32 rounding
    assert np.allclose(stats_gpu[:, [0, 2]], st_ref[:, [0, 2]], rtol=2 ** -22, atol=1e-30 + 2 ** -22 * st_ref[:, [1, 3]])
    assert np.allclose(stats_gpu[:, [1, 3]], st_ref[:, [1, 3]], rtol=1e-6)
    err = np.abs(p_gpu.astype(np.float64) - p_ref) / np.maximum(p_ref, 1.0)
    assert err.max() <= P_TOL, err.max()
    return p_ref


def check_maxima(p64, mx_gpu, am_gpu, w_max, seg_len, seg_range=None):
    """Stage B: oracle maxima on the GPU power vs the GPU dump-mode maxima."""
    mx_ref, am_ref = obox.segment_maxima(p64, w_max, seg_len, seg_range=seg_range)
    rows = slice(None) if seg_range is None else slice(*seg_range)
    mr, ar = mx_ref[rows], am_ref[rows]
    mg, ag = mx_gpu[rows].astype(np.float64), am_gpu[rows]
    empty = np.isnan(mr)
    assert np.array_equal(empty, np.isnan(mg)), "valid (segment, width) pairs differ"
    assert np.all(ag[empty] == -1)
    w = np.broadcast_to(np.arange(1, w_max + 1)[None, :], mr.shape)
    scale = np.maximum(mr, w)
    ok = ~empty
    err = np.abs(mg[ok] - mr[ok]) / scale[ok]
    assert err.max(initial=0.0) <= S_TOL, err.max()
    # argmax: exact, or a near tie checked on the oracle's own sums
    diff = ok & (ag != ar)
    for s, wi in zip(*np.nonzero(diff)):
        k = int(ag[s, wi])
        width = wi + 1
        v = float(np.sum(p64[k:k + width]))
        assert v >= mr[s, wi] - S_TOL * scale[s, wi], (s, width, k, ar[s, wi])
    return mx_ref, am_ref


def oracle_decisions(mx_ref, n_trials, sigma_thr, widths=None, shape_mult=1):
    """(passes, ambiguous) per (segment, width) from the oracle maxima; only
    searched widths (all when widths is None) can pass.  shape_mult: gamma
    shape per unit width (H(H+1)/2 for an H-harmonic sum)."""
    n_seg, w_max = mx_ref.shape
    dec = np.zeros(mx_ref.shape, dtype=bool)
    amb = np.zeros(mx_ref.shape, dtype=bool)
    for wi in (range(w_max) if widths is None else [w - 1 for w in widths]):
        col = mx_ref[:, wi]
        ok = ~np.isnan(col)
        if not ok.any():
            continue
        s = col[ok]
        a = shape_mult * (wi + 1)
        d = osig.passes(a, s, n_trials, sigma_thr)
        lo = osig.passes(a, s * (1 - BAND), n_trials, sigma_thr)
        hi = osig.passes(a, s * (1 + BAND), n_trials, sigma_thr)
        dec[ok, wi] = d
        amb[ok, wi] = lo != hi
    return dec, amb


def check_candidates(cands, p64, mx_ref, am_ref, w_max, seg_len, sigma_thr, n_trials, series=0, seg_rows=None,
                     widths=None, shape_mult=1):
    """Candidate set of one series vs the oracle decisions on its maxima."""
    m = len(p64)
    n_seg = mx_ref.shape[0]
    dec, amb = oracle_decisions(mx_ref, n_trials, sigma_thr, widths, shape_mult)
    if seg_rows is not None:
        keep = np.zeros(n_seg, dtype=bool)
        keep[seg_rows[0]:seg_rows[1]] = True
        dec &= keep[:, None]
        amb &= keep[:, None]
    mine = cands[cands["series"] == series]
    got = {}
    for r in mine:
        s = min(int(r["bin"]) // seg_len, n_seg - 1)
        if seg_rows is not None and not (seg_rows[0] <= s < seg_rows[1]):
            continue
        key = (s, int(r["width"]))
        assert key not in got, f"duplicate candidate {key}"
        got[key] = r
    exp = set(zip(*np.nonzero(dec)))
    exp = {(int(a), int(b) + 1) for a, b in exp}
    gk = set(got)
    for s, w in (gk - exp) | (exp - gk):
        assert amb[s, w - 1], f"candidate mismatch at segment {s} width {w}"
    for (s, w) in gk & exp:
        r = got[(s, w)]
        sref = mx_ref[s, w - 1]
        scale = max(sref, w)
        assert abs(float(r["power"]) - sref) <= S_TOL * scale
        if int(r["bin"]) != am_ref[s, w - 1]:
            k = int(r["bin"])
            assert float(np.sum(p64[k:k + w])) >= sref - S_TOL * scale
        sg_ref = osig.sigma_of(shape_mult * w, float(r["power"]), n_trials)[0]
        assert abs(float(r["sigma"]) - sg_ref) <= SIG_TOL * max(1.0, abs(sg_ref)), (s, w, r["sigma"], sg_ref)
        assert float(r["sigma"]) >= sigma_thr - 1e-3
    del m
    return len(gk)


def n_trials_of(m, w_max):
    return opipe.n_trials_default(m, w_max)
