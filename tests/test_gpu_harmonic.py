"""GPU harmonic summing (§2.3) against the oracle, through the C ABI.

Per stage H = 1..4: the stage spectrum X_H in the power buffer against the
oracle's decimation sum of the GPU's own normalised power (FP32 sums of at
most 10 terms: 1e-6 relative), its per-(segment, width) maxima (the same
1e-5 rules as the power), and its candidates (shape H(H+1)/2 w, Bonferroni
count floor(M/H) x W) with the same near-threshold band as everywhere.
"""
import numpy as np
import pytest

from oracle import harmonic as oharm
from oracle import pipeline as opipe
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


def _pulsar(n, seed, f0=1500.0, amp=0.04):
    """Noise plus a narrow pulse train: harmonics at f0, 2 f0, 3 f0, 4 f0 (drifting a little)."""
    x = synth.noise(n, seed)
    return synth.inject(x, [dict(amp=amp / h, r0=h * f0, z=2.0 * h, w=0.0, phi0=0.3 * h) for h in range(1, 5)])


def _check_stage(out, plan, h, w_max, seg_len, sigma, series=0):
    po, so, nb = plan.stage_offsets(h)
    bpo = plan.offsets()[2]
    m = plan.stage_offsets(1)[2][series]
    p_base = out["power"][bpo[series]: bpo[series] + m].astype(np.float64)
    x_gpu = out["power"][po[series]: po[series] + nb[series]].astype(np.float64)
    x_ref = oharm.harmonic_sum(p_base, h)
    assert x_gpu.shape == x_ref.shape
    assert np.all(np.abs(x_gpu - x_ref) <= 1e-6 * np.maximum(x_ref, 1.0))
    n_seg = max(1, int(nb[series]) // seg_len)   # stage entries follow the layout order, not the caller's
    rows = slice(so[series], so[series] + n_seg)
    mx_ref, am_ref = parity.check_maxima(x_gpu, out["mx"][rows], out["am"][rows], w_max, seg_len)
    c = out["cands"][(out["cands"]["harmonics"] == h)]
    return parity.check_candidates(c, x_gpu, mx_ref, am_ref, w_max, seg_len, sigma,
                                   opipe.n_trials_default(x_gpu.shape[0], w_max), series=series,
                                   shape_mult=oharm.shape_per_width(h))


@pytest.mark.parametrize("numharm", [2, 4])
def test_single_series_stages(pkg, numharm):
    n, w_max, seg_len, sigma = 1 << 16, 32, 512, 2.0
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma, numharm=numharm)
    out = parity.run_gpu(plan, _pulsar(n, 21))
    assert set(np.unique(out["cands"]["harmonics"])) <= set(range(1, numharm + 1))
    counts = [_check_stage(out, plan, h, w_max, seg_len, sigma) for h in range(1, numharm + 1)]
    assert min(counts) > 0


def test_batch_of_uneven_series_with_harmonics(pkg):
    lengths = [1 << 14, 1 << 15, 1 << 14, 3 * (1 << 13)]
    w_max, seg_len, sigma = 24, 256, 2.5
    plan = pkg.Plan(lengths=lengths, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma, numharm=3)
    xo = plan.offsets()[0]
    x = np.zeros(plan.x_floats, np.float32)
    for i, n in enumerate(lengths):
        x[xo[i]: xo[i] + n] = _pulsar(n, 40 + i, f0=700.0 + 50 * i)
    out = parity.run_gpu(plan, x)
    for i in range(len(lengths)):
        for h in (1, 2, 3):
            _check_stage(out, plan, h, w_max, seg_len, sigma, series=i)


def test_harmonic_plan_validation(pkg):
    lib = pkg.load()
    import ctypes
    h = ctypes.c_void_p()
    arr = (ctypes.c_int64 * 1)(1 << 12)
    # segment_len above floor(M / numharm)
    assert lib.pulscan_plan_create_harmonic(ctypes.byref(h), arr, 1, 8, 600, 6.0, 4) == -1
    assert lib.pulscan_plan_create_harmonic(ctypes.byref(h), arr, 1, 8, 256, 6.0, 9) == -1
    assert lib.pulscan_plan_create_harmonic(ctypes.byref(h), arr, 1, 8, 256, 6.0, 4) == 0
    lib.pulscan_plan_destroy(h)
