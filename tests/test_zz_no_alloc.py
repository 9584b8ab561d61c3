"""The allocation-free segment-maxima entry point, through the C ABI.

For callers that cannot call cudaMalloc (their device memory comes from a
pool they own, or an allocation would stall a real-time stream), the library
offers pulscan_segment_maxima_noalloc: its only scratch is a static device
array inside the library.  This test checks its maxima against the FP64
oracle (on the GPU's own power spectrum, under the stage-B rule of
tests/parity.py) and against the plan-based pulscan_segment_maxima, on two
calls in a row (the shared scratch must be left clean by each call),
including shapes that fill the array exactly.  The refusal of shapes beyond
its capacity needs no GPU and is tested in tests/test_capi.py.  This file
is collected last, so that a failure here never hides another test.
"""
import numpy as np
import pytest

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


def _series(n, seed):
    from paper_2406_15186_gb300 import synth
    return synth.inject(synth.noise(n, seed), [dict(amp=0.2, r0=0.3 * n / 2, z=25.0, w=0.0, phi0=0.1)])


def _noalloc(pkg, d_power, n, w_max, seg_len, n_seg):
    lib = pkg.load()
    mx = torch.full((n_seg * w_max,), -7.0, dtype=torch.float32, device="cuda")
    am = torch.full((n_seg * w_max,), -7, dtype=torch.int64, device="cuda")
    rc = lib.pulscan_segment_maxima_noalloc(d_power.data_ptr(), n, w_max, seg_len, mx.data_ptr(), am.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    assert rc == 0, lib.pulscan_last_error().decode()
    torch.cuda.synchronize()
    return mx.cpu().numpy().reshape(n_seg, w_max), am.cpu().numpy().reshape(n_seg, w_max)


# (n, z_max, segment_len, oracle rows): the last two fill the static array
# exactly (segments x z_max = 2^20 slots); the z_max = 4096 case runs the
# widest tiles (4 warps per CTA) with the largest halo the array accepts
CASES = [(1 << 16, 100, 1024, None), (1 << 17, 64, 777, None), (1 << 21, 256, 256, None),
         (1 << 23, 4096, 16384, [(0, 1), (77, 78), (255, 256)])]


@pytest.mark.parametrize("n,w_max,seg_len,rows", CASES)
def test_noalloc_matches_the_oracle_and_the_plan_twice(pkg, n, w_max, seg_len, rows):
    m = n // 2 + 1
    n_seg = max(1, m // seg_len)
    for call, seed in enumerate((1, 2)):
        plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=6.0)
        d_x, d_spec, d_power = plan.buffers()
        d_x.copy_(torch.from_numpy(_series(n, seed)))
        plan.rfft(d_x, d_spec)
        plan.power_normalise(d_spec, d_power)
        ref_mx = torch.empty(plan.total_segments * w_max, dtype=torch.float32, device="cuda")
        ref_am = torch.empty(plan.total_segments * w_max, dtype=torch.int64, device="cuda")
        plan.segment_maxima(d_power, ref_mx, ref_am)
        torch.cuda.synchronize()
        g_mx, g_am = _noalloc(pkg, d_power, n, w_max, seg_len, n_seg)
        # the oracle on the GPU's power (stage B: maxima within 1e-5 max(S, w),
        # argmax equal or a near tie)
        p64 = d_power.cpu().numpy()[:m].astype(np.float64)
        for r in (rows or [None]):
            parity.check_maxima(p64, g_mx, g_am, w_max, seg_len, seg_range=r)
        # and the plan-based entry point: the same kernel, bit for bit
        r_mx = ref_mx.cpu().numpy().reshape(n_seg, w_max)
        r_am = ref_am.cpu().numpy().reshape(n_seg, w_max)
        assert np.array_equal(np.isnan(g_mx), np.isnan(r_mx)), f"call {call}"
        ok = ~np.isnan(r_mx)
        assert np.array_equal(g_mx[ok], r_mx[ok]), f"call {call}"
        assert np.array_equal(g_am, r_am), f"call {call}"
        plan.close()
