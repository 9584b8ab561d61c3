"""The allocation-free segment-maxima entry point, through the C ABI.

For callers that cannot call cudaMalloc (their device memory comes from a
pool they own, or an allocation would stall a real-time stream), the library
offers pulscan_segment_maxima_noalloc: its only scratch is a static device
array inside the library.  This test compares it with the plan-based
pulscan_segment_maxima on the same power spectra, twice in a row (the shared
scratch must be left clean by each call), and checks that shapes beyond its
fixed capacity are refused on the host.  It lives in its own file, collected
last, so that a failure here never hides another test.
"""
import numpy as np
import pytest

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


def _power(n, seed):
    from paper_2406_15186_gb300 import synth
    x = synth.inject(synth.noise(n, seed), [dict(amp=0.2, r0=0.3 * n / 2, z=25.0, w=0.0, phi0=0.1)])
    return x


def _noalloc(pkg, d_power, n, w_max, seg_len, n_seg):
    lib = pkg.load()
    mx = torch.full((n_seg * w_max,), -7.0, dtype=torch.float32, device="cuda")
    am = torch.full((n_seg * w_max,), -7, dtype=torch.int64, device="cuda")
    rc = lib.pulscan_segment_maxima_noalloc(d_power.data_ptr(), n, w_max, seg_len, mx.data_ptr(), am.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    assert rc == 0, lib.pulscan_last_error().decode()
    torch.cuda.synchronize()
    return mx.cpu().numpy(), am.cpu().numpy()


@pytest.mark.parametrize("n,w_max,seg_len", [(1 << 16, 100, 1024), (1 << 17, 64, 777)])
def test_noalloc_matches_plan_maxima_twice(pkg, n, w_max, seg_len):
    for call, seed in enumerate((1, 2)):
        x = _power(n, seed)
        plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=6.0)
        d_x, d_spec, d_power = plan.buffers()
        d_x.copy_(torch.from_numpy(x))
        plan.rfft(d_x, d_spec)
        plan.power_normalise(d_spec, d_power)
        ref_mx = torch.empty(plan.total_segments * w_max, dtype=torch.float32, device="cuda")
        ref_am = torch.empty(plan.total_segments * w_max, dtype=torch.int64, device="cuda")
        plan.segment_maxima(d_power, ref_mx, ref_am)
        torch.cuda.synchronize()
        r_mx, r_am = ref_mx.cpu().numpy(), ref_am.cpu().numpy()
        g_mx, g_am = _noalloc(pkg, d_power, n, w_max, seg_len, plan.total_segments)
        assert np.array_equal(np.isnan(g_mx), np.isnan(r_mx)), f"call {call}"
        ok = ~np.isnan(r_mx)
        w = np.tile(np.arange(1, w_max + 1), plan.total_segments)
        assert np.all(np.abs(g_mx[ok] - r_mx[ok]) <= 1e-5 * np.maximum(r_mx[ok], w[ok])), f"call {call}"
        assert np.array_equal(g_am, r_am), f"call {call}"


def test_noalloc_refuses_shapes_beyond_its_capacity(pkg):
    lib = pkg.load()
    d = torch.zeros(8, dtype=torch.float32, device="cuda")
    # 2^21 bins in segments of 64 at z_max 64: 2^21 slots > 2^20
    rc = lib.pulscan_segment_maxima_noalloc(d.data_ptr(), 1 << 22, 64, 64, d.data_ptr(), d.data_ptr(), None)
    assert rc == -6
    rc = lib.pulscan_segment_maxima_noalloc(d.data_ptr(), 1 << 22, 5000, 8192, d.data_ptr(), d.data_ptr(), None)
    assert rc == -6
    rc = lib.pulscan_segment_maxima_noalloc(d.data_ptr(), 1023, 4, 16, d.data_ptr(), d.data_ptr(), None)
    assert rc == -1
