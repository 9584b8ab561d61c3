"""Paper-GPU fidelity mode (§2.5 median of medians, §2.6 polynomial log p)
against its oracle, through the C ABI.

Median of medians: the same stride-4 reduction of the same float32 values;
each level rounds one mean, so medians agree to 2^-20 (|med| + MAD) and MADs
to 2^-20 relative; P to 1e-5.  Candidates: every (segment, width) maximum is
a candidate of the polynomial rule; decisions are compared on the oracle's
FP64 maxima of the GPU power, and a pair whose decision changes between
S (1 - 1e-4), S and S (1 + 1e-4) may differ (the polynomial is not monotone,
so the band is tested at all three points).
"""
import ctypes

import numpy as np
import pytest

from oracle import boxcar as obox
from oracle import fidelity as ofid
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


def _series(n, seed):
    x = synth.noise(n, seed)
    return synth.inject(x, [dict(amp=0.2, r0=0.31 * n / 2, z=30.0, w=0.0, phi0=0.2),
                            dict(amp=0.05, r0=0.12 * n / 2, z=3.0, w=0.0, phi0=1.0)])


@pytest.mark.parametrize("n,seg_len", [(1 << 16, 1024), (1 << 15, 256), (1 << 18, 4096)])
def test_median_of_medians_normalisation(pkg, n, seg_len):
    plan = pkg.Plan(n=n, z_max=16, segment_len=seg_len, threshold_sigma=6.0)
    plan.set_fidelity(pkg.FIDELITY_PAPER_GPU)
    out = parity.run_gpu(plan, _series(n, 3), stats=True, maxima=False)
    m = n // 2 + 1
    spec = parity.spectrum_complex(out["spec"], 0, m)
    p_ref, st_ref, flags = ofid.normalise_power_mom(spec, seg_len)
    assert not flags.any()
    st = out["stats"].astype(np.float64)
    med, mad = st_ref[:, [0, 2]], st_ref[:, [1, 3]]
    assert np.all(np.abs(st[:, [0, 2]] - med) <= 2 ** -20 * (np.abs(med) + mad))
    assert np.all(np.abs(st[:, [1, 3]] - mad) <= 2 ** -20 * mad)
    p = out["power"][:m].astype(np.float64)
    assert np.max(np.abs(p - p_ref) / np.maximum(p_ref, 1.0)) <= 1e-5


def test_polynomial_candidates(pkg):
    n, w_max, seg_len, sigma = 1 << 16, 24, 1024, 6.0
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=sigma)
    plan.set_fidelity(pkg.FIDELITY_PAPER_GPU)
    out = parity.run_gpu(plan, _series(n, 4))
    m = n // 2 + 1
    p64 = out["power"][:m].astype(np.float64)
    mx_ref, am_ref = parity.check_maxima(p64, out["mx"], out["am"], w_max, seg_len)
    nt = float(m * w_max)
    target = float(osig.log_sf_normal(sigma))
    got = {}
    for r in out["cands"]:
        key = (min(int(r["bin"]) // seg_len, mx_ref.shape[0] - 1), int(r["width"]))
        assert key not in got
        got[key] = r
    n_match = 0
    for s in range(mx_ref.shape[0]):
        for w in range(1, w_max + 1):
            sref = mx_ref[s, w - 1]
            if np.isnan(sref):
                assert (s, w) not in got
                continue
            dec = [float(ofid.log_p_adjusted_poly(w, sref * f, nt)) <= target for f in (1 - 1e-4, 1.0, 1 + 1e-4)]
            if (s, w) in got:
                r = got[(s, w)]
                assert dec[1] or any(dec), (s, w)
                lp = float(ofid.log_p_adjusted_poly(w, float(r["power"]), nt))
                sg = float(osig.sigma_from_log_p(np.array([lp]))[0])
                assert abs(float(r["sigma"]) - sg) <= 1e-5 * max(1.0, abs(sg)), (s, w, r["sigma"], sg)
                assert abs(float(r["power"]) - sref) <= parity.S_TOL * max(sref, w)
                n_match += 1
            else:
                assert not all(dec), (s, w, sref)
    assert n_match > 0


def test_fidelity_mode_validation(pkg):
    plan = pkg.Plan(n=1 << 14, z_max=16, segment_len=512, threshold_sigma=6.0)
    with pytest.raises(pkg.PulscanError):
        plan.set_fidelity(pkg.FIDELITY_PAPER_GPU)        # 512 is not a power of four
    plan = pkg.Plan(n=1 << 14, z_max=16, segment_len=1024, threshold_sigma=6.0)
    plan.set_fidelity(pkg.FIDELITY_PAPER_GPU)
    lib = pkg.load()
    z = [torch.zeros(k, device="cuda") for k in (plan.x_floats, plan.spec_floats, plan.power_floats,
                                                  4 * plan.total_segments, 8 * plan.total_segments,
                                                  plan.total_segments * plan.z_max, plan.total_segments * plan.z_max)]
    rc = lib.pulscan_lse_forward(plan._h, *[t.data_ptr() for t in z], ctypes.c_float(0.1), None)
    assert rc == -6
    plan.set_fidelity(pkg.FIDELITY_EXACT)
