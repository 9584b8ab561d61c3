"""GPU parity of the differentiable extension (logsumexp statistic and adjoint).

Forward: Y from the GPU power against the oracle's logsumexp of the same
power (FP64).  Backward: dL/dx against the oracle's hand-written FP64 adjoint
taken from the GPU spectrum, and a central finite difference of the GPU
forward itself.  Amplitude: dL/dA through pulscan_inject /
pulscan_amplitude_grad and torch.autograd against the oracle's dL/dA.

Tolerances.  Y: 1e-5 * max(|Y_ref|, w), as for the boxcar maxima (Y is a
smoothed maximum of the same sums).  Gradients: rel-L2 <= 1e-4, the
contract for the GPU against the FP64 oracle.  The softmax weights
exp((S - Y) / tau) turn an error dS - dY into a relative weight error
(dS - dY) / tau, so the kernels keep every weighted window's S and Y itself
as float pairs (S - Y formed without rounding either); what is left is the
FP32 power (a few ulp per bin: 1e-6 of S at most, and neighbouring windows
share all but their end bins), the FP32 difference array, normalisation
adjoint and C2R (~1e-6).  dL/dA = <dL/dx, template>: its error is at most
||dL/dx error|| ||template|| (Cauchy-Schwarz), 1e-4 of ||dL/dx|| ||template||.
"""
import numpy as np
import pytest

from oracle import lse as olse
from oracle import normalise as onorm
from paper_2406_15186_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GRAD_TOL = {0.1: 1e-4, 1.0: 1e-4}


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2406_15186_gb300 as p
    from paper_2406_15186_gb300 import build
    build.build()
    p.load()
    return p


def _forward(pkg, plan, x, tau):
    lib = pkg.load()
    d = dict(x=torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda(),
             spec=torch.empty(plan.spec_floats, device="cuda"), power=torch.empty(plan.power_floats, device="cuda"),
             stats=torch.empty(4 * plan.total_segments, device="cuda"),
             sel=torch.empty(8 * plan.total_segments, device="cuda"),
             y=torch.empty(plan.total_segments * plan.z_max, device="cuda"),
             ylo=torch.empty(plan.total_segments * plan.z_max, device="cuda"))
    rc = lib.pulscan_lse_forward(plan._h, d["x"].data_ptr(), d["spec"].data_ptr(), d["power"].data_ptr(),
                                 d["stats"].data_ptr(), d["sel"].data_ptr(), d["y"].data_ptr(), d["ylo"].data_ptr(),
                                 tau, None)
    assert rc == 0, lib.pulscan_last_error().decode()
    torch.cuda.synchronize()
    return d


def _backward(pkg, plan, d, gy, tau):
    lib = pkg.load()
    g = torch.from_numpy(np.ascontiguousarray(gy, dtype=np.float32)).cuda()
    gx = torch.empty(plan.x_floats, device="cuda")
    rc = lib.pulscan_lse_backward(plan._h, d["spec"].data_ptr(), d["power"].data_ptr(), d["stats"].data_ptr(),
                                  d["sel"].data_ptr(), d["y"].data_ptr(), d["ylo"].data_ptr(), g.data_ptr(),
                                  gx.data_ptr(), tau, None)
    assert rc == 0, lib.pulscan_last_error().decode()
    torch.cuda.synchronize()
    return gx.cpu().numpy().astype(np.float64)


def _series(n, seed):
    x = synth.noise(n, seed)
    return synth.inject(x, [dict(amp=0.15, r0=0.21 * n / 2, z=20.0, w=5.0, phi0=0.7)])


def _spec(d, m):
    z = d["spec"].cpu().numpy().reshape(-1, 2)[:m]
    return z[:, 0].astype(np.float64) + 1j * z[:, 1].astype(np.float64)


@pytest.mark.parametrize("tau", [0.1, 1.0])
# segments of one warp's 1056 bins or less, and (the last two) CTAs of four
# warps: segments of 2500 bins with a last block of 3193, one block of 4097
@pytest.mark.parametrize("n,w_max,seg_len", [(1 << 14, 48, 512), (1 << 13, 33, 300), (1 << 12, 7, 64),
                                             (1 << 14, 40, 2500), (1 << 13, 100, 4000)])
def test_forward_and_backward_against_oracle(pkg, n, w_max, seg_len, tau):
    x = _series(n, 17)
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=6.0)
    m = n // 2 + 1
    d = _forward(pkg, plan, x, tau)
    p_gpu = d["power"].cpu().numpy()[:m].astype(np.float64)
    y_gpu = d["y"].cpu().numpy().reshape(plan.total_segments, w_max).astype(np.float64)
    y_ref = olse.forward_power(p_gpu, w_max, seg_len, tau)
    w = np.arange(1, w_max + 1)[None, :]
    assert np.all(np.abs(y_gpu - y_ref) <= 1e-5 * np.maximum(np.abs(y_ref), w))
    # backward from the GPU spectrum
    gy = np.random.default_rng(3).standard_normal(y_ref.shape)
    gx = _backward(pkg, plan, d, gy, tau)
    spec = _spec(d, m)
    p_ref, stats, flags = onorm.normalise_power(spec, seg_len)
    assert not flags.any()
    y_o = olse.forward_power(p_ref, w_max, seg_len, tau)
    gx_ref = olse.backward(x.astype(np.float64), dict(spec=spec, p=p_ref, stats=stats), y_o, gy, w_max, seg_len, tau)
    rel = np.linalg.norm(gx - gx_ref) / np.linalg.norm(gx_ref)
    assert rel <= GRAD_TOL[tau], rel


@pytest.mark.parametrize("tau", [0.1, 1.0])
def test_finite_difference_away_from_order_statistic_kinks(pkg, tau):
    """<dL/dx, v> by the adjoint vs a central difference of the GPU forward.

    The median and MAD are only almost-everywhere differentiable: a step that
    carries a bin across the selected order statistic measures a different
    slope.  So v moves only Fourier bins whose real and imaginary parts lie at
    least 0.3 MAD from the block median and from the MAD order statistic, by
    at most 0.05 MAD each: no order statistic changes along the step, and the
    difference is well posed."""
    n, w_max, seg_len = 1 << 13, 24, 256
    x = _series(n, 29).astype(np.float64)
    m = n // 2 + 1
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=6.0)
    d = _forward(pkg, plan, x, tau)
    spec = np.fft.rfft(x)
    rng = np.random.default_rng(21)
    dz = np.zeros(m, dtype=complex)
    for lo, hi in onorm.block_bounds(m, seg_len):
        blk = spec[lo:hi].copy()
        if lo == 0:
            blk[0] = 0.0
        ok = np.ones(hi - lo, dtype=bool)
        scl = []
        for comp in (blk.real, blk.imag):
            med = onorm.median(comp)
            mad = onorm.mad(comp, med)
            dev = np.abs(comp - med)
            ok &= (dev > 0.3 * mad) & (np.abs(dev - mad) > 0.3 * mad)
            scl.append(mad)
        ok[0] &= lo != 0
        idx = np.nonzero(ok)[0]
        dz[lo + idx] = 0.05 * (scl[0] * rng.uniform(-1, 1, idx.size) + 1j * scl[1] * rng.uniform(-1, 1, idx.size))
    dz[-1] = dz[-1].real                                  # the Nyquist bin of a real series is real
    v = np.fft.irfft(dz, n)                               # rfft(v) = dz
    gy = rng.standard_normal(plan.total_segments * w_max)
    gx = _backward(pkg, plan, d, gy, tau)
    loss = lambda xx: float(np.dot(gy, _forward(pkg, plan, xx, tau)["y"].cpu().numpy().astype(np.float64)))
    fd = (loss(x + v) - loss(x - v)) / 2.0
    assert float(np.dot(gx, v)) == pytest.approx(fd, rel=2e-2)


@pytest.mark.parametrize("tau", [0.1, 1.0])
def test_gradient_is_orthogonal_to_rescaling(pkg, tau):
    """Eq. 8 divides by the MAD, so Y(c x) = Y(x): <dL/dx, x> = 0 exactly.

    Without the median/MAD terms of the adjoint this fails by O(1)."""
    n, w_max, seg_len = 1 << 13, 24, 256
    x = _series(n, 31).astype(np.float64)
    plan = pkg.Plan(n=n, z_max=w_max, segment_len=seg_len, threshold_sigma=6.0)
    d = _forward(pkg, plan, x, tau)
    gy = np.random.default_rng(12).standard_normal(plan.total_segments * w_max)
    gx = _backward(pkg, plan, d, gy, tau)
    assert abs(float(np.dot(gx, x))) <= 1e-3 * np.linalg.norm(gx) * np.linalg.norm(x)


def test_amplitude_gradient_through_autograd(pkg):
    """dL/dA through torch.autograd (pulscan_inject, the logsumexp forward and
    backward, pulscan_amplitude_grad) against the oracle's dL/dA: its
    adjoint taken from the GPU spectrum of the same x, projected on the
    template (oracle.lse.amplitude_grad)."""
    from paper_2406_15186_gb300 import lse
    lengths = [1 << 12] * 5
    w_max, seg_len, tau = 16, 128, 0.1
    plan = pkg.Plan(lengths=lengths, z_max=w_max, segment_len=seg_len, threshold_sigma=6.0)
    xo, so, _, go = plan.offsets()
    noise = np.zeros(plan.x_floats, np.float32)
    tmpl = np.zeros(plan.x_floats, np.float32)
    amps = np.array([0.02, 0.05, 0.1, 0.2, 0.0], np.float32)
    for i, nn in enumerate(lengths):
        noise[xo[i]: xo[i] + nn] = synth.noise(nn, 100 + i)
        tmpl[xo[i]: xo[i] + nn] = synth.chirp(nn, 300.0 + 40 * i, 12.0, -3.0, 0.4).astype(np.float32)
    t_noise, t_tmpl = torch.from_numpy(noise).cuda(), torch.from_numpy(tmpl).cuda()
    amp = torch.from_numpy(amps).cuda().requires_grad_(True)
    x = lse.inject(t_noise, t_tmpl, amp, plan)
    y = lse.lse_statistic(x, plan, tau)
    gy = torch.from_numpy(np.random.default_rng(4).standard_normal(tuple(y.shape)).astype(np.float32)).cuda()
    (y * gy).sum().backward()
    g_gpu = amp.grad.cpu().numpy().astype(np.float64)
    spec_all = torch.empty(plan.spec_floats, device="cuda")
    plan.rfft(x.detach(), spec_all)
    torch.cuda.synchronize()
    xs = x.detach().cpu().numpy()
    zs = spec_all.cpu().numpy()
    gyn = gy.cpu().numpy().astype(np.float64)
    for i, nn in enumerate(lengths):
        m = nn // 2 + 1
        xi = xs[xo[i]: xo[i] + nn].astype(np.float64)
        z = zs[2 * so[i]: 2 * (so[i] + m)].reshape(-1, 2).astype(np.float64)
        zi = z[:, 0] + 1j * z[:, 1]
        p_ref, stats, flags = onorm.normalise_power(zi, seg_len)
        assert not flags.any()
        y_o = olse.forward_power(p_ref, w_max, seg_len, tau)
        rows = slice(go[i], go[i] + y_o.shape[0])
        gxi = olse.backward(xi, dict(spec=zi, p=p_ref, stats=stats), y_o, gyn[rows], w_max, seg_len, tau)
        ti = tmpl[xo[i]: xo[i] + nn].astype(np.float64)
        ref = olse.amplitude_grad(gxi, ti)
        bound = 1e-4 * np.linalg.norm(gxi) * np.linalg.norm(ti)
        assert abs(g_gpu[i] - ref) <= bound, (i, g_gpu[i], ref, bound)
