"""GPU normalisation (Eq. 8) on crafted spectra, through pulscan_power_normalise.

The spectra are written straight into the spectrum buffer, so each case
reaches a chosen branch of the order-statistic select: crowded value buckets
(a few huge outliers stretch a block's range, so the fast select's target
bucket overflows and the multi-level select takes over), heavy ties
(integer-valued components), a median inside a run of equal values, a
constant block (MAD 0: P = 0, flagged by the oracle), odd and even block
sizes, blocks of up to 256 x 32 bins (register kernel) and larger ones
(shared-memory kernel).  The medians and MADs are order statistics of the
same float32 values, so they must agree with the oracle to FP32 rounding of
the mean of the two middle values (MADs: and of the deviations from that
median); P to 1e-5 relative.
"""
import numpy as np
import pytest

from oracle import normalise as onorm

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


def _run(pkg, spec, n, seg_len):
    m = n // 2 + 1
    assert spec.shape == (m,)
    plan = pkg.Plan(n=n, z_max=8, segment_len=seg_len, threshold_sigma=6.0)
    z = np.zeros(plan.spec_floats, np.float32)
    z[0: 2 * m: 2] = spec.real.astype(np.float32)
    z[1: 2 * m: 2] = spec.imag.astype(np.float32)
    d_spec = torch.from_numpy(z).cuda()
    d_power = torch.zeros(plan.power_floats, device="cuda")
    d_stats = torch.zeros(4 * plan.total_segments, device="cuda")
    plan.power_normalise(d_spec, d_power, d_stats)
    torch.cuda.synchronize()
    p_gpu = d_power.cpu().numpy()[:m].astype(np.float64)
    st_gpu = d_stats.cpu().numpy().reshape(-1, 4).astype(np.float64)
    # the oracle sees exactly the float32 values the kernel read
    spec32 = z[0: 2 * m: 2].astype(np.float64) + 1j * z[1: 2 * m: 2].astype(np.float64)
    p_ref, st_ref, flags = onorm.normalise_power(spec32, seg_len)
    return p_gpu, st_gpu, p_ref, st_ref, flags


def _check(p_gpu, st_gpu, p_ref, st_ref, flags, seg_len):
    # medians: the mean of two float32 values rounded to float32; MADs: order
    # statistics of float32 deviations from that rounded median
    med, mad = st_ref[:, [0, 2]], st_ref[:, [1, 3]]
    assert np.all(np.abs(st_gpu[:, [0, 2]] - med) <= 2 ** -23 * (np.abs(med) + mad))
    assert np.all(np.abs(st_gpu[:, [1, 3]] - mad) <= 1e-6 * mad + 2 ** -23 * np.abs(med))
    bounds = onorm.block_bounds(p_ref.shape[0], seg_len)
    for s, (lo, hi) in enumerate(bounds):
        if flags[s]:
            assert np.all(p_gpu[lo:hi] == 0.0)
    err = np.abs(p_gpu - p_ref) / np.maximum(p_ref, 1.0)
    assert err.max() <= 1e-5, err.max()


def _gauss(m, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(m) + 1j * rng.standard_normal(m)


@pytest.mark.parametrize("n,seg_len", [(1 << 14, 2048), (1 << 13, 1000), (1 << 15, 4096), (1 << 16, 8192),
                                       (1 << 17, 16384), (1 << 16, 16384), (1 << 12, 37)])
def test_gaussian_blocks(pkg, n, seg_len):
    spec = _gauss(n // 2 + 1, n + seg_len)
    _check(*_run(pkg, spec, n, seg_len), seg_len)


@pytest.mark.parametrize("n,seg_len", [(1 << 14, 2048), (1 << 15, 8192), (1 << 16, 16384)])
def test_crowded_buckets_fall_back_to_levels(pkg, n, seg_len):
    """A few outliers 1e5 times the noise: ~all values land in one bucket."""
    m = n // 2 + 1
    spec = _gauss(m, 5)
    rng = np.random.default_rng(6)
    for lo, hi in onorm.block_bounds(m, seg_len):
        idx = rng.choice(np.arange(lo, hi), size=3, replace=False)
        spec[idx] = 1e5 * (rng.standard_normal(3) + 1j * rng.standard_normal(3))
    _check(*_run(pkg, spec, n, seg_len), seg_len)


@pytest.mark.parametrize("n,seg_len", [(1 << 14, 2048), (1 << 17, 16384)])
def test_integer_ties(pkg, n, seg_len):
    m = n // 2 + 1
    rng = np.random.default_rng(8)
    spec = rng.integers(-3, 4, m).astype(np.float64) + 1j * rng.integers(-2, 3, m).astype(np.float64)
    _check(*_run(pkg, spec, n, seg_len), seg_len)


@pytest.mark.parametrize("n,seg_len", [(1 << 13, 1024), (1 << 15, 8192)])
def test_median_inside_a_run_of_equal_values(pkg, n, seg_len):
    m = n // 2 + 1
    spec = _gauss(m, 9)
    rng = np.random.default_rng(10)
    for lo, hi in onorm.block_bounds(m, seg_len):
        idx = rng.choice(np.arange(lo, hi), size=(hi - lo) // 2, replace=False)
        spec[idx] = 0.5 + 0.25j
    _check(*_run(pkg, spec, n, seg_len), seg_len)


def test_constant_block_gives_zero_power(pkg):
    n, seg_len = 1 << 13, 1024
    m = n // 2 + 1
    spec = _gauss(m, 11)
    spec[1024:2048] = 1.0 + 1.0j       # block 1: MAD 0
    p_gpu, st_gpu, p_ref, st_ref, flags = _run(pkg, spec, n, seg_len)
    assert flags[1] and not flags[0]
    _check(p_gpu, st_gpu, p_ref, st_ref, flags, seg_len)


@pytest.mark.parametrize("n,seg_len", [(1 << 13, 2048), (1 << 15, 8192)])
def test_middle_pair_split_over_two_crowded_buckets(pkg, n, seg_len):
    """Each block holds half its values in a narrow cluster at -1 and half at
    +1 (each within 1e-4), per component: the two middle order statistics sit
    in two crowded buckets with only empty buckets between them (decided from
    the two buckets' extremes), and every deviation from the median lies in
    one crowded bucket (the multi-level select)."""
    m = n // 2 + 1
    rng = np.random.default_rng(12)
    spec = np.empty(m, dtype=complex)
    for lo, hi in onorm.block_bounds(m, seg_len):
        k = hi - lo
        half = np.r_[-np.ones(k // 2), np.ones(k - k // 2)]
        re = rng.permutation(half) * (1.0 + 1e-4 * rng.random(k))
        im = rng.permutation(half) * (1.0 + 1e-4 * rng.random(k))
        spec[lo:hi] = re + 1j * im
    _check(*_run(pkg, spec, n, seg_len), seg_len)


@pytest.mark.parametrize("n,seg_len", [(1 << 14, 2048), (1 << 15, 4096)])
def test_tight_cluster_far_from_zero(pkg, n, seg_len):
    """Components in narrow clusters far from zero (1e6 + 0.1 noise, -3e5 +
    0.05 noise), every other block: the value-bucket offset magic - lo s is
    then far beyond integer resolution in FP32, so those blocks must take the
    exact multi-level select, while their neighbours keep the fast one."""
    m = n // 2 + 1
    rng = np.random.default_rng(13)
    spec = _gauss(m, 14)
    for i, (lo, hi) in enumerate(onorm.block_bounds(m, seg_len)):
        if i % 2 == 1:
            k = hi - lo
            spec[lo:hi] = (1e6 + 0.1 * rng.standard_normal(k)) + 1j * (-3e5 + 0.05 * rng.standard_normal(k))
    _check(*_run(pkg, spec, n, seg_len), seg_len)
