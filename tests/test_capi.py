"""The C ABI library builds, loads and exports every symbol of include/pulscan.h.

Runs without a GPU: only argument validation that happens before any CUDA
call is exercised here.
"""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_2406_15186_gb300 import build
    build.build()
    import paper_2406_15186_gb300 as pkg
    return pkg.load()


def _declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^PULSCAN_API\b[^(]*?\b(pulscan_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("pulscan_plan_create", "pulscan_power_normalise", "pulscan_boxcar_search",
                     "pulscan_candidates", "pulscan_segment_maxima", "pulscan_rfft"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_invalid_arguments_rejected_before_cuda(lib):
    import paper_2406_15186_gb300 as pkg
    h = ctypes.c_void_p()
    cases = [
        (7, 4, 4, 6.0),          # odd n
        (0, 4, 4, 6.0),          # too short
        (1024, 0, 16, 6.0),      # z_max < 1
        (1024, 32, 16, 6.0),     # segment_len < z_max
        (1024, 4, 600, 6.0),     # segment_len > n/2 + 1
        (1024, 4, 16, float("nan")),
        (1024, 4, 16, -1.0),
    ]
    for n, w, l, s in cases:
        rc = lib.pulscan_plan_create(ctypes.byref(h), n, w, l, s)
        assert rc == -1, (n, w, l, s)
        assert lib.pulscan_last_error()
    lengths = (ctypes.c_int64 * 2)(1024, 1023)
    assert lib.pulscan_plan_create_batch(ctypes.byref(h), lengths, 2, 4, 16, 6.0) == -1
    assert lib.pulscan_plan_create_batch(ctypes.byref(h), lengths, 0, 4, 16, 6.0) == -1
    with pytest.raises(pkg.PulscanError):
        pkg.Plan(n=1024, z_max=64, segment_len=32)
    # null plan handles
    assert lib.pulscan_boxcar_search(None, None, None) == -1
    n_out = ctypes.c_int64(0)
    assert lib.pulscan_candidates(None, None, 0, ctypes.byref(n_out), None) == -1
    assert lib.pulscan_search_host_async(None, None, 1, None) == -1
    assert lib.pulscan_search_host(None, None, None, 0, ctypes.byref(n_out), 1, None) == -1
    assert lib.pulscan_plan_set_pipeline(None, 1 << 26) == -1
    assert lib.pulscan_plan_pipeline_parts(None, ctypes.byref(n_out)) == -1
    assert lib.pulscan_plan_set_fused(None, 1) == -1
    assert lib.pulscan_plan_set_defer_form(None, 1) == -1
    f32 = ctypes.c_int32(0)
    assert lib.pulscan_plan_defer_form(None, ctypes.byref(f32)) == -1
    t = ctypes.c_float(0.0)
    assert lib.pulscan_threshold_power(0.0, 1.0e6, 6.0, ctypes.byref(t)) == -1
    assert lib.pulscan_version() >= 10000


def test_candidate_record_layout():
    import paper_2406_15186_gb300 as pkg
    assert pkg.CAND_DTYPE.itemsize == 32
    assert [pkg.CAND_DTYPE.fields[k][1] for k in ("series", "width", "bin", "power", "sigma")] == [0, 4, 8, 16, 20]


def test_noalloc_refuses_before_any_cuda_call(lib):
    """pulscan_segment_maxima_noalloc checks every size against the static
    array before it touches CUDA, so refusals need no GPU: the pointers here
    are aligned stand-ins that are never dereferenced."""
    fake = ctypes.c_void_p(1 << 12)
    f = lib.pulscan_segment_maxima_noalloc
    assert f(fake, 1 << 22, 64, 64, fake, fake, None) == -6        # 2^21 segments x 64 widths > 2^20 slots
    assert f(fake, (1 << 21) + 1024, 256, 256, fake, fake, None) == -6   # 4098 segments x 256 > 2^20
    assert f(fake, 1 << 24, 5000, 8192, fake, fake, None) == -6     # z_max above 4096
    assert f(fake, 1 << 33, 4, 16, fake, fake, None) == -6          # bins would not fit 32 bits
    assert f(fake, 1023, 4, 16, fake, fake, None) == -1             # odd n
    assert f(fake, 1024, 32, 16, fake, fake, None) == -1            # segment_len < z_max
    assert f(ctypes.c_void_p((1 << 12) + 4), 1024, 4, 16, fake, fake, None) == -1   # unaligned power
    assert f(None, 1024, 4, 16, fake, fake, None) == -1
    assert lib.pulscan_last_error()
    h = ctypes.c_void_p()
    assert lib.pulscan_plan_create(ctypes.byref(h), 1 << 33, 4, 16, 6.0) == -6
