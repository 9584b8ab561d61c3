"""GB300 boxcar (unmatched-filter) search of Pulscan (arXiv 2406.15186).

Thin ctypes binding over ``libpulscan.so`` and its C ABI (``include/pulscan.h``).
The binding only marshals arguments: every step of the search runs in the
library's CUDA kernels (and cuFFT for the transform).  PyTorch is used, when
given, for device memory and streams only.  There is no CPU fallback: if the
library has not been built, ``load()`` raises.

Typical use (one series of n float32 samples already on the GPU)::

    import paper_2406_15186_gb300 as ps
    from paper_2406_15186_gb300 import build
    build.build()                                   # in-tree libpulscan.so, sm_103a
    plan = ps.Plan(n=n, z_max=1024, segment_len=4096, threshold_sigma=6.0)
    d_x, d_spec, d_power = plan.buffers("cuda")     # torch tensors sized for the plan
    d_x.copy_(x)
    plan.search(d_x, d_spec, d_power, use_graph=True)   # FFT, normalise, bank, threshold
    cands = plan.candidates()                       # numpy records (CAND_DTYPE)
    plan.autotune(d_power)                          # optional, once: the bank's launch shape

From host memory: ``plan.search_host(x_pinned)``; a stream of series:
``search_host_async`` on two plans in turn, then ``candidates``.  Batches
of uneven lengths: ``Plan(lengths=[...], ...)``; harmonic sums:
``Plan(..., numharm=H)``; the logsumexp statistic and its gradient:
``paper_2406_15186_gb300.lse``.
"""
import ctypes
import os

import numpy as np

__all__ = ["Plan", "PulscanError", "load", "lib_path", "CAND_DTYPE"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

CAND_DTYPE = np.dtype([("series", "<u4"), ("width", "<u4"), ("bin", "<u8"), ("power", "<f4"), ("sigma", "<f4"),
                       ("harmonics", "<u4"), ("reserved", "<u4")])
assert CAND_DTYPE.itemsize == 32


class PulscanError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pulscan error {code}: {msg}")
        self.code = code


class _Info(ctypes.Structure):
    _fields_ = [("n_series", ctypes.c_int64), ("x_floats", ctypes.c_int64), ("spec_floats", ctypes.c_int64),
                ("power_floats", ctypes.c_int64), ("total_segments", ctypes.c_int64), ("z_max", ctypes.c_int32),
                ("segment_len", ctypes.c_int32), ("threshold_sigma", ctypes.c_double),
                ("max_candidates", ctypes.c_int64)]


def lib_path():
    return os.path.join(_HERE, "libpulscan.so")


# name -> (restype, argtypes); mirrors include/pulscan.h
_P = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_SIGS = {
    "pulscan_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_double]),
    "pulscan_plan_create_batch": (ctypes.c_int, [ctypes.POINTER(_P), _I64P, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.c_double]),
    "pulscan_plan_destroy": (None, [_P]),
    "pulscan_plan_get_info": (ctypes.c_int, [_P, ctypes.POINTER(_Info)]),
    "pulscan_plan_offsets": (ctypes.c_int, [_P, _I64P, _I64P, _I64P, _I64P]),
    "pulscan_plan_create_harmonic": (ctypes.c_int, [ctypes.POINTER(_P), _I64P, ctypes.c_int32, ctypes.c_int32,
                                                    ctypes.c_int32, ctypes.c_double, ctypes.c_int32]),
    "pulscan_plan_stage_offsets": (ctypes.c_int, [_P, ctypes.c_int32, _I64P, _I64P, _I64P]),
    "pulscan_plan_set_trials": (ctypes.c_int, [_P, ctypes.c_double]),
    "pulscan_plan_set_widths": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "pulscan_plan_set_rblock": (ctypes.c_int, [_P, ctypes.c_int64]),
    "pulscan_plan_set_fidelity": (ctypes.c_int, [_P, ctypes.c_int32]),
    "pulscan_plan_autotune": (ctypes.c_int, [_P, _P, _P]),
    "pulscan_plan_tiling": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32)]),
    "pulscan_plan_set_tiling": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "pulscan_plan_set_pipeline": (ctypes.c_int, [_P, ctypes.c_int64]),
    "pulscan_plan_set_fused": (ctypes.c_int, [_P, ctypes.c_int32]),
    "pulscan_plan_pipeline_parts": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "pulscan_plan_test_wait_timeout": (ctypes.c_int, [_P, ctypes.c_int32]),
    "pulscan_plan_thresholds": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]),
    "pulscan_threshold_power": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.POINTER(ctypes.c_float)]),
    "pulscan_rfft": (ctypes.c_int, [_P, _P, _P, _P]),
    "pulscan_power_normalise": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "pulscan_boxcar_search": (ctypes.c_int, [_P, _P, _P]),
    "pulscan_candidates": (ctypes.c_int, [_P, _P, ctypes.c_int64, _I64P, _P]),
    "pulscan_segment_maxima": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "pulscan_segment_maxima_noalloc": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P, _P,
                                                      _P]),
    "pulscan_search": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, _P]),
    "pulscan_search_host": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _I64P, ctypes.c_int, _P]),
    "pulscan_search_host_async": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "pulscan_lse_forward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_float, _P]),
    "pulscan_lse_backward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_float, _P]),
    "pulscan_inject": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "pulscan_amplitude_grad": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "pulscan_plan_enable_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "pulscan_plan_counters": (ctypes.c_int, [_P, _I64P, ctypes.c_int32]),
    "pulscan_plan_set_defer_capacity": (ctypes.c_int, [_P, ctypes.c_int64]),
    "pulscan_plan_set_defer_form": (ctypes.c_int, [_P, ctypes.c_int32]),
    "pulscan_plan_defer_form": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "pulscan_plan_timings": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int32]),
    "pulscan_measure_add_peak": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int32, _P]),
    "pulscan_last_error": (ctypes.c_char_p, []),
    "pulscan_version": (ctypes.c_int, []),
}


def load():
    """Load libpulscan.so (built by ``paper_2406_15186_gb300.build``)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2406_15186_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _check(rc):
    if rc != 0:
        raise PulscanError(rc, _LIB.pulscan_last_error().decode())


def threshold_power(shape, n_trials, sigma_thr):
    """pulscan_threshold_power: the FP32 power threshold of one width (host only)."""
    t = ctypes.c_float(0.0)
    _check(load().pulscan_threshold_power(float(shape), float(n_trials), float(sigma_thr), ctypes.byref(t)))
    return t.value


def measure_add_peak(reps=5, stream=None):
    """The GPU's FP32 add rate (pulscan_measure_add_peak): adds/s with packed
    pairs and with scalar adds, and the SM clock (MHz) during each."""
    lib = load()
    out = (ctypes.c_double * 4)()
    _check(lib.pulscan_measure_add_peak(out, 4, int(reps), _stream(stream)))
    return {"packed_adds_per_s": out[0], "scalar_adds_per_s": out[1], "packed_sm_mhz": out[2],
            "scalar_sm_mhz": out[3]}


def _ptr(a):
    """Device/host address of a torch tensor, a numpy array or a raw int."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    raise TypeError(f"cannot take the address of {type(a)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


WIDTHS_ALL, WIDTHS_STEP, WIDTHS_LOG2 = 0, 1, 2
FIDELITY_EXACT, FIDELITY_PAPER_GPU = 0, 1


class Plan:
    """A search plan: one series (``n``) or a batch (``lengths``)."""

    def __init__(self, n=None, z_max=256, segment_len=1024, threshold_sigma=6.0, lengths=None, numharm=1):
        lib = load()
        h = _P()
        if numharm != 1:
            ls = [int(n)] if lengths is None else [int(v) for v in lengths]
            arr = (ctypes.c_int64 * len(ls))(*ls)
            _check(lib.pulscan_plan_create_harmonic(ctypes.byref(h), arr, len(ls), int(z_max), int(segment_len),
                                                    float(threshold_sigma), int(numharm)))
        elif lengths is None:
            _check(lib.pulscan_plan_create(ctypes.byref(h), int(n), int(z_max), int(segment_len),
                                           float(threshold_sigma)))
        else:
            arr = (ctypes.c_int64 * len(lengths))(*[int(v) for v in lengths])
            _check(lib.pulscan_plan_create_batch(ctypes.byref(h), arr, len(lengths), int(z_max),
                                                 int(segment_len), float(threshold_sigma)))
        self.numharm = int(numharm)
        self._h = h
        info = _Info()
        _check(lib.pulscan_plan_get_info(h, ctypes.byref(info)))
        self.n_series = info.n_series
        self.x_floats = info.x_floats
        self.spec_floats = info.spec_floats
        self.power_floats = info.power_floats
        self.total_segments = info.total_segments
        self.z_max = info.z_max
        self.segment_len = info.segment_len
        self.threshold_sigma = info.threshold_sigma
        self.max_candidates = info.max_candidates

    def close(self):
        if getattr(self, "_h", None):
            load().pulscan_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- layout
    def offsets(self):
        """(x_off, spec_off, power_off, seg_off): int64 arrays of n_series + 1."""
        n = self.n_series + 1
        outs = [np.zeros(n, dtype=np.int64) for _ in range(4)]
        _check(load().pulscan_plan_offsets(self._h, *[o.ctypes.data_as(_I64P) for o in outs]))
        return tuple(outs)

    def thresholds(self, series=0):
        out = np.zeros(self.z_max, dtype=np.float32)
        _check(load().pulscan_plan_thresholds(self._h, int(series),
                                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def set_trials(self, n_trials):
        _check(load().pulscan_plan_set_trials(self._h, float(n_trials)))

    def set_widths(self, mode=0, step=1):
        """Searched widths: WIDTHS_ALL, WIDTHS_STEP (z mod step == 0) or WIDTHS_LOG2 (z a power of two)."""
        _check(load().pulscan_plan_set_widths(self._h, int(mode), int(step)))

    def set_fidelity(self, mode):
        """FIDELITY_EXACT (default) or FIDELITY_PAPER_GPU (median of medians + polynomial log p)."""
        _check(load().pulscan_plan_set_fidelity(self._h, int(mode)))

    def autotune(self, d_power, stream=None):
        """Pick the bank's warps per CTA and launch form by timing the search on d_power."""
        _check(load().pulscan_plan_autotune(self._h, _ptr(d_power), _stream(stream)))
        return self.tiling()

    def set_pipeline(self, part_bins):
        """Parts of about part_bins bins for the pipelined captured search (0: off)."""
        _check(load().pulscan_plan_set_pipeline(self._h, int(part_bins)))

    def set_fused(self, on):
        """Fused normalisation + search in search(): P formed in the bank, d_power unused."""
        _check(load().pulscan_plan_set_fused(self._h, int(bool(on))))

    def pipeline_parts(self):
        n = ctypes.c_int64(0)
        _check(load().pulscan_plan_pipeline_parts(self._h, ctypes.byref(n)))
        return int(n.value)

    def set_tiling(self, warps, persistent=-1, packed=0):
        _check(load().pulscan_plan_set_tiling(self._h, int(warps), int(persistent), int(packed)))

    def tiling(self):
        """(warps per CTA, persistent, packed) of the bank's launch shape."""
        w, m, k = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        _check(load().pulscan_plan_tiling(self._h, ctypes.byref(w), ctypes.byref(m), ctypes.byref(k)))
        return w.value, m.value, k.value

    def test_wait_timeout(self, limit_us=20):
        """Arm the next search to exercise its timeout path (pulscan_plan_test_wait_timeout)."""
        _check(load().pulscan_plan_test_wait_timeout(self._h, int(limit_us)))

    def set_rblock(self, block_width):
        """Report block indices floor(bin / block_width) instead of bins (0: exact bins)."""
        _check(load().pulscan_plan_set_rblock(self._h, int(block_width)))

    # -- the path
    def rfft(self, d_x, d_spec, stream=None):
        _check(load().pulscan_rfft(self._h, _ptr(d_x), _ptr(d_spec), _stream(stream)))

    def power_normalise(self, d_spec, d_power, d_stats=None, stream=None):
        _check(load().pulscan_power_normalise(self._h, _ptr(d_spec), _ptr(d_power), _ptr(d_stats),
                                              _stream(stream)))

    def boxcar_search(self, d_power, stream=None):
        _check(load().pulscan_boxcar_search(self._h, _ptr(d_power), _stream(stream)))

    def candidates(self, cap=None, stream=None, allow_overflow=False):
        """Candidates of the last search as a numpy structured array (CAND_DTYPE)."""
        lib = load()
        n = ctypes.c_int64(0)
        size = 4096 if cap is None else int(cap)
        while True:
            out = np.empty(size, dtype=CAND_DTYPE)
            rc = lib.pulscan_candidates(self._h, out.ctypes.data, size, ctypes.byref(n), _stream(stream))
            if rc == -4 and cap is None and size < n.value <= self.max_candidates:
                size = n.value          # grow to the true count and read again
                continue
            if rc == -4 and allow_overflow:
                return out[:size], n.value
            _check(rc)
            return out[: n.value]

    def segment_maxima(self, d_power, d_max, d_argmax, stream=None):
        _check(load().pulscan_segment_maxima(self._h, _ptr(d_power), _ptr(d_max), _ptr(d_argmax),
                                             _stream(stream)))

    def search(self, d_x, d_spec, d_power, use_graph=False, stream=None):
        _check(load().pulscan_search(self._h, _ptr(d_x), _ptr(d_spec), _ptr(d_power), int(bool(use_graph)),
                                     _stream(stream)))

    def search_host_async(self, h_x, use_graph=True, stream=None):
        """Enqueue the copy of h_x (pinned tensor or numpy array, kept alive by
        the caller until the copy has run) and the search; no wait.  Collect
        with candidates(stream=...)."""
        _check(load().pulscan_search_host_async(self._h, _ptr(h_x), int(bool(use_graph)), _stream(stream)))

    def search_host(self, h_x, use_graph=True, cap=None, stream=None):
        """Whole path from host memory (numpy array or pinned CPU tensor); returns candidates."""
        lib = load()
        n = ctypes.c_int64(0)
        size = min(self.max_candidates, 1 << 16) if cap is None else int(cap)
        out = np.empty(size, dtype=CAND_DTYPE)
        rc = lib.pulscan_search_host(self._h, _ptr(h_x), out.ctypes.data, size, ctypes.byref(n),
                                     int(bool(use_graph)), _stream(stream))
        if rc == -4 and cap is None and n.value <= self.max_candidates:
            return self.candidates(cap=n.value, stream=stream)   # more than the first read held
        _check(rc)
        return out[: n.value]

    # -- timing
    def enable_timing(self, on=True):
        """on: True/1 every stage's events, 2 the boxcar search kernel's only, False/0 none."""
        _check(load().pulscan_plan_enable_timing(self._h, 2 if on == 2 else int(bool(on))))

    def timings(self):
        """ms of the last [rfft, normalise, boxcar kernel, deferred blocks, finalise, segment maxima,
        harmonic sums] (-1: not run)."""
        out = (ctypes.c_float * 7)()
        _check(load().pulscan_plan_timings(self._h, out, 7))
        return list(out)

    def stage_offsets(self, harmonics):
        """(power offsets, first segments, bins) of harmonic stage H per series (entry n_series: the end)."""
        po = np.zeros(self.n_series + 1, dtype=np.int64)
        so = np.zeros(self.n_series + 1, dtype=np.int64)
        nb = np.zeros(self.n_series + 1, dtype=np.int64)
        _check(load().pulscan_plan_stage_offsets(self._h, int(harmonics), po.ctypes.data_as(_I64P),
                                                 so.ctypes.data_as(_I64P), nb.ctypes.data_as(_I64P)))
        return po, so, nb

    def counters(self):
        """[deferred blocks, deferred capacity, candidates, candidate capacity] of the last search."""
        out = np.zeros(4, dtype=np.int64)
        _check(load().pulscan_plan_counters(self._h, out.ctypes.data_as(_I64P), 4))
        return [int(v) for v in out]

    def set_defer_capacity(self, cap):
        _check(load().pulscan_plan_set_defer_capacity(self._h, int(cap)))

    def set_defer_form(self, form):
        """Deferred blocks inspected by three warps per block (0) or one warp per block (1)."""
        _check(load().pulscan_plan_set_defer_form(self._h, int(form)))

    def defer_form(self):
        f = ctypes.c_int32(0)
        _check(load().pulscan_plan_defer_form(self._h, ctypes.byref(f)))
        return f.value

    # -- convenience: device buffers sized for this plan (torch)
    def buffers(self, device="cuda"):
        import torch
        x = torch.zeros(self.x_floats, dtype=torch.float32, device=device)
        spec = torch.zeros(self.spec_floats, dtype=torch.float32, device=device)
        power = torch.zeros(self.power_floats, dtype=torch.float32, device=device)
        return x, spec, power
