"""ctypes binding of libssp (``include/ssp.h``): argument marshalling only.

The function names are the C ABI's.  Every step of the periodogram runs in
the library's CUDA kernels; nothing here computes.  ``lib()`` raises if the
shared library has not been built (``paper_2111_07396_gb300.build.build()``):
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "libssp.so")

SSP_SS, SSP_SP, SSP_SPG = 0, 1, 2
SSP_FP64, SSP_FP32C = 0, 1
SSP_OK, SSP_ERR_ARG, SSP_ERR_NOMEM, SSP_ERR_CUDA, SSP_ERR_TIMEOUT, SSP_ERR_UNSUPPORTED = (
    0, -1, -2, -3, -4, -5)
SSP_ERR_BUSY, SSP_PENDING = -6, 1
SSP_FAULT_ALLOC, SSP_FAULT_STALL, SSP_FAULT_UPLOAD = 1, 2, 3
VARIANTS = {"ss": SSP_SS, "sp": SSP_SP, "spg": SSP_SPG, SSP_SS: SSP_SS, SSP_SP: SSP_SP,
            SSP_SPG: SSP_SPG}
PRECISIONS = {"fp64": SSP_FP64, "fp32c": SSP_FP32C, SSP_FP64: SSP_FP64, SSP_FP32C: SSP_FP32C}


class ssp_params(ctypes.Structure):
    _fields_ = [("spans", ctypes.c_double * 3), ("alpha", ctypes.c_double),
                ("periodic", ctypes.c_int), ("precision", ctypes.c_int),
                ("hbm_fraction", ctypes.c_double), ("span", ctypes.c_double)]


class ssp_phase_time(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double)]


class ssp_server_config(ctypes.Structure):
    _fields_ = [("max_batch_ptf", ctypes.c_double), ("max_wait_ms", ctypes.c_double),
                ("max_in_flight", ctypes.c_int64), ("stall_ms", ctypes.c_double),
                ("slots", ctypes.c_int64), ("device_bytes", ctypes.c_double)]


PHASES = ("prep", "pgram_ss", "pgram_sp", "redo", "argmax")


class SSPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


_lib = None


def lib():
    """Load libssp.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(SO):
            raise RuntimeError(f"libssp.so is not built ({SO}); run "
                               "paper_2111_07396_gb300.build.build() first")
        L = ctypes.CDLL(SO)
        P, i64 = ctypes.c_void_p, ctypes.c_int64
        L.ssp_default_params.argtypes = [ctypes.POINTER(ssp_params)]
        L.ssp_default_params.restype = None
        L.ssp_periodogram.argtypes = [P, P, P, P, i64, P, i64, ctypes.c_int,
                                      ctypes.POINTER(ssp_params), P, P]
        L.ssp_periodogram.restype = ctypes.c_int
        L.ssp_periodogram_device.argtypes = [P, P, P, P, i64, P, i64, ctypes.c_int,
                                             ctypes.POINTER(ssp_params), P, P, P]
        L.ssp_periodogram_device.restype = ctypes.c_int
        L.ssp_status_string.argtypes = [ctypes.c_int]
        L.ssp_status_string.restype = ctypes.c_char_p
        L.ssp_last_error.argtypes = []
        L.ssp_last_error.restype = ctypes.c_char_p
        L.ssp_version.argtypes = []
        L.ssp_version.restype = ctypes.c_char_p
        L.ssp_periodogram_device_noalloc.argtypes = [P, P, P, P, i64, P, i64, ctypes.c_int,
                                                     ctypes.POINTER(ssp_params), P, P, P]
        L.ssp_periodogram_device_noalloc.restype = ctypes.c_int
        L.ssp_fold_fixed.argtypes = [P, i64, ctypes.c_double, P]
        L.ssp_fold_fixed.restype = ctypes.c_int
        L.ssp_profile_enable.argtypes = [ctypes.c_int]
        L.ssp_profile_enable.restype = None
        L.ssp_profile_read.argtypes = [ctypes.POINTER(ssp_phase_time), ctypes.c_int]
        L.ssp_profile_read.restype = ctypes.c_int
        L.ssp_server_create.argtypes = [P, i64, ctypes.POINTER(ssp_params),
                                        ctypes.POINTER(ssp_server_config), ctypes.POINTER(P)]
        L.ssp_server_create.restype = ctypes.c_int
        L.ssp_server_submit.argtypes = [P, P, P, P, i64, ctypes.c_int, ctypes.POINTER(i64)]
        L.ssp_server_submit.restype = ctypes.c_int
        L.ssp_server_next.argtypes = [P, ctypes.c_int, ctypes.POINTER(i64)]
        L.ssp_server_next.restype = ctypes.c_int
        L.ssp_server_poll.argtypes = [P, i64, ctypes.c_int, P, P, P]
        L.ssp_server_poll.restype = ctypes.c_int
        L.ssp_server_destroy.argtypes = [P]
        L.ssp_server_destroy.restype = ctypes.c_int
        L.ssp_autotune.argtypes = [P, P, P, P, i64, P, i64, ctypes.c_int,
                                   ctypes.POINTER(ssp_params), ctypes.c_double, P]
        L.ssp_autotune.restype = ctypes.c_int
        L.ssp_autotune_clear.argtypes = []
        L.ssp_autotune_clear.restype = None
        L.ssp_measure_alu_peaks.argtypes = [P, P]
        L.ssp_measure_alu_peaks.restype = ctypes.c_int
        L.ssp_search_refine.argtypes = [P, P, P, P, i64, P, i64, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.POINTER(ssp_params), P,
                                        P]
        L.ssp_search_refine.restype = ctypes.c_int
        L.ssp_plan_create.argtypes = [P, i64, i64, ctypes.c_int, ctypes.POINTER(ssp_params),
                                      ctypes.POINTER(P)]
        L.ssp_plan_create.restype = ctypes.c_int
        L.ssp_plan_execute.argtypes = [P, P, P, P, P, P, P, P]
        L.ssp_plan_execute.restype = ctypes.c_int
        L.ssp_plan_destroy.argtypes = [P]
        L.ssp_plan_destroy.restype = ctypes.c_int
        L.ssp_test_fault.argtypes = [ctypes.c_int, ctypes.c_int]
        L.ssp_test_fault.restype = ctypes.c_int
        _lib = L
    return _lib


def ssp_default_params(precision="fp32c", alpha=None, spans=None, hbm_fraction=None,
                       periodic=True, span=0.0) -> ssp_params:
    p = ssp_params()
    lib().ssp_default_params(ctypes.byref(p))
    p.precision = PRECISIONS[precision]
    p.periodic = 1 if periodic else 0
    p.span = float(span)
    if alpha is not None:
        p.alpha = float(alpha)
    if spans is not None:
        for k in range(3):
            p.spans[k] = float(spans[k])
    if hbm_fraction is not None:
        p.hbm_fraction = float(hbm_fraction)
    return p


def ssp_status_string(status: int) -> str:
    return lib().ssp_status_string(int(status)).decode()


def ssp_last_error() -> str:
    return lib().ssp_last_error().decode()


def ssp_version() -> str:
    return lib().ssp_version().decode()


def ssp_fold_fixed(tt, f):
    """The kernels' FP32C phase fold on the host: floor(frac(fl(tt*f)) * 2^64)."""
    tt = _f64(tt)
    out = np.empty(tt.size, dtype=np.uint64)
    _check(lib().ssp_fold_fixed(_ptr(tt), tt.size, float(f), _ptr(out)))
    return out


def ssp_profile_enable(on: bool = True) -> None:
    lib().ssp_profile_enable(1 if on else 0)


def ssp_profile_read(reset: bool = True) -> dict:
    out = (ssp_phase_time * len(PHASES))()
    _check(lib().ssp_profile_read(out, 1 if reset else 0))
    return {name: (int(out[k].launches), float(out[k].ms)) for k, name in enumerate(PHASES)}


def _check(rc: int):
    if rc != SSP_OK:
        raise SSPError(rc, f"{ssp_status_string(rc)}: {ssp_last_error()}")


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _expect(a, name, f64, count, out=False):
    """Checks an array the library will read or write before the call: element
    type (float64, or float32 for FP32C powers), exactly `count` elements, a
    contiguous layout and, for outputs in host memory, writeable.  A buffer of
    the wrong type or size would otherwise be read or written past its end.
    Raw device addresses (ints) are taken as given."""
    if isinstance(a, int):
        return
    if hasattr(a, "data_ptr"):
        import torch
        want = torch.float64 if f64 else torch.float32
        ok = a.dtype == want and a.numel() == count and a.is_contiguous()
        got = f"{a.dtype}, {a.numel()} elements"
    else:
        want = np.float64 if f64 else np.float32
        ok = (isinstance(a, np.ndarray) and a.dtype == want and a.size == count
              and a.flags.c_contiguous and (a.flags.writeable or not out))
        got = f"{getattr(a, 'dtype', type(a).__name__)}, {getattr(a, 'size', '?')} elements"
    if not ok:
        kind = "float64" if f64 else "float32"
        raise ValueError(f"{name} must be a contiguous{' writeable' if out else ''} {kind} array "
                         f"of {count} elements (got {got})")


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def ssp_periodogram(t, y, dy, n_per_object, freq_grid, variant="ss", precision="fp32c",
                    alpha=9.0, spans=None, params=None, out_power=None, out_best_period=None,
                    periodic=True, span=0.0):
    """Host-memory entry point.  Arrays may be numpy arrays or CPU torch
    tensors (pinned or not); returns (power [n_objects, n_freq], best_period)."""
    p = params if params is not None else ssp_default_params(precision, alpha, spans,
                                                             periodic=periodic, span=span)
    t_, y_, dy_ = (_host_array(a) for a in (t, y, dy))
    npo = np.ascontiguousarray(n_per_object, dtype=np.int64)
    fq = _host_array(freq_grid)
    n_obj, n_freq = int(npo.size), _numel(fq)
    dt = np.float64 if p.precision == SSP_FP64 else np.float32
    if out_power is None:
        out_power = np.empty((n_obj, n_freq), dtype=dt)
    if out_best_period is None:
        out_best_period = np.empty(n_obj, dtype=np.float64)
    n_pts = int(npo.sum())
    for a, name in ((t_, "t"), (y_, "y"), (dy_, "dy")):
        _expect(a, name, True, n_pts)
    _expect(out_power, "out_power", p.precision == SSP_FP64, n_obj * n_freq, out=True)
    _expect(out_best_period, "out_best_period", True, n_obj, out=True)
    rc = lib().ssp_periodogram(_host_ptr(t_), _host_ptr(y_), _host_ptr(dy_), _ptr(npo), n_obj,
                               _host_ptr(fq), n_freq, VARIANTS[variant], ctypes.byref(p),
                               _host_ptr(out_power), _host_ptr(out_best_period))
    _check(rc)
    return out_power, out_best_period


def ssp_periodogram_device(t, y, dy, n_per_object, freq_grid, out_power, out_best_period,
                           variant="ss", precision="fp32c", alpha=9.0, spans=None, params=None,
                           stream=None):
    """Device-memory entry point.  t, y, dy, freq_grid, out_power and
    out_best_period are CUDA torch tensors (or raw device addresses as ints);
    n_per_object is a host array.  Enqueued on `stream` (a torch stream or a
    raw cudaStream_t address; default: torch's current stream)."""
    p = params if params is not None else ssp_default_params(precision, alpha, spans)
    npo = np.ascontiguousarray(n_per_object, dtype=np.int64)
    n_freq = int(freq_grid.numel()) if hasattr(freq_grid, "numel") else None
    if n_freq is None:
        raise ValueError("freq_grid must be a tensor (its length is needed)")
    _expect_device(p, npo, n_freq, t, y, dy, freq_grid, out_power, out_best_period)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    s = stream if isinstance(stream, int) else stream.cuda_stream
    rc = lib().ssp_periodogram_device(_dev_ptr(t), _dev_ptr(y), _dev_ptr(dy), _ptr(npo),
                                      int(npo.size), _dev_ptr(freq_grid), n_freq,
                                      VARIANTS[variant], ctypes.byref(p), _dev_ptr(out_power),
                                      _dev_ptr(out_best_period), ctypes.c_void_p(s))
    _check(rc)
    return out_power, out_best_period


def ssp_periodogram_device_noalloc(t, y, dy, n_per_object, freq_grid, out_power, out_best_period,
                                   variant="ss", precision="fp32c", alpha=9.0, spans=None,
                                   params=None, stream=None):
    """As ssp_periodogram_device, with no device allocation: scratch lives in
    the library's fixed device array (see include/ssp.h for its limits)."""
    p = params if params is not None else ssp_default_params(precision, alpha, spans)
    npo = np.ascontiguousarray(n_per_object, dtype=np.int64)
    if not hasattr(freq_grid, "numel"):
        raise ValueError("freq_grid must be a tensor (its length is needed)")
    _expect_device(p, npo, int(freq_grid.numel()), t, y, dy, freq_grid, out_power,
                   out_best_period)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    s = stream if isinstance(stream, int) else stream.cuda_stream
    rc = lib().ssp_periodogram_device_noalloc(
        _dev_ptr(t), _dev_ptr(y), _dev_ptr(dy), _ptr(npo), int(npo.size), _dev_ptr(freq_grid),
        int(freq_grid.numel()), VARIANTS[variant], ctypes.byref(p), _dev_ptr(out_power),
        _dev_ptr(out_best_period), ctypes.c_void_p(s))
    _check(rc)
    return out_power, out_best_period


def ssp_autotune(t, y, dy, n_per_object, freq_grid, variant="ss", precision="fp32c", alpha=9.0,
                 spans=None, params=None, budget_ptf=0.0):
    """Times the threads-per-CTA candidates of every length range these
    objects occupy and keeps the fastest; returns the five ranges' choices."""
    p = params if params is not None else ssp_default_params(precision, alpha, spans)
    t_, y_, dy_, fq = _f64(t), _f64(y), _f64(dy), _f64(freq_grid)
    npo = np.ascontiguousarray(n_per_object, dtype=np.int64)
    for a, name in ((t_, "t"), (y_, "y"), (dy_, "dy")):
        _expect(a, name, True, int(npo.sum()))
    out = np.zeros(5, dtype=np.int32)
    _check(lib().ssp_autotune(_ptr(t_), _ptr(y_), _ptr(dy_), _ptr(npo), int(npo.size), _ptr(fq),
                              int(fq.size), VARIANTS[variant], ctypes.byref(p), float(budget_ptf),
                              _ptr(out)))
    return out


def ssp_measure_alu_peaks():
    """(FP32, FP64) FMA-chain peaks of the current GPU in TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = lib().ssp_measure_alu_peaks(ctypes.byref(a), ctypes.byref(b))
    if rc:
        raise SSPError(rc, "ALU peak microbenchmark failed")
    return a.value, b.value


def ssp_search_refine(t, y, dy, n_per_object, coarse_grid, coarse_variant="sp",
                      fine_variant="ss", n_peaks=3, n_fine=64, precision="fp32c", alpha=9.0,
                      spans=None, params=None, periodic=True):
    """Coarse search, then the fine variant on dense grids around each
    object's top peaks; returns (best_period[n_objects], best_power[n_objects])."""
    p = params if params is not None else ssp_default_params(precision, alpha, spans,
                                                             periodic=periodic)
    t_, y_, dy_, cg = _f64(t), _f64(y), _f64(dy), _f64(coarse_grid)
    npo = np.ascontiguousarray(n_per_object, dtype=np.int64)
    for a, name in ((t_, "t"), (y_, "y"), (dy_, "dy")):
        _expect(a, name, True, int(npo.sum()))
    bp, bw = np.empty(npo.size), np.empty(npo.size)
    _check(lib().ssp_search_refine(_ptr(t_), _ptr(y_), _ptr(dy_), _ptr(npo), int(npo.size),
                                   _ptr(cg), int(cg.size), VARIANTS[coarse_variant],
                                   VARIANTS[fine_variant], int(n_peaks), int(n_fine),
                                   ctypes.byref(p), _ptr(bp), _ptr(bw)))
    return bp, bw


class Plan:
    """A launch plan (ssp_plan_create / execute / destroy): the device pipeline
    of one shape captured into a CUDA graph, run on new device arrays."""

    def __init__(self, n_per_object, n_freq, variant="ss", precision="fp32c", alpha=9.0,
                 spans=None, params=None):
        self._p = params if params is not None else ssp_default_params(precision, alpha, spans)
        self._npo = np.ascontiguousarray(n_per_object, dtype=np.int64)
        self.n_freq = int(n_freq)
        h = ctypes.c_void_p()
        _check(lib().ssp_plan_create(_ptr(self._npo), int(self._npo.size), self.n_freq,
                                     VARIANTS[variant], ctypes.byref(self._p), ctypes.byref(h)))
        self._h = h

    def ssp_plan_execute(self, t, y, dy, freq_grid, out_power, out_best_period, stream=None):
        """Device arrays (torch CUDA tensors or raw addresses); enqueued on
        `stream` (default: torch's current stream)."""
        _expect_device(self._p, self._npo, self.n_freq, t, y, dy, freq_grid, out_power,
                       out_best_period)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream()
        s = stream if isinstance(stream, int) else stream.cuda_stream
        _check(lib().ssp_plan_execute(self._h, _dev_ptr(t), _dev_ptr(y), _dev_ptr(dy),
                                      _dev_ptr(freq_grid), _dev_ptr(out_power),
                                      _dev_ptr(out_best_period), ctypes.c_void_p(s)))

    def ssp_plan_destroy(self) -> None:
        if self._h:
            h, self._h = self._h, None
            _check(lib().ssp_plan_destroy(h))

    execute, close = ssp_plan_execute, ssp_plan_destroy

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ssp_test_fault(kind, count=1) -> None:
    """Testing only: make the library's next `count` device allocations fail
    (SSP_FAULT_ALLOC), its server's next `count` batches count as stalled
    (SSP_FAULT_STALL) or its server's next `count` request uploads fail
    (SSP_FAULT_UPLOAD).  Needs SSP_TESTING=1 in the environment."""
    _check(lib().ssp_test_fault(int(kind), int(count)))


def ssp_autotune_clear() -> None:
    lib().ssp_autotune_clear()


class Server:
    """The serving API (ssp_server_create / submit / next / poll / destroy):
    one light curve per request, results collected asynchronously.  Host
    numpy arrays in and out; the batching, copies and kernels are the
    library's."""

    def __init__(self, freq_grid, precision="fp32c", alpha=9.0, spans=None, params=None,
                 max_batch_ptf=0.0, max_wait_ms=0.0, max_in_flight=0, stall_ms=0.0, slots=0,
                 device_bytes=0.0):
        self._p = params if params is not None else ssp_default_params(precision, alpha, spans)
        self.freq = _f64(freq_grid)
        self.n_freq = int(self.freq.size)
        self.dtype = np.float64 if self._p.precision == SSP_FP64 else np.float32
        cfg = ssp_server_config(float(max_batch_ptf), float(max_wait_ms), int(max_in_flight),
                                float(stall_ms), int(slots), float(device_bytes))
        h = ctypes.c_void_p()
        _check(lib().ssp_server_create(_ptr(self.freq), self.n_freq, ctypes.byref(self._p),
                                       ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def ssp_server_submit(self, t, y, dy, variant="ss") -> int:
        t_, y_, dy_ = _f64(t), _f64(y), _f64(dy)
        if not (t_.size == y_.size == dy_.size):
            raise ValueError("t, y and dy must have the same length")
        ticket = ctypes.c_int64()
        _check(lib().ssp_server_submit(self._h, _ptr(t_), _ptr(y_), _ptr(dy_), t_.size,
                                       VARIANTS[variant], ctypes.byref(ticket)))
        return int(ticket.value)

    def ssp_server_next(self, wait_ms=0):
        """Ticket of a finished request not reported before, or None."""
        ticket = ctypes.c_int64()
        rc = lib().ssp_server_next(self._h, int(wait_ms), ctypes.byref(ticket))
        if rc == SSP_PENDING:
            return None
        _check(rc)
        return int(ticket.value)

    def ssp_server_poll(self, ticket, wait_ms=0):
        """(power [n_freq], best_period, latency_ms) once finished, else None."""
        power = np.empty(self.n_freq, dtype=self.dtype)
        best, lat = ctypes.c_double(), ctypes.c_double()
        rc = lib().ssp_server_poll(self._h, int(ticket), int(wait_ms), _ptr(power),
                                   ctypes.byref(best), ctypes.byref(lat))
        if rc == SSP_PENDING:
            return None
        _check(rc)
        return power, float(best.value), float(lat.value)

    def ssp_server_destroy(self) -> None:
        if self._h:
            h, self._h = self._h, None
            _check(lib().ssp_server_destroy(h))

    submit, next, poll, close = ssp_server_submit, ssp_server_next, ssp_server_poll, \
        ssp_server_destroy

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _numel(a):
    return int(a.numel()) if hasattr(a, "numel") else int(a.size)


def _host_array(a):
    if hasattr(a, "data_ptr"):  # torch CPU tensor
        import torch
        if a.is_cuda:
            raise ValueError("ssp_periodogram takes host arrays; use ssp_periodogram_device")
        if a.dtype != torch.float64:
            raise ValueError("host tensors must be float64")
        return a.contiguous()
    return _f64(a)


def _host_ptr(a):
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return _ptr(a)


def _expect_device(p, npo, n_freq, t, y, dy, freq_grid, out_power, out_best_period):
    # element types and counts of a device call's arrays (see _expect)
    n_pts, n_obj = int(npo.sum()), int(npo.size)
    for a, name in ((t, "t"), (y, "y"), (dy, "dy")):
        _expect(a, name, True, n_pts)
    _expect(freq_grid, "freq_grid", True, n_freq)
    _expect(out_power, "out_power", p.precision == SSP_FP64, n_obj * n_freq, out=True)
    _expect(out_best_period, "out_best_period", True, n_obj, out=True)


def _dev_ptr(a):
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    if not a.is_cuda or not a.is_contiguous():
        raise ValueError("device entry point needs contiguous CUDA tensors")
    return ctypes.c_void_p(a.data_ptr())
