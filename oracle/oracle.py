"""ctypes binding of the plain FP64 C oracle (``ssp_oracle.c``).

Test infrastructure only.  ``build()`` compiles ``libssp_oracle.so`` next to
this file with gcc and ``-ffp-contract=off`` (no fused multiply-adds, so the
phase fold rounds exactly as written).  Every function here marshals numpy
arrays and calls the C code; no arithmetic of the method lives in Python.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "build", "lib", "SS", "SP", "SPG", "DEFAULT_SPANS", "prep", "phase", "fold_sort",
    "half_width", "vsmlsq", "runline_raw", "runline", "tie_average", "supsmu",
    "supsmu_sp", "supsmu_spg", "chi2", "power_one", "periodogram", "peaks", "fine_grid",
    "search_refine",
]

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ssp_oracle.c")
SO = os.path.join(HERE, "libssp_oracle.so")

SS, SP, SPG = 0, 1, 2
DEFAULT_SPANS = (0.05, 0.2, 0.5)  # Listing 1: tweeter, midrange, woofer

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C, FP64, no FMA contraction)."""
    if (not force and os.path.exists(SO)
            and os.path.getmtime(SO) >= max(os.path.getmtime(SRC),
                                            os.path.getmtime(os.path.join(HERE, "ssp_oracle.h")))):
        return SO
    tmp = SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, SO)
    return SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(SO)
            d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
            P = ctypes.c_void_p
            L.ssp_oracle_prep.argtypes = [i, P, P, P, P, P, P]
            L.ssp_oracle_phase.argtypes = [d, d]
            L.ssp_oracle_phase.restype = d
            L.ssp_oracle_fold_sort.argtypes = [i, P, d, P, P]
            L.ssp_oracle_half_width.argtypes = [i, d]
            L.ssp_oracle_half_width.restype = i
            L.ssp_oracle_vsmlsq.argtypes = [i, P]
            L.ssp_oracle_vsmlsq.restype = d
            L.ssp_oracle_runline_raw.argtypes = [i, P, P, P, d, i, d, P, P]
            L.ssp_oracle_runline.argtypes = [i, P, P, P, d, i, d, P, P]
            L.ssp_oracle_tie_average.argtypes = [i, P, P, P]
            L.ssp_oracle_supsmu.argtypes = [i, P, P, P, i, d, d, P, P]
            L.ssp_oracle_supsmu_sp.argtypes = [i, P, P, P, i, d, P, P]
            L.ssp_oracle_supsmu_spg.argtypes = [i, P, P, P, i, P, P, P]
            L.ssp_oracle_supsmu_spg.restype = None
            L.ssp_oracle_chi2.argtypes = [i, P, P, P]
            L.ssp_oracle_chi2.restype = d
            L.ssp_oracle_power_one.argtypes = [i, P, P, P, d, i, d, P, i, d]
            L.ssp_oracle_power_one.restype = d
            L.ssp_oracle_periodogram.argtypes = [P, P, P, P, i64, P, i64, i, d, P, i, d, i, P, P]
            L.ssp_oracle_periodogram.restype = i
            L.ssp_oracle_peaks.argtypes = [P, i64, i, P]
            L.ssp_oracle_peaks.restype = None
            L.ssp_oracle_fine_grid.argtypes = [P, i64, i64, i, P]
            L.ssp_oracle_fine_grid.restype = None
            L.ssp_oracle_search_refine.argtypes = [P, P, P, P, i64, P, i64, i, i, d, P, i, i, i, i,
                                                   P, P]
            L.ssp_oracle_search_refine.restype = i
            _lib = L
        return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _spans(spans):
    return _f64(DEFAULT_SPANS if spans is None else spans)


def prep(t, y, dy):
    t, y, dy = _f64(t), _f64(y), _f64(dy)
    n = t.size
    tt, w = np.empty(n), np.empty(n)
    chi0 = ctypes.c_double()
    lib().ssp_oracle_prep(n, _p(t), _p(y), _p(dy), _p(tt), _p(w), ctypes.byref(chi0))
    return tt, w, chi0.value


def phase(tt, f):
    return lib().ssp_oracle_phase(float(tt), float(f))


def fold_sort(tt, f):
    tt = _f64(tt)
    x = np.empty(tt.size)
    perm = np.empty(tt.size, dtype=np.int32)
    lib().ssp_oracle_fold_sort(tt.size, _p(tt), float(f), _p(x), _p(perm))
    return x, perm


def half_width(n, span):
    return lib().ssp_oracle_half_width(int(n), float(span))


def vsmlsq(x):
    x = _f64(x)
    return lib().ssp_oracle_vsmlsq(x.size, _p(x))


def runline_raw(x, v, w, span, iper, vsm):
    x, v, w = _f64(x), _f64(v), _f64(w)
    smo, acvr = np.empty(x.size), np.zeros(x.size)
    lib().ssp_oracle_runline_raw(x.size, _p(x), _p(v), _p(w), float(span), int(iper),
                                 float(vsm), _p(smo), _p(acvr))
    return smo, acvr


def runline(x, v, w, span, iper, vsm):
    x, v, w = _f64(x), _f64(v), _f64(w)
    smo, acvr = np.empty(x.size), np.zeros(x.size)
    lib().ssp_oracle_runline(x.size, _p(x), _p(v), _p(w), float(span), int(iper),
                             float(vsm), _p(smo), _p(acvr))
    return smo, acvr


def tie_average(x, w, smo):
    x, w = _f64(x), _f64(w)
    out = _f64(smo).copy()
    lib().ssp_oracle_tie_average(x.size, _p(x), _p(w), _p(out))
    return out


def supsmu(x, y, w, iper=2, span=0.0, alpha=9.0, spans=None):
    x, y, w = _f64(x), _f64(y), _f64(w)
    smo = np.empty(x.size)
    sp = _spans(spans)
    lib().ssp_oracle_supsmu(x.size, _p(x), _p(y), _p(w), int(iper), float(span),
                            float(alpha), _p(sp), _p(smo))
    return smo


def supsmu_spg(x, y, w, iper=2, spans=None):
    """Global generalized-validation reading of Sec. 3: (smooth, chosen span index)."""
    x, y, w = _f64(x), _f64(y), _f64(w)
    smo = np.empty(x.size)
    k = ctypes.c_int(-1)
    lib().ssp_oracle_supsmu_spg(x.size, _p(x), _p(y), _p(w), int(iper), _p(_spans(spans)), _p(smo),
                                ctypes.byref(k))
    return smo, k.value


def supsmu_sp(x, y, w, iper=2, alpha=9.0, spans=None):
    x, y, w = _f64(x), _f64(y), _f64(w)
    smo = np.empty(x.size)
    sp = _spans(spans)
    lib().ssp_oracle_supsmu_sp(x.size, _p(x), _p(y), _p(w), int(iper), float(alpha),
                               _p(sp), _p(smo))
    return smo


def chi2(y, w, smo):
    y, w, smo = _f64(y), _f64(w), _f64(smo)
    return lib().ssp_oracle_chi2(y.size, _p(y), _p(w), _p(smo))


def power_one(t, y, dy, f, variant=SS, alpha=9.0, spans=None, iper=2, span=0.0):
    """Power at one frequency.  iper 2 = periodic windows, 1 = clamped;
    span > 0 = Listing 1's fixed-span smooth (either variant)."""
    t, y, dy = _f64(t), _f64(y), _f64(dy)
    if not (t.size == y.size == dy.size):
        raise ValueError("t, y and dy must have the same length")
    sp = _spans(spans)
    return lib().ssp_oracle_power_one(t.size, _p(t), _p(y), _p(dy), float(f), int(variant),
                                      float(alpha), _p(sp), int(iper), float(span))


def periodogram(t, y, dy, n_per_object, freq, variant=SS, alpha=9.0, spans=None,
                n_threads=None, iper=2, span=0.0):
    """Whole periodogram: returns (power[n_objects, n_freq], best_period[n_objects])."""
    t, y, dy, freq = _f64(t), _f64(y), _f64(dy), _f64(freq)
    npo = np.ascontiguousarray(n_per_object, dtype=np.int64)
    if not (t.size == y.size == dy.size == int(npo.sum())):
        raise ValueError("t, y and dy must hold sum(n_per_object) points each")
    nobj, nf = npo.size, freq.size
    power = np.empty((nobj, nf))
    best = np.empty(nobj)
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    sp = _spans(spans)
    rc = lib().ssp_oracle_periodogram(_p(t), _p(y), _p(dy), _p(npo), nobj, _p(freq), nf,
                                      int(variant), float(alpha), _p(sp), int(iper), float(span),
                                      int(n_threads), _p(power), _p(best))
    if rc != 0:
        raise ValueError("oracle rejected the input (every object needs n >= 4)")
    return power, best


def peaks(p, k):
    """Indices of the top k local maxima of p (ties by lower index)."""
    p = _f64(p)
    out = np.empty(int(k), dtype=np.int64)
    lib().ssp_oracle_peaks(_p(p), p.size, int(k), _p(out))
    return out


def fine_grid(f, q, n_fine):
    f = _f64(f)
    out = np.empty(int(n_fine))
    lib().ssp_oracle_fine_grid(_p(f), f.size, int(q), int(n_fine), _p(out))
    return out


def search_refine(t, y, dy, n_per_object, coarse, coarse_variant=SP, fine_variant=SS,
                  n_peaks=3, n_fine=64, alpha=9.0, spans=None, iper=2, n_threads=None):
    """(best_period[n_objects], best_power[n_objects]) of search-and-refine."""
    t, y, dy, coarse = _f64(t), _f64(y), _f64(dy), _f64(coarse)
    npo = np.ascontiguousarray(n_per_object, dtype=np.int64)
    if not (t.size == y.size == dy.size == int(npo.sum())):
        raise ValueError("t, y and dy must hold sum(n_per_object) points each")
    bp, bw = np.empty(npo.size), np.empty(npo.size)
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    rc = lib().ssp_oracle_search_refine(_p(t), _p(y), _p(dy), _p(npo), npo.size, _p(coarse),
                                        coarse.size, int(coarse_variant), int(fine_variant),
                                        float(alpha), _p(_spans(spans)), int(iper), int(n_peaks),
                                        int(n_fine), int(n_threads), _p(bp), _p(bw))
    if rc != 0:
        raise ValueError("oracle rejected the input")
    return bp, bw
