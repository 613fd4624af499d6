"""The C ABI library loads without a GPU, exports every function that
include/ssp.h declares, and rejects invalid arguments before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2111_07396_gb300 import build as ssp_build
from paper_2111_07396_gb300 import ssp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    ssp_build.build()


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(ssp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported():
    names = _declared_functions()
    assert {"ssp_periodogram", "ssp_periodogram_device", "ssp_default_params"} <= names
    lib = ctypes.CDLL(ssp.SO)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults_and_strings():
    p = ssp.ssp_default_params()
    assert list(p.spans) == [0.05, 0.2, 0.5]
    assert p.alpha == 9.0 and p.periodic == 1 and p.precision == ssp.SSP_FP32C
    assert p.hbm_fraction == 0.75
    assert ssp.ssp_status_string(ssp.SSP_ERR_ARG) == "invalid argument"
    assert ssp.ssp_version().startswith("ssp ")
    assert ctypes.sizeof(ssp.ssp_params) == 56


def _call(**kw):
    args = dict(t=np.arange(8.0), y=np.ones(8), dy=np.ones(8), n_per_object=[8],
                freq_grid=[0.3, 0.4])
    args.update(kw)
    return ssp.ssp_periodogram(**args)


@pytest.mark.parametrize("kw,status", [
    (dict(n_per_object=[3], t=np.arange(3.0), y=np.ones(3), dy=np.ones(3)), ssp.SSP_ERR_ARG),
    (dict(freq_grid=[0.3, -1.0]), ssp.SSP_ERR_ARG),
    (dict(freq_grid=[0.3, np.nan]), ssp.SSP_ERR_ARG),
    (dict(dy=np.r_[np.ones(7), 0.0]), ssp.SSP_ERR_ARG),
    (dict(y=np.r_[np.ones(7), np.inf]), ssp.SSP_ERR_ARG),
    (dict(t=np.r_[np.arange(7.0), np.nan]), ssp.SSP_ERR_ARG),
    (dict(alpha=11.0), ssp.SSP_ERR_ARG),
    (dict(spans=(0.2, 0.1, 0.5)), ssp.SSP_ERR_ARG),
    (dict(variant=7), ssp.SSP_ERR_ARG),
    (dict(dy=np.r_[np.ones(7), 1e-30]), ssp.SSP_ERR_UNSUPPORTED),
])
def test_invalid_arguments_rejected_before_cuda(kw, status):
    if kw.get("variant") == 7:
        p = ssp.ssp_default_params()
        rc = ssp.lib().ssp_periodogram(None, None, None, None, 1, None, 1, 7, ctypes.byref(p),
                                       None, None)
        assert rc == status
        return
    with pytest.raises(ssp.SSPError) as ei:
        _call(**kw)
    assert ei.value.status == status


def test_frequency_count_limit():
    # work items hold frequency bounds as int: 2^31 frequencies are refused
    # by the shape check, before any array is read
    p = ssp.ssp_default_params()
    npo = (ctypes.c_int64 * 1)(8)
    rc = ssp.lib().ssp_periodogram(None, None, None, npo, 1, None, 2 ** 31, ssp.SSP_SS,
                                   ctypes.byref(p), None, None)
    assert rc == ssp.SSP_ERR_ARG and "n_freq too large" in ssp.ssp_last_error()
    rc = ssp.lib().ssp_periodogram(None, None, None, npo, 1, None, 2 ** 31 - 1, ssp.SSP_SS,
                                   ctypes.byref(p), None, None)
    assert rc == ssp.SSP_ERR_ARG and "NULL array" in ssp.ssp_last_error()


def _status(params=None, n=8):
    # the call's status: past the argument checks a call reaches CUDA, which
    # fails without a GPU (SSP_ERR_CUDA) and runs with one (SSP_OK)
    t, y, dy = np.arange(float(n)), np.ones(n), np.ones(n)
    try:
        ssp.ssp_periodogram(t, y, dy, [n], [0.3, 0.4], params=params)
        return ssp.SSP_OK
    except ssp.SSPError as e:
        return e.status


@pytest.mark.parametrize("field,ok,bad", [
    ("alpha", [0.0, 10.0], [-1e-9, 10.000001]),
    ("hbm_fraction", [1.0, 1e-6], [0.0, 1.0000001]),
    ("span", [0.0, 1.0], [-1e-12, 1.0000001]),
    ("spans", [(0.05, 0.2, 1.0), (1e-6, 0.2, 0.5)],
     [(0.0, 0.2, 0.5), (0.2, 0.2, 0.5), (0.05, 0.5, 0.5), (0.05, 0.2, 1.0000001)]),
])
def test_parameter_limits(field, ok, bad):
    # each documented range: its ends accepted, just beyond them refused
    for values, accepted in ((ok, True), (bad, False)):
        for v in values:
            p = ssp.ssp_default_params()
            if field == "spans":
                for i in range(3):
                    p.spans[i] = v[i]
            else:
                setattr(p, field, v)
            status = _status(params=p)
            assert (status != ssp.SSP_ERR_ARG) == accepted, (field, v, status)


def test_object_size_limits():
    # 4 <= n <= 65,535 points per object
    assert _status(n=3) == ssp.SSP_ERR_ARG
    assert _status(n=4) != ssp.SSP_ERR_ARG
    assert _status(n=65535) != ssp.SSP_ERR_ARG
    assert _status(n=65536) == ssp.SSP_ERR_ARG


@pytest.mark.parametrize("field,value", [("periodic", 2), ("periodic", -1), ("span", -0.1),
                                         ("span", 1.5), ("span", float("nan"))])
def test_mode_fields_checked(field, value):
    p = ssp.ssp_default_params()
    assert p.periodic == 1 and p.span == 0.0
    setattr(p, field, value)
    with pytest.raises(ssp.SSPError) as ei:
        _call(params=p)
    assert ei.value.status == ssp.SSP_ERR_ARG


def test_binding_checks_buffers_before_the_call():
    # a buffer of the wrong element type, size or layout would be read or
    # written past its end: the binding refuses it before calling the library
    t, y, dy = np.arange(8.0), np.ones(8), np.ones(8)
    ok = dict(t=t, y=y, dy=dy, n_per_object=[8], freq_grid=[0.3, 0.4])
    bad_outputs = [
        dict(out_power=np.empty((1, 2), dtype=np.float64)),        # FP32C writes float32
        dict(out_power=np.empty((1, 3), dtype=np.float32)),        # wrong size
        dict(out_power=np.empty((1, 4), dtype=np.float32)[:, ::2]),  # not contiguous
        dict(out_best_period=np.empty(2)),
        dict(t=np.arange(7.0), y=np.ones(7), dy=np.ones(7)),       # fewer points than n_per_object
    ]
    ro = np.empty((1, 2), dtype=np.float32)
    ro.flags.writeable = False
    bad_outputs.append(dict(out_power=ro))
    for kw in bad_outputs:
        args = dict(ok)
        args.update(kw)
        with pytest.raises(ValueError):
            ssp.ssp_periodogram(**args)
    # FP64 writes float64
    with pytest.raises(ValueError):
        ssp.ssp_periodogram(**ok, precision="fp64", out_power=np.empty((1, 2), dtype=np.float32))
    # the other host entry points: points to match n_per_object
    with pytest.raises(ValueError):
        ssp.ssp_autotune(np.arange(7.0), np.ones(7), np.ones(7), [8], [0.3, 0.4])
    with pytest.raises(ValueError):
        ssp.ssp_search_refine(np.arange(7.0), np.ones(7), np.ones(7), [8], [0.3, 0.4])


def test_binding_checks_device_buffers_before_the_call():
    torch = pytest.importorskip("torch")
    t = torch.arange(8.0, dtype=torch.float64)
    fq = torch.tensor([0.3, 0.4], dtype=torch.float64)
    pw, bp = torch.empty((1, 2), dtype=torch.float32), torch.empty(1, dtype=torch.float64)
    cases = [
        dict(t=t.float()),                              # float32 times
        dict(t=t[:7]),                                  # too few points
        dict(freq_grid=fq.float()),
        dict(out_power=torch.empty((1, 2), dtype=torch.float64)),
        dict(out_best_period=torch.empty(2, dtype=torch.float64)),
    ]
    for kw in cases:
        args = dict(t=t, y=t, dy=t, n_per_object=[8], freq_grid=fq, out_power=pw,
                    out_best_period=bp)
        args.update(kw)
        for fn in (ssp.ssp_periodogram_device, ssp.ssp_periodogram_device_noalloc):
            with pytest.raises(ValueError, match="must be a contiguous"):
                fn(**args)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(ssp, "SO", str(tmp_path / "nope.so"))
    monkeypatch.setattr(ssp, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        ssp.lib()


def test_server_rejects_bad_grid_and_params_before_cuda():
    with pytest.raises(ssp.SSPError) as ei:
        ssp.Server([0.3, 0.0])
    assert ei.value.status == ssp.SSP_ERR_ARG
    with pytest.raises(ssp.SSPError) as ei:
        ssp.Server([0.3, 0.4], alpha=-1.0)
    assert ei.value.status == ssp.SSP_ERR_ARG
    assert ssp.ssp_status_string(ssp.SSP_ERR_BUSY) == "too many requests in flight"
    assert ssp.ssp_status_string(ssp.SSP_PENDING) == "pending"
    assert ctypes.sizeof(ssp.ssp_server_config) == 48
    # at most 16 batch slots: 17 is refused before any device work, 16 passes
    # the checks (and then needs a device)
    with pytest.raises(ssp.SSPError) as ei:
        ssp.Server([0.3, 0.4], slots=17)
    assert ei.value.status == ssp.SSP_ERR_ARG
    try:
        ssp.Server([0.3, 0.4], slots=16).close()
    except ssp.SSPError as e:
        assert e.status != ssp.SSP_ERR_ARG
    # calls on a NULL handle are argument errors, not crashes
    t = ctypes.c_int64()
    assert ssp.lib().ssp_server_next(None, 0, ctypes.byref(t)) == ssp.SSP_ERR_ARG
    assert ssp.lib().ssp_server_poll(None, 1, 0, None, None, None) == ssp.SSP_ERR_ARG
    assert ssp.lib().ssp_server_destroy(None) == ssp.SSP_ERR_ARG


def test_autotune_rejects_bad_arguments_before_cuda():
    t, y, dy = np.arange(8.0), np.ones(8), np.ones(8)
    for kw, status in ((dict(n_per_object=[3], t=t[:3], y=y[:3], dy=dy[:3]), ssp.SSP_ERR_ARG),
                       (dict(freq_grid=[0.3, 0.0]), ssp.SSP_ERR_ARG),
                       (dict(dy=np.r_[np.ones(7), -1.0]), ssp.SSP_ERR_ARG)):
        args = dict(t=t, y=y, dy=dy, n_per_object=[8], freq_grid=[0.3, 0.4])
        args.update(kw)
        with pytest.raises(ssp.SSPError) as ei:
            ssp.ssp_autotune(**args)
        assert ei.value.status == status
    ssp.ssp_autotune_clear()   # needs no device


def test_search_refine_rejects_bad_arguments_before_cuda():
    t, y, dy = np.arange(8.0), np.ones(8), np.ones(8)
    base = dict(t=t, y=y, dy=dy, n_per_object=[8], coarse_grid=[0.3, 0.4, 0.5])
    for kw in (dict(coarse_grid=[0.3]), dict(coarse_grid=[0.3, 0.2]), dict(n_peaks=0),
               dict(n_peaks=65), dict(n_fine=0), dict(coarse_grid=[0.0, 0.4])):
        args = dict(base)
        args.update(kw)
        with pytest.raises(ssp.SSPError) as ei:
            ssp.ssp_search_refine(**args)
        assert ei.value.status == ssp.SSP_ERR_ARG


def test_search_refine_limits():
    # n_peaks in 1..64, n_peaks * n_fine <= 2^22, at least 2 coarse
    # frequencies: the ends accepted, just beyond them refused
    t, y, dy = np.arange(8.0), np.ones(8), np.ones(8)
    base = dict(t=t, y=y, dy=dy, n_per_object=[8], coarse_grid=[0.3, 0.4])

    def status(**kw):
        args = dict(base)
        args.update(kw)
        try:
            ssp.ssp_search_refine(**args)
            return ssp.SSP_OK
        except ssp.SSPError as e:
            return e.status

    for kw in (dict(n_peaks=1, n_fine=1), dict(n_peaks=64, n_fine=1), dict(n_peaks=64, n_fine=1 << 16)):
        assert status(**kw) != ssp.SSP_ERR_ARG, kw
    for kw in (dict(n_peaks=64, n_fine=(1 << 16) + 1), dict(coarse_grid=[0.3], n_peaks=1, n_fine=1)):
        assert status(**kw) == ssp.SSP_ERR_ARG, kw


def test_fault_injection_is_off_unless_testing(monkeypatch):
    # the failure hooks are test-only: without SSP_TESTING=1 they refuse
    monkeypatch.delenv("SSP_TESTING", raising=False)
    with pytest.raises(ssp.SSPError) as ei:
        ssp.ssp_test_fault(ssp.SSP_FAULT_ALLOC, 1)
    assert ei.value.status == ssp.SSP_ERR_UNSUPPORTED
    monkeypatch.setenv("SSP_TESTING", "1")
    with pytest.raises(ssp.SSPError) as ei:
        ssp.ssp_test_fault(99, 1)
    assert ei.value.status == ssp.SSP_ERR_ARG
    with pytest.raises(ssp.SSPError) as ei:
        ssp.ssp_test_fault(ssp.SSP_FAULT_STALL, -1)
    assert ei.value.status == ssp.SSP_ERR_ARG
    # arm and clear without touching a GPU
    ssp.ssp_test_fault(ssp.SSP_FAULT_ALLOC, 2)
    ssp.ssp_test_fault(ssp.SSP_FAULT_ALLOC, 0)
    ssp.ssp_test_fault(ssp.SSP_FAULT_STALL, 0)
    ssp.ssp_test_fault(ssp.SSP_FAULT_UPLOAD, 1)
    ssp.ssp_test_fault(ssp.SSP_FAULT_UPLOAD, 0)
