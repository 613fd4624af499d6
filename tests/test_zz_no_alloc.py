"""The entry point that allocates no device memory.

Callers that cannot call cudaMalloc (device memory owned by another
allocator or capped by a pool, services that forbid allocation after
start-up) use ssp_periodogram_device_noalloc, whose scratch is a fixed array
the library declares in device memory.  Both entry points run the same
kernels with the same launch plan on these objects, so the results must be
bit for bit those of ssp_periodogram_device, call after call, although every
call reuses the same array.

Kept in a file of its own that pytest collects last, so a run that stops at
the first failure has already run every other test; it passes alone in a
fresh process too.
"""
import numpy as np
import pytest

from paper_2111_07396_gb300 import build as ssp_build
from paper_2111_07396_gb300 import ssp, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ssp_build.build()
    ssp.lib()


def _device(cat):
    import torch
    put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return put(cat.t), put(cat.y), put(cat.dy), put(cat.freq)


def _outputs(cat, precision):
    import torch
    dt = torch.float64 if precision == "fp64" else torch.float32
    return (torch.empty((cat.n_objects, cat.freq.size), dtype=dt, device="cuda"),
            torch.empty(cat.n_objects, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
@pytest.mark.parametrize("variant", ["ss", "sp"])
def test_no_alloc_matches_device_entry_on_consecutive_calls(variant, precision):
    import torch
    # two different requests back to back: the second must not see the
    # first one's counters, flags or offsets left in the shared array
    cats = [synth.config3(n_objects=24, n_freq=411), synth.config1(n_freq=257)]
    refs = []
    for cat in cats:
        t, y, dy, fq = _device(cat)
        pw, bp = _outputs(cat, precision)
        ssp.ssp_periodogram_device(t, y, dy, cat.n_per_object, fq, pw, bp, variant=variant,
                                   precision=precision)
        torch.cuda.synchronize()
        refs.append((pw.cpu().numpy(), bp.cpu().numpy()))
    for call in range(2):
        for cat, (ref_pw, ref_bp) in zip(cats, refs):
            t, y, dy, fq = _device(cat)
            pw, bp = _outputs(cat, precision)
            ssp.ssp_periodogram_device_noalloc(t, y, dy, cat.n_per_object, fq, pw, bp,
                                               variant=variant, precision=precision)
            torch.cuda.synchronize()
            got_pw, got_bp = pw.cpu().numpy(), bp.cpu().numpy()
            np.testing.assert_array_equal(got_pw, ref_pw, err_msg=f"call {call}, {cat.name}")
            np.testing.assert_array_equal(got_bp, ref_bp)


def test_no_alloc_rejects_objects_beyond_its_limit():
    import torch
    cat = synth.config4(n_objects=1, n_freq=64)   # 10,000+ points: frame too large
    t, y, dy, fq = _device(cat)
    pw, bp = _outputs(cat, "fp32c")
    with pytest.raises(ssp.SSPError) as ei:
        ssp.ssp_periodogram_device_noalloc(t, y, dy, cat.n_per_object, fq, pw, bp)
    assert ei.value.status == ssp.SSP_ERR_UNSUPPORTED
    assert "no-allocation" in str(ei.value)
    torch.cuda.synchronize()
