"""Launch plans (ssp_plan_*): the device pipeline captured once into a CUDA
graph and replayed on new arrays of the same shape.  Each execution must give
ssp_periodogram_device's results bit for bit, execution after execution."""
import numpy as np
import pytest

from paper_2111_07396_gb300 import build as ssp_build
from paper_2111_07396_gb300 import ssp, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ssp_build.build()
    ssp.lib()


def _dev(cat):
    import torch
    put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return put(cat.t), put(cat.y), put(cat.dy), put(cat.freq)


def _outs(cat, precision):
    import torch
    dt = torch.float64 if precision == "fp64" else torch.float32
    return (torch.empty((cat.n_objects, cat.freq.size), dtype=dt, device="cuda"),
            torch.empty(cat.n_objects, dtype=torch.float64, device="cuda"))


def _same_shape_catalogs():
    # two catalogs with the same point counts and grid size, different values
    a = synth.config3(n_objects=20, n_freq=301)
    b = synth.config3(n_objects=20, n_freq=301)
    g = np.random.default_rng(4)
    b.t = b.t + g.uniform(0, 3.0, b.t.size)
    b.y = b.y[::-1].copy()
    b.freq = b.freq * 1.01
    return a, b


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("variant", ["ss", "sp"])
def test_plan_executions_equal_device_entry(variant, precision):
    import torch
    cats = _same_shape_catalogs()
    with ssp.Plan(cats[0].n_per_object, cats[0].freq.size, variant=variant,
                  precision=precision) as plan:
        for rep in range(2):
            for cat in cats:
                t, y, dy, fq = _dev(cat)
                pw, bp = _outs(cat, precision)
                ref_pw, ref_bp = _outs(cat, precision)
                ssp.ssp_periodogram_device(t, y, dy, cat.n_per_object, fq, ref_pw, ref_bp,
                                           variant=variant, precision=precision)
                plan.execute(t, y, dy, fq, pw, bp)
                torch.cuda.synchronize()
                np.testing.assert_array_equal(pw.cpu().numpy(), ref_pw.cpu().numpy(),
                                              err_msg=f"execution {rep}")
                np.testing.assert_array_equal(bp.cpu().numpy(), ref_bp.cpu().numpy())


def test_plan_long_object_with_binary64_recompute():
    # 3,000 points: the long-object SS kernel, whose flagged frequencies are
    # recomputed in binary64 inside it (its own slab, in the plan's workspace)
    import torch
    cat = synth.config2(n_freq=4000)
    t, y, dy, fq = _dev(cat)
    pw, bp = _outs(cat, "fp32c")
    ref_pw, ref_bp = _outs(cat, "fp32c")
    ssp.ssp_periodogram_device(t, y, dy, cat.n_per_object, fq, ref_pw, ref_bp, variant="ss")
    with ssp.Plan(cat.n_per_object, cat.freq.size, variant="ss") as plan:
        plan.execute(t, y, dy, fq, pw, bp)
        plan.execute(t, y, dy, fq, pw, bp)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(pw.cpu().numpy(), ref_pw.cpu().numpy())
    np.testing.assert_array_equal(bp.cpu().numpy(), ref_bp.cpu().numpy())


def test_plan_rejects_bad_arguments():
    with pytest.raises(ssp.SSPError) as ei:
        ssp.Plan([3], 10)                 # fewer than 4 points
    assert ei.value.status == ssp.SSP_ERR_ARG
    with pytest.raises(ssp.SSPError) as ei:
        ssp.Plan([10], 0)
    assert ei.value.status == ssp.SSP_ERR_ARG
