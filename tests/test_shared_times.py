"""Objects with identical times share each frequency's fold and sort: the
shared path must give every object exactly what it gets alone."""
import numpy as np
import pytest

import oracle
from paper_2111_07396_gb300 import build as ssp_build
from paper_2111_07396_gb300 import ssp, synth
from tests.parity import TOL, gate_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ssp_build.build()
    ssp.lib()


def _catalog(bad=False):
    g = np.random.default_rng(23)
    cadences = [np.sort(g.uniform(0, 200, n)) for n in (150, 700, 2600)]
    cadences[1][100:103] = cadences[1][100]          # a tie run in one cadence
    objs = []
    for k in range(14):
        t = cadences[k % 3] if k < 12 else np.sort(g.uniform(0, 200, 90))   # two singletons
        P = g.uniform(0.3, 20)
        y = 15 + 0.2 * np.sin(2 * np.pi * t / P) + g.normal(0, 0.05, t.size)
        dy = g.uniform(0.03, 0.08, t.size)
        if bad and k == 4:
            y = y.copy()
            y[7] = np.nan
        objs.append((t, y, dy))
    freq = synth.uniform_grid(0.05, 6.0, 157)
    return synth.concat([synth.single_object(*o, freq) for o in objs])


@pytest.mark.parametrize("variant", ["ss", "sp", "spg"])
@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_shared_sort_equals_separate_objects(variant, precision):
    cat = _catalog()
    got, best = ssp.ssp_periodogram(cat.t, cat.y, cat.dy, cat.n_per_object, cat.freq,
                                    variant=variant, precision=precision)
    for o in range(cat.n_objects):
        t, y, dy = cat.obj(o)
        alone, ab = ssp.ssp_periodogram(t, y, dy, [t.size], cat.freq, variant=variant,
                                        precision=precision)
        np.testing.assert_array_equal(got[o], alone[0])
        assert best[o] == ab[0]


@pytest.mark.parametrize("variant,code", [("ss", oracle.SS), ("sp", oracle.SP)])
def test_shared_sort_parity(variant, code):
    cat = _catalog()
    ref, _ = oracle.periodogram(cat.t, cat.y, cat.dy, cat.n_per_object, cat.freq, code)
    got, _ = ssp.ssp_periodogram(cat.t, cat.y, cat.dy, cat.n_per_object, cat.freq,
                                 variant=variant, precision="fp64")
    assert gate_error(got, ref) <= TOL["fp64"]


def test_invalid_member_of_a_group():
    cat = _catalog(bad=True)
    import torch
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    pw = torch.empty((cat.n_objects, cat.freq.size), dtype=torch.float32, device="cuda")
    bp = torch.empty(cat.n_objects, dtype=torch.float64, device="cuda")
    # the host entry point rejects NaN inputs; the device one marks the object
    ssp.ssp_periodogram_device(dev(cat.t), dev(cat.y), dev(cat.dy), cat.n_per_object,
                               dev(cat.freq), pw, bp)
    torch.cuda.synchronize()
    p = pw.cpu().numpy()
    assert np.all(np.isnan(p[4])) and np.all(np.isfinite(np.delete(p, 4, axis=0)))
