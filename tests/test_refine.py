"""ssp_search_refine on the GPU against the oracle's search-and-refine."""
import numpy as np
import pytest

import oracle
from paper_2111_07396_gb300 import build as ssp_build
from paper_2111_07396_gb300 import ssp, synth
from tests.parity import TOL

pytestmark = pytest.mark.gpu

CODES = {"ss": oracle.SS, "sp": oracle.SP, "spg": oracle.SPG}


@pytest.fixture(scope="module", autouse=True)
def built():
    ssp_build.build()
    ssp.lib()


def _catalog():
    # short light curves (peaks ~1/40 wide) on a 0.01-step coarse grid
    g = np.random.default_rng(17)
    objs = []
    for k, P in enumerate((0.37, 1.9, 0.61, 5.3)):
        n = (60, 140, 300, 90)[k]
        t = np.sort(g.uniform(0, 40, n))
        y = 15 + 0.3 * np.sin(2 * np.pi * t / P) + g.normal(0, 0.05, n)
        objs.append((t, y, np.full(n, 0.05)))
    coarse = 0.1 + 0.01 * np.arange(500)
    return synth.concat([synth.single_object(*o, coarse) for o in objs]), coarse


@pytest.mark.parametrize("coarse_v,fine_v", [("spg", "ss"), ("sp", "sp"), ("ss", "spg")])
def test_search_refine_matches_oracle(coarse_v, fine_v):
    cat, coarse = _catalog()
    ref_p, ref_w = oracle.search_refine(cat.t, cat.y, cat.dy, cat.n_per_object, coarse,
                                        coarse_variant=CODES[coarse_v],
                                        fine_variant=CODES[fine_v], n_peaks=3, n_fine=33)
    for precision in ("fp64", "fp32c"):
        bp, bw = ssp.ssp_search_refine(cat.t, cat.y, cat.dy, cat.n_per_object, coarse,
                                       coarse_variant=coarse_v, fine_variant=fine_v, n_peaks=3,
                                       n_fine=33, precision=precision)
        np.testing.assert_array_equal(bp, ref_p)
        err = np.abs(bw - ref_w) / np.maximum(np.abs(ref_w), 1e-2)
        assert err.max() <= TOL[precision], precision
