"""ssp_autotune: picks a threads-per-CTA choice per length range from timed
candidates; results after tuning stay within tolerance, and clearing the
table restores the fixed rule bit for bit."""
import numpy as np
import pytest

from oracle import oracle
from paper_2111_07396_gb300 import build as ssp_build
from paper_2111_07396_gb300 import ssp, synth
from tests.parity import TOL, gate_error, oracle_powers, sample_freqs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ssp_build.build()
    ssp.lib()
    yield
    ssp.ssp_autotune_clear()


@pytest.mark.parametrize("variant,code", [("ss", oracle.SS), ("sp", oracle.SP)])
def test_autotune_choices_and_results(variant, code):
    cat = synth.config3(n_objects=200, n_freq=400, n_hi=2400)
    args = (cat.t, cat.y, cat.dy, cat.n_per_object, cat.freq)
    ssp.ssp_autotune_clear()
    before, _ = ssp.ssp_periodogram(*args, variant=variant)
    g = ssp.ssp_autotune(*args, variant=variant, budget_ptf=2e8)
    assert g.shape == (5,)
    assert all(v in (32, 64, 128, 256, 512) for v in g)
    tuned, tuned_best = ssp.ssp_periodogram(*args, variant=variant)
    ref64, _ = ssp.ssp_periodogram(*args, variant=variant, precision="fp64")
    assert gate_error(tuned, ref64) <= TOL["fp32c"]
    # oracle at sampled frequencies for a few objects
    for o in (0, 57, 199):
        t, y, dy = cat.obj(o)
        qs = sample_freqs(cat.freq.size, 6, seed=o)
        ref = oracle_powers(t, y, dy, cat.freq[qs], code)
        assert gate_error(tuned[o, qs], ref) <= TOL["fp32c"]
    ssp.ssp_autotune_clear()
    again, _ = ssp.ssp_periodogram(*args, variant=variant)
    np.testing.assert_array_equal(again, before)
