"""The FP32C kernels fold phases with integer arithmetic; ssp_fold_fixed runs
the same code on the host.  It must give the binary64 phase of Alg. 1,
frac(fl(tt*f)), bit for bit (as a 64-bit fixed-point fraction)."""
import numpy as np
import pytest

from paper_2111_07396_gb300 import build as ssp_build
from paper_2111_07396_gb300 import ssp


@pytest.fixture(scope="module", autouse=True)
def built():
    ssp_build.build()


def _expected(tt, f):
    p = tt * f                    # IEEE binary64 product, round to nearest even
    ph = p - np.floor(p)          # exact
    return np.array([int(v * 2.0 ** 64) for v in ph], dtype=object)


@pytest.mark.parametrize("seed", range(6))
def test_fold_matches_binary64_phase(seed):
    g = np.random.default_rng(seed)
    tt = np.concatenate([g.uniform(0, 3000, 4000), g.uniform(0, 1, 500),
                         10.0 ** g.uniform(-8, 6, 1500), [0.0, 1.0, 2.0, 4096.0, 1e-300]])
    for f in np.concatenate([g.uniform(0.01, 24, 6), 10.0 ** g.uniform(-6, 3, 4),
                             [1.0, 0.5, 2.0 ** -20, 3.0]]):
        got = ssp.ssp_fold_fixed(tt, f)
        exp = _expected(tt, f)
        big = tt * f >= 2.0 ** -11
        # phases >= 2^-11 are exact; tiny ones truncate the same way
        mism = [i for i in range(tt.size) if int(got[i]) != exp[i]]
        assert not mism, (f, [(tt[i], int(got[i]), exp[i]) for i in mism[:5]])
        assert big.sum() > 0


def test_fold_at_extreme_magnitudes():
    # products from just above 2^-11 to near the top of binary64: at and
    # beyond 2^53 the rounded product is an integer and the phase is 0
    g = np.random.default_rng(17)
    tt = np.concatenate([[1e15, 3.3e15, 2.0 ** 52 + 1, 2.0 ** 53, 2.0 ** 53 + 2, 1e16, 1e20, 1e300],
                         10.0 ** g.uniform(8, 300, 400)])
    for f in (1e-3, 0.37, 1.0, 3.3, 1e3):
        keep = np.isfinite(tt * f)
        got = ssp.ssp_fold_fixed(tt[keep], f)
        assert [int(v) for v in got] == list(_expected(tt[keep], f)), f


def test_fold_rounding_halfway_cases():
    # products that sit exactly halfway between two binary64 values
    tt = np.array([1.0 + 2.0 ** -52, 3.0 + 2.0 ** -51, 2.0 ** 40 + 1.0])
    for f in (1.0 + 2.0 ** -52, 1.5, 1.0 + 3 * 2.0 ** -52, 0.7):
        got = ssp.ssp_fold_fixed(tt, f)
        exp = _expected(tt, f)
        assert [int(v) for v in got] == list(exp)


def test_fold_rejects_bad_input():
    with pytest.raises(ssp.SSPError):
        ssp.ssp_fold_fixed([-1.0], 0.5)
    with pytest.raises(ssp.SSPError):
        ssp.ssp_fold_fixed([1.0], 0.0)
