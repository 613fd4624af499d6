"""Shared helpers of the GPU parity tests (no arithmetic of the method)."""
import numpy as np

TOL = {"fp64": 1e-9, "fp32c": 2e-4}
FLOOR = 1e-2  # powers below this are compared on an absolute scale


def gate_error(got, ref):
    """Largest |got - ref| / max(|ref|, 1e-2): relative error on every power
    value, absolute (scaled by 1e-2) where the reference power is near 0."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape
    assert np.all(np.isfinite(got)), "non-finite power"
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), FLOOR)))


def chi2_rel_error(got, ref):
    """Relative error of chi2 = chi0 (1 - power), well conditioned at any power."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(1.0 - ref), 1e-12)))


def sample_freqs(n_freq, k, seed, include=()):
    g = np.random.default_rng(seed)
    idx = set(int(i) for i in g.choice(n_freq, size=min(k, n_freq), replace=False))
    idx |= {0, n_freq - 1}
    idx |= {int(i) for i in include if 0 <= i < n_freq}
    return np.array(sorted(idx))


def oracle_powers(t, y, dy, freqs, code, threads=None):
    """Oracle power at each frequency, one C call per frequency, in parallel
    threads (the C oracle releases the GIL)."""
    import concurrent.futures as cf
    import os

    import oracle
    threads = threads or os.cpu_count() or 1
    with cf.ThreadPoolExecutor(threads) as ex:
        return np.array(list(ex.map(lambda f: oracle.power_one(t, y, dy, f, code), freqs)))
