"""Pins of the oracle's search-and-refine (Sec. 6 outlook): the peak rule
against a brute-force restatement, the fine grids, consistency with a direct
periodogram on the same grids, and a sharper period than the coarse grid
alone gives."""
import numpy as np
import pytest

import oracle
from paper_2111_07396_gb300 import synth


def _brute_peaks(p, k):
    n = p.size
    cands = [q for q in range(n)
             if (q == 0 or p[q] >= p[q - 1]) and (q == n - 1 or p[q] > p[q + 1])]
    taken = []
    for q in sorted(cands, key=lambda q: (-p[q], q)):
        if len(taken) == k:
            break
        if any(abs(q - t) <= 1 for t in taken):
            continue
        taken.append(q)
    while len(taken) < k:
        taken.append(taken[0] if taken else 0)
    return taken


@pytest.mark.parametrize("seed", range(12))
def test_peak_rule(seed):
    g = np.random.default_rng(seed)
    n = int(g.integers(2, 40))
    p = np.round(g.uniform(0, 1, n), 1)      # coarse values: plateaus and ties
    for k in (1, 3, 5):
        assert list(oracle.peaks(p, k)) == _brute_peaks(p, k)


def test_fine_grid_spans_the_neighbours():
    f = np.array([0.5, 0.8, 1.1, 1.4])
    np.testing.assert_allclose(oracle.fine_grid(f, 1, 7), np.linspace(0.5, 1.1, 7))
    np.testing.assert_allclose(oracle.fine_grid(f, 0, 3), [0.2, 0.5, 0.8])    # one 0.3 step back
    np.testing.assert_allclose(oracle.fine_grid(np.array([0.1, 0.5]), 0, 3), [0.05, 0.275, 0.5])
    np.testing.assert_allclose(oracle.fine_grid(f, 3, 3), [1.1, 1.4, 1.7])


def test_refine_is_the_periodogram_on_the_fine_grids():
    cat = synth.config3(n_objects=5, n_freq=300)
    for variant in (oracle.SS, oracle.SP):
        bp, bw = oracle.search_refine(cat.t, cat.y, cat.dy, cat.n_per_object, cat.freq,
                                      coarse_variant=oracle.SPG, fine_variant=variant,
                                      n_peaks=3, n_fine=9)
        cp, _ = oracle.periodogram(cat.t, cat.y, cat.dy, cat.n_per_object, cat.freq, oracle.SPG)
        for o in range(5):
            t, y, dy = cat.obj(o)
            grid = np.concatenate([oracle.fine_grid(cat.freq, q, 9)
                                   for q in oracle.peaks(cp[o], 3)])
            pw, best = oracle.periodogram(t, y, dy, [t.size], grid, variant)
            assert bp[o] == best[0] and bw[o] == pw[0].max()


def test_refine_sharpens_the_period():
    # a 30-day light curve: its peaks are ~1/30 wide, which a 0.01-step
    # coarse grid resolves but does not pin down
    g = np.random.default_rng(3)
    t = np.sort(g.uniform(0, 30, 150))
    y = 15 + 0.3 * np.sin(2 * np.pi * t / 0.37) + g.normal(0, 0.05, t.size)
    dy = np.full(t.size, 0.05)
    coarse = 0.5 + 0.01 * np.arange(400)
    f_true = 1.0 / 0.37
    cp, cb = oracle.periodogram(t, y, dy, [t.size], coarse, oracle.SS)
    bp, bw = oracle.search_refine(t, y, dy, [t.size], coarse, coarse_variant=oracle.SS,
                                  fine_variant=oracle.SS, n_peaks=2, n_fine=201)
    assert abs(1.0 / cb[0] - f_true) < 0.01
    assert abs(1.0 / bp[0] - f_true) < 0.002
    assert bw[0] >= cp[0].max()
