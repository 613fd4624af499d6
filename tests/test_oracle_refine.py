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


@pytest.mark.parametrize("seed", range(8))
def test_peak_rule_on_broad_peaks(seed):
    # smooth periodograms: a few broad peaks with long slopes, so a point on
    # a slope that is not a local maximum would outrank the lesser peaks if
    # the rule admitted it; k up to the number of points (the fill rule)
    g = np.random.default_rng(100 + seed)
    n = int(g.integers(8, 60))
    q = np.arange(n)
    p = np.zeros(n)
    for _ in range(int(g.integers(1, 4))):
        p += g.uniform(0.2, 1.0) * np.exp(-0.5 * ((q - g.uniform(0, n)) / g.uniform(1.5, 6.0)) ** 2)
    p = np.round(p, 3)
    for k in (1, 2, 4, n):
        assert list(oracle.peaks(p, k)) == _brute_peaks(p, k)


def test_peak_rule_hand_cases():
    # one broad peak: the rest repeat it; plateaus count at their left end
    assert list(oracle.peaks(np.array([0.1, 0.5, 0.9, 0.7, 0.3]), 3)) == [2, 2, 2]
    assert list(oracle.peaks(np.array([0.2, 0.6, 0.6, 0.1]), 2)) == [2, 2]
    assert list(oracle.peaks(np.array([0.9, 0.1, 0.1, 0.8]), 2)) == [0, 3]
    assert list(oracle.peaks(np.array([0.3, 0.2, 0.1]), 2)) == [0, 0]
    assert list(oracle.peaks(np.array([0.1, 0.2, 0.3]), 2)) == [2, 2]
    # a peak next to one already taken is skipped
    assert list(oracle.peaks(np.array([0.1, 0.9, 0.2, 0.8, 0.1, 0.5, 0.1]), 3)) == [1, 3, 5]


def test_fine_grid_spans_the_neighbours():
    f = np.array([0.5, 0.8, 1.1, 1.4])
    np.testing.assert_allclose(oracle.fine_grid(f, 1, 7), np.linspace(0.5, 1.1, 7))
    np.testing.assert_allclose(oracle.fine_grid(f, 0, 3), [0.2, 0.5, 0.8])    # one 0.3 step back
    np.testing.assert_allclose(oracle.fine_grid(np.array([0.1, 0.5]), 0, 3), [0.05, 0.275, 0.5])
    np.testing.assert_allclose(oracle.fine_grid(f, 3, 3), [1.1, 1.4, 1.7])
    # a start exactly at 0 also moves to f[q] / 2
    np.testing.assert_allclose(oracle.fine_grid(np.array([0.5, 1.0, 1.5]), 0, 3), [0.25, 0.625, 1.0])
    # one fine frequency is the peak's own; a one-frequency grid has no step
    np.testing.assert_array_equal(oracle.fine_grid(f, 2, 1), [1.1])
    np.testing.assert_array_equal(oracle.fine_grid(np.array([0.7]), 0, 3), [0.7, 0.7, 0.7])


def test_search_refine_smallest_arguments():
    # two coarse frequencies, one peak, one fine frequency: the refine step
    # evaluates the coarse peak itself, so it returns the coarse best
    cat = synth.config1(n_freq=2)
    for o in range(1):
        t, y, dy = cat.obj(o)
        bp, bw = oracle.search_refine(t, y, dy, [t.size], cat.freq, coarse_variant=oracle.SS,
                                      fine_variant=oracle.SS, n_peaks=1, n_fine=1)
        pw, best = oracle.periodogram(t, y, dy, [t.size], cat.freq, oracle.SS)
        assert bp[0] == best[0] and bw[0] == pw[0].max()


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
