"""Pins of the oracle's running-line smoother (the `smoothkernel` that Listing 1
calls; Friedman 1984) against facts that do not come from the oracle itself:
explicit weighted least squares, explicit leave-one-out refits, exact
reproduction of constant and linear data, and hand-computed window sizes."""
import numpy as np
import pytest

import oracle
from tests import brute


def _data(n, seed, distinct=True):
    g = np.random.default_rng(seed)
    x = np.sort(g.uniform(0.0, 1.0, n))
    if distinct:
        assert np.all(np.diff(x) > 0)
    v = g.normal(0.0, 1.0, n)
    w = g.uniform(0.5, 4.0, n)
    return x, v, w


@pytest.mark.parametrize("n,span,expect", [
    (100, 0.05, 3), (100, 0.2, 10), (100, 0.5, 25), (3000, 0.05, 75), (3000, 0.2, 300),
    (3000, 0.5, 750), (10, 0.05, 2), (4, 0.5, 1), (5, 0.05, 2), (30, 0.05, 2), (41, 0.2, 4),
    # fixed spans above 0.5 reach the cap: 2h + 1 <= n
    (7, 1.0, 3), (21, 1.0, 10), (8, 1.0, 3), (9, 0.9, 4),
])
def test_half_width_table(n, span, expect):
    # floor(0.5*span*n + 0.5), at least 2, at most (n-1)/2
    assert oracle.half_width(n, span) == expect


@pytest.mark.parametrize("iper", [1, 2, -1, -2])
@pytest.mark.parametrize("span", [0.05, 0.3, 0.5])
@pytest.mark.parametrize("n", [5, 7, 12])
def test_runline_matches_weighted_least_squares(n, span, iper):
    x, v, w = _data(n, 1000 * n + int(100 * span) + iper)
    smo, _ = oracle.runline_raw(x, v, w, span, iper, 0.0)
    ref, _ = brute.runline(x, v, w, span, iper, 0.0, tie_average=False)
    np.testing.assert_allclose(smo, ref, rtol=1e-12, atol=1e-12)


def test_runline_constant_slope_dropped_below_vsmlsq():
    x, v, w = _data(9, 5)
    smo, _ = oracle.runline_raw(x, v, w, 0.5, 2, 1e9)  # threshold above any spread
    ref, _ = brute.runline(x, v, w, 0.5, 2, 1e9, tie_average=False)
    np.testing.assert_allclose(smo, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("iper", [1, 2])
def test_runline_reproduces_constant(iper):
    x, _, w = _data(40, 11)
    v = np.full(40, 3.25)
    smo, acvr = oracle.runline(x, v, w, 0.2, iper, 0.0)
    np.testing.assert_allclose(smo, v, rtol=0, atol=1e-13)
    np.testing.assert_allclose(acvr, 0.0, atol=1e-12)


def test_runline_reproduces_linear_nonperiodic():
    x, _, w = _data(50, 12)
    v = -2.0 + 7.5 * x
    for span in (0.05, 0.2, 0.5):
        smo, acvr = oracle.runline(x, v, w, span, 1, 0.0)
        np.testing.assert_allclose(smo, v, rtol=0, atol=1e-12)
        np.testing.assert_allclose(acvr, 0.0, atol=1e-11)


def test_runline_reproduces_linear_periodic_interior():
    n = 60
    x, _, w = _data(n, 13)
    v = 1.0 + 4.0 * x
    span = 0.2
    ibw = brute.half_width(n, span)
    smo, _ = oracle.runline(x, v, w, span, 2, 0.0)
    interior = np.arange(ibw, n - ibw)  # windows that do not wrap
    np.testing.assert_allclose(smo[interior], v[interior], rtol=0, atol=1e-12)
    # wrapped windows see x-1 / x+1 for the far points and cannot be linear
    assert np.max(np.abs(smo[:ibw] - v[:ibw])) > 1e-3


@pytest.mark.parametrize("iper", [1, 2])
@pytest.mark.parametrize("n", [6, 9, 14])
def test_cv_residual_is_leave_one_out(n, iper):
    x, v, w = _data(n, 77 * n + iper)
    for span in (0.05, 0.2, 0.5):
        _, acvr = oracle.runline_raw(x, v, w, span, iper, 0.0)
        _, ref = brute.runline(x, v, w, span, iper, 0.0, tie_average=False)
        np.testing.assert_allclose(acvr, ref, rtol=1e-9, atol=1e-11)


def test_cv_fallback_when_leverage_reaches_one():
    n = 9
    x, v, w = _data(n, 21)
    w = np.ones(n)
    w[0] = 1e20   # w_0 / W rounds to 1: the residual of point 0 falls back to 0
    w[4] = 1e20   # and point 4 copies point 3's residual
    _, acvr = oracle.runline_raw(x, v, w, 0.2, 2, 0.0)
    assert acvr[0] == 0.0
    assert acvr[4] == acvr[3]
    assert acvr[3] > 0.0


def test_tie_average_equals_weighted_mean_of_fits():
    g = np.random.default_rng(3)
    x = np.sort(np.concatenate([g.uniform(0, 1, 12), [0.25, 0.25, 0.7]]))
    x = np.sort(np.concatenate([x, [0.25]]))  # a run of 3+ equal abscissae
    v = g.normal(0, 1, x.size)
    w = g.uniform(0.5, 2, x.size)
    smo, _ = oracle.runline(x, v, w, 0.3, 2, 0.0)
    raw, _ = brute.runline(x, v, w, 0.3, 2, 0.0, tie_average=False)
    ref = brute.tie_avg(x, w, raw)
    np.testing.assert_allclose(smo, ref, rtol=1e-12, atol=1e-12)
    run = np.flatnonzero(x == 0.25)
    assert run.size >= 3 and np.ptp(smo[run]) == 0.0


@pytest.mark.parametrize("iper", [1, 2])
def test_window_of_equal_abscissae_has_no_slope(iper):
    # Seven of ten abscissae equal and vsmlsq = 0 (the middle half of the
    # points tie, so Listing 1's scale is 0).  A window holding only the
    # tied points has spread 0, which is not above vsmlsq: its line is the
    # weighted mean, and the cross-validated residual is the distance to the
    # weighted mean of the window's other points, with no leverage-1
    # fallback (the residuals are per point, before tie averaging).  Centres 3, 4 and 5 have such windows at half width 2.
    x = np.r_[0.05, np.full(7, 0.3), 0.6, 0.7]   # scale = x[5] - x[1] = 0
    g = np.random.default_rng(31)
    v = g.normal(0, 1, 10)
    w = g.uniform(0.5, 2, 10)
    assert oracle.vsmlsq(x) == 0.0
    _, cv = oracle.runline(x, v, w, 0.05, iper, 0.0)
    for j in (3, 4, 5):
        win = np.arange(j - 2, j + 3)
        assert np.all(x[win] == 0.3)
        others = win[win != j]
        loo = np.sum(w[others] * v[others]) / np.sum(w[others])
        np.testing.assert_allclose(cv[j], abs(v[j] - loo), rtol=1e-12)


@pytest.mark.parametrize("run", [2, 3])
def test_tie_average_of_a_run_at_the_end(run):
    # a run of equal abscissae that ends at the last point is averaged too
    g = np.random.default_rng(4 + run)
    x = np.sort(np.concatenate([g.uniform(0, 0.8, 9), np.full(run, 0.9)]))
    v = g.normal(0, 1, x.size)
    w = g.uniform(0.5, 2, x.size)
    smo = oracle.tie_average(x, w, v)
    np.testing.assert_allclose(smo, brute.tie_avg(x, w, v), rtol=1e-14, atol=1e-15)
    tail = smo[-run:]
    assert np.ptp(tail) == 0.0
    np.testing.assert_allclose(tail[0], np.sum(w[-run:] * v[-run:]) / np.sum(w[-run:]), rtol=1e-14)


def test_cv_fallback_for_exact_leverage_one_at_a_clamped_end():
    # Non-periodic windows at the last point: its 5-point window holds four
    # tied abscissae and the point itself, whose leverage is exactly 1 in
    # exact arithmetic (w_j h_j = 1).  Rounding leaves 1 - w h at +-1e-16;
    # the residual must fall back to the previous one, not divide by noise.
    n = 12
    g = np.random.default_rng(5)
    x = np.sort(g.uniform(0.0, 0.8, n))
    x[n - 5:n - 1] = 0.85
    x[n - 1] = 0.97
    v = g.normal(0, 1, n)
    w = g.uniform(0.5, 2.0, n)
    assert brute.half_width(n, 0.05) == 2
    _, acvr = oracle.runline_raw(x, v, w, 0.05, 1, 0.0)
    assert acvr[n - 1] == acvr[n - 2]
    assert np.all(np.isfinite(acvr)) and np.max(acvr) < 1e3
    # the same window by brute force: the fit through the other four points
    # (all at one abscissa) cannot reach x_{n-1}, so no leave-one-out value
    # exists there, while every other residual is the leave-one-out one
    _, ref = brute.runline(x, v, w, 0.05, 1, 0.0, tie_average=False)
    np.testing.assert_allclose(acvr[:n - 1], ref[:n - 1], rtol=1e-9, atol=1e-11)


def test_cv_fallback_is_decided_exactly_not_by_rounding():
    # Periodic windows of 5 points.  A point 8e10 times heavier than its four
    # neighbours has leverage 1 - w h of about 5e-11: no absolute cut-off
    # near 0 may send it to the fallback, its cross-validated residual is the
    # leave-one-out one.  The same point 1e20 times heavier rounds w h to 1:
    # the fallback.
    n = 11
    g = np.random.default_rng(17)
    x = np.sort(g.uniform(0.0, 1.0, n))
    v = g.normal(0, 1, n)
    w = np.ones(n)
    j = 5
    assert brute.half_width(n, 0.3) == 2
    w[j] = 8e10
    _, acvr = oracle.runline_raw(x, v, w, 0.3, 2, 0.0)
    _, ref = brute.runline(x, v, w, 0.3, 2, 0.0, tie_average=False)
    assert acvr[j] != acvr[j - 1]
    np.testing.assert_allclose(acvr[j], ref[j], rtol=1e-4)
    w[j] = 1e20
    _, acvr = oracle.runline_raw(x, v, w, 0.3, 2, 0.0)
    assert acvr[j] == acvr[j - 1]


@pytest.mark.parametrize("gap", [1e-2, 1e-4, 1e-6, 1e-9])
def test_cv_fallback_for_exact_leverage_one_whatever_the_gap(gap):
    # The clamped end window of the last point holds four tied abscissae and
    # the point itself, gap above them: its leverage is exactly 1 however
    # small the gap, while the computed 1 - w h is rounding noise that grows
    # as the gap shrinks (about 1e-13 already at 1e-4).  The residual must
    # fall back to the previous one at every gap.
    n = 12
    g = np.random.default_rng(5)
    x = np.sort(g.uniform(0.0, 0.8, n))
    x[n - 5:n - 1] = 0.85
    x[n - 1] = 0.85 + gap
    v = g.normal(0, 1, n)
    w = g.uniform(0.5, 2.0, n)
    _, acvr = oracle.runline_raw(x, v, w, 0.05, 1, 0.0)
    assert acvr[n - 1] == acvr[n - 2]
    _, ref = brute.runline(x, v, w, 0.05, 1, 0.0, tie_average=False)
    # (the other residuals come from nearly coincident abscissae at the
    # smallest gap: both computations lose about log10(1/gap) digits)
    np.testing.assert_allclose(acvr[:n - 1], ref[:n - 1], rtol=1e-5, atol=1e-11)
