"""Pins of the oracle's Super Smoother (Listing 1) and single-pass variant
(Sec. 3, reading) against brute-force restatements built on explicit least
squares, and against invariants the method has by construction."""
import numpy as np
import pytest

import oracle
from tests import brute


def _lc(n, seed):
    g = np.random.default_rng(seed)
    x = np.sort(g.uniform(0.0, 1.0, n))
    y = np.sin(2 * np.pi * x) + g.normal(0.0, 0.3, n)
    w = g.uniform(0.5, 3.0, n)
    return x, y, w


@pytest.mark.parametrize("alpha", [0.0, 5.0, 9.0, 10.0])
@pytest.mark.parametrize("n,seed", [(8, 1), (13, 2), (21, 3), (34, 4)])
def test_supsmu_matches_brute_force(n, seed, alpha):
    x, y, w = _lc(n, seed)
    got = oracle.supsmu(x, y, w, iper=2, alpha=alpha)
    ref = brute.supsmu(x, y, w, alpha=alpha, iper=2)
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("alpha", [0.0, 9.0])
@pytest.mark.parametrize("n,seed", [(8, 5), (17, 6), (40, 7)])
def test_supsmu_sp_matches_brute_force(n, seed, alpha):
    x, y, w = _lc(n, seed)
    got = oracle.supsmu_sp(x, y, w, iper=2, alpha=alpha)
    ref = brute.supsmu_sp(x, y, w, alpha=alpha, iper=2)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-11)


def test_supsmu_nonperiodic_matches_brute_force():
    x, y, w = _lc(19, 8)
    np.testing.assert_allclose(oracle.supsmu(x, y, w, iper=1),
                               brute.supsmu(x, y, w, iper=1), rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(oracle.supsmu_sp(x, y, w, iper=1),
                               brute.supsmu_sp(x, y, w, iper=1), rtol=1e-10, atol=1e-11)


def test_linear_data_reproduced_nonperiodic():
    g = np.random.default_rng(9)
    x = np.sort(g.uniform(0, 1, 80))
    y = 0.5 - 3.0 * x
    w = g.uniform(1, 2, 80)
    np.testing.assert_allclose(oracle.supsmu(x, y, w, iper=1), y, atol=1e-11)
    np.testing.assert_allclose(oracle.supsmu_sp(x, y, w, iper=1), y, atol=1e-11)


def test_degenerate_abscissae_give_weighted_mean():
    x = np.full(10, 0.3)
    y = np.arange(10.0)
    w = np.linspace(1, 2, 10)
    m = np.sum(w * y) / np.sum(w)
    np.testing.assert_allclose(oracle.supsmu(x, y, w), m, rtol=1e-15)
    np.testing.assert_allclose(oracle.supsmu_sp(x, y, w), m, rtol=1e-15)


@pytest.mark.parametrize("fn", ["supsmu", "supsmu_sp"])
def test_affine_equivariance(fn):
    x, y, w = _lc(60, 10)
    f = getattr(oracle, fn)
    base = f(x, y, w)
    np.testing.assert_allclose(f(x, 2.5 * y + 40.0, w), 2.5 * base + 40.0, rtol=1e-12, atol=1e-10)


def test_one_distinct_abscissa_is_not_degenerate():
    # Listing 1 falls back to the weighted mean only when every abscissa is
    # equal (x[n-1] <= x[0]); with all but the last tied the smoother runs
    x = np.r_[np.full(9, 0.3), 0.7]
    g = np.random.default_rng(12)
    y = g.normal(0, 1, 10)
    w = g.uniform(0.5, 2, 10)
    for iper in (1, 2):
        got = oracle.supsmu(x, y, w, iper=iper)
        np.testing.assert_allclose(got, brute.supsmu(x, y, w, iper=iper), rtol=1e-9, atol=1e-10)
        assert np.ptp(got) > 1e-3
        np.testing.assert_allclose(oracle.supsmu_sp(x, y, w, iper=iper),
                                   brute.supsmu_sp(x, y, w, iper=iper), rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("fn", ["supsmu", "supsmu_sp"])
def test_periodic_mode_needs_abscissae_in_the_unit_interval(fn):
    # Listing 1 keeps periodic windows (iper = 2) only for 0 <= x[0] and
    # x[n-1] <= 1; outside, it smooths with clamped windows (jper = 1)
    f, bf = getattr(oracle, fn), getattr(brute, fn)
    x, y, w = _lc(17, 21)
    for xs in (np.r_[x[:-1], 1.2], np.r_[-0.1, x[1:]]):
        np.testing.assert_allclose(f(xs, y, w, iper=2), bf(xs, y, w, iper=1), rtol=1e-9, atol=1e-10)
    xs = np.r_[x[:-1], 1.0]                       # the closed end stays periodic
    periodic = bf(xs, y, w, iper=2)
    np.testing.assert_allclose(f(xs, y, w, iper=2), periodic, rtol=1e-9, atol=1e-10)
    assert np.max(np.abs(periodic - bf(xs, y, w, iper=1))) > 1e-3


@pytest.mark.parametrize("fn", ["supsmu", "supsmu_sp"])
def test_periodic_rotation_invariance(fn):
    # rotating the phase circle permutes the points but keeps every window's
    # relative geometry; a wrong sign in the +-1 wrap shift breaks this
    x, y, w = _lc(50, 11)
    f = getattr(oracle, fn)
    base = f(x, y, w)
    for delta in (0.13, 0.5, 0.91):
        xr = (x + delta) % 1.0
        order = np.argsort(xr, kind="stable")
        rot = f(xr[order], y[order], w[order])
        back = np.empty_like(rot)
        back[order] = rot
        np.testing.assert_allclose(back, base, rtol=1e-9, atol=1e-10)


def test_alpha_zero_never_enhances():
    # with alpha = 0 the chosen span is always one of the three spans, so the
    # final output equals brute force without the bass step
    x, y, w = _lc(30, 12)
    np.testing.assert_allclose(oracle.supsmu(x, y, w, alpha=0.0),
                               brute.supsmu(x, y, w, alpha=0.0), rtol=1e-9, atol=1e-10)
    assert not np.allclose(oracle.supsmu(x, y, w, alpha=0.0), oracle.supsmu(x, y, w, alpha=9.0))


def test_fixed_span_mode_is_one_running_line():
    x, y, w = _lc(25, 13)
    vs = brute.vsmlsq_of(x)
    ref, _ = brute.runline(x, y, w, 0.3, 2, vs)
    np.testing.assert_allclose(oracle.supsmu(x, y, w, span=0.3), ref, rtol=1e-10, atol=1e-11)


def test_vsmlsq_hand_values():
    # Listing 1: scale = x[3(n/4)-1] - x[n/4-1] (0-based), vsmlsq = 1e-6 scale^2
    x = np.arange(8) / 8.0          # i = 1, j = 5
    assert oracle.vsmlsq(x) == pytest.approx(1e-6 * (5 / 8 - 1 / 8) ** 2, rel=1e-15)
    x = np.arange(13) / 13.0        # n/4 = 3: i = 2, j = 8
    assert oracle.vsmlsq(x) == pytest.approx(1e-6 * (8 / 13 - 2 / 13) ** 2, rel=1e-15)
    x = np.array([0.0, 0.1, 0.4, 0.9])  # n = 4: i = 0, j = 2
    assert oracle.vsmlsq(x) == pytest.approx(1e-6 * 0.4 ** 2, rel=1e-15)


def test_vsmlsq_threshold_drops_slope_where_spread_is_small():
    # weights scaled so that window spreads straddle vsmlsq: the slope is then
    # dropped in some windows only, which the brute force reproduces only with
    # the same threshold
    x, y, w = _lc(24, 14)
    vs = brute.vsmlsq_of(x)
    for scale in (3e-5, 1e-4, 3e-4):
        ws = w * scale
        np.testing.assert_allclose(oracle.supsmu(x, y, ws), brute.supsmu(x, y, ws),
                                   rtol=1e-9, atol=1e-10)
    assert vs > 0


def test_clamp_of_smoothed_span_matters():
    # clustered phases make the midrange line through the chosen spans
    # overshoot [0.05, 0.5]; Listing 1 clamps before interpolating
    g = np.random.default_rng(2)
    x = np.sort(np.concatenate([g.uniform(0.0, 0.08, 10), g.uniform(0.5, 0.55, 10),
                                g.uniform(0, 1, 4)]))
    y = np.where(x < 0.3, 0.0, 1.0) + g.normal(0, 0.05, 24) + 3 * np.sin(6 * x)
    w = g.uniform(0.5, 3, 24)
    np.testing.assert_allclose(oracle.supsmu(x, y, w), brute.supsmu(x, y, w),
                               rtol=1e-9, atol=1e-10)


def test_both_clamps_of_smoothed_span_matter():
    # with clamped (one-sided at the ends) windows the same kind of input
    # drives the smoothed span below the tweeter's 0.05 at one end and above
    # the woofer's 0.5 elsewhere, so each clamp bound changes the output
    # (40 points, so that the tweeter's and the midrange's half widths differ
    # and the interpolation below the tweeter's span is not flat)
    g = np.random.default_rng(138)
    x = np.sort(np.concatenate([g.uniform(0.0, 0.08, 16), g.uniform(0.5, 0.55, 16),
                                g.uniform(0, 1, 8)]))
    y = np.where(x < 0.3, 0.0, 1.0) + g.normal(0, 0.05, 40) + 3 * np.sin(6 * x)
    w = g.uniform(0.5, 3, 40)
    assert oracle.half_width(40, 0.05) < oracle.half_width(40, 0.2)
    ref, span = brute.supsmu(x, y, w, iper=1, return_span=True)
    assert span.min() < 0.03 and span.max() > 0.52
    np.testing.assert_allclose(oracle.supsmu(x, y, w, iper=1), ref, rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("iper", [1, 2])
@pytest.mark.parametrize("n", [8, 17, 40])
def test_spg_matches_brute_force(n, iper):
    g = np.random.default_rng(1000 + n + iper)
    x = np.sort(g.uniform(0, 1, n))
    if n >= 17:
        x[5:8] = x[5]            # a tie run
    y = np.sin(2 * np.pi * 3 * x) + g.normal(0, 0.3, n)
    w = g.uniform(0.5, 2.0, n)
    smo, k = oracle.supsmu_spg(x, y, w, iper=iper)
    ref, kref = brute.supsmu_spg(x, y, w, iper=iper)
    assert k == kref
    np.testing.assert_allclose(smo, ref, rtol=1e-10, atol=1e-12)


def test_spg_chooses_the_span_the_data_want():
    # a fast oscillation is followed best by the tweeter, a flat noisy line
    # by the woofer: the global score picks each, and equal spans reduce
    # SPG to that span's running line
    g = np.random.default_rng(7)
    n = 300
    x = np.sort(g.uniform(0, 1, n))
    w = np.ones(n)
    fast = np.sin(2 * np.pi * 12 * x) + g.normal(0, 0.05, n)
    flat = g.normal(0, 1.0, n)
    assert oracle.supsmu_spg(x, fast, w)[1] == 0
    assert oracle.supsmu_spg(x, flat, w)[1] == 2
    smo, k = oracle.supsmu_spg(x, fast, w, spans=(0.2, 0.2, 0.2))
    ref, _ = oracle.runline(x, fast, w, 0.2, -2, oracle.vsmlsq(x))
    assert k == 0
    np.testing.assert_allclose(smo, ref, rtol=1e-12, atol=1e-12)
