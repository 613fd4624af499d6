"""Pins of the oracle's span choice, bass enhancement and interpolation
(Listing 1) on inputs whose whole Super Smoother output has a closed form.

On a uniform periodic grid x_j = j/n with unit weights every window is
symmetric about its centre, so a running line evaluated at the centre is the
mean of its window and the cross-validated residual (leave-one-out, Sec. 2.2)
is |y_j - mean of the other window points|.  For y = cos(2 pi x) and for the
alternating sequence y = (-1)^j these means are known sums, the residual
columns are one column times a constant per span, and so the span choice is
the same at every centre.  The expected outputs below are written from those
sums and from hand-evaluated span arithmetic; nothing re-walks the Listing.
A wrong argmin, a woofer/tweeter swap, a wrong bass exponent or target, or an
interpolation toward the wrong fit changes the output at every point; so does,
on an exact three-way tie, taking the last minimum or a bass step at equality.
"""
import numpy as np
import pytest

from oracle import oracle


def _grid(n):
    return np.arange(n) / n, np.ones(n)


def _cos_sum(h, n):
    # sum_{k=-h}^{h} cos(2 pi k / n): the Dirichlet kernel
    return float(np.cos(2 * np.pi * np.arange(-h, h + 1) / n).sum())


def test_half_widths_of_the_cases():
    # trunc(0.5 span n + 0.5), as the cases below assume
    assert [oracle.half_width(100, s) for s in (0.05, 0.2, 0.5)] == [3, 10, 25]
    assert [oracle.half_width(110, s) for s in (0.05, 0.2, 0.5)] == [3, 11, 28]
    assert [oracle.half_width(96, s) for s in (0.05, 0.2, 0.5)] == [2, 10, 24]
    assert [oracle.half_width(28, s) for s in (0.05, 0.2, 0.5)] == [2, 3, 7]


@pytest.mark.parametrize("alpha", [0.0, 9.0])
def test_tweeter_wins_on_a_cosine(alpha):
    # y = cos(2 pi x): a window mean is cos(2 pi x_j) m_h, m_h = D_h / (2h+1),
    # and the leave-one-out mean cos(2 pi x_j) c_h, c_h = (D_h - 1) / (2h).
    # The residual |cos| (1 - c_h) grows with h (more curvature bias), so the
    # tweeter (h = 3) wins everywhere.  Midrange smoothing of the residual
    # columns keeps their ratio, so the bass step sees the same ratio
    # q = (1 - c_3) / (1 - c_25) at every centre: span 0.05 + 0.45 q for
    # alpha = 9 (exponent 10 - 9 = 1), 0.05 for alpha = 0 (no bass).
    n = 100
    x, w = _grid(n)
    y = np.cos(2 * np.pi * x)
    m = {h: _cos_sum(h, n) / (2 * h + 1) for h in (3, 10, 25)}
    c = {h: (_cos_sum(h, n) - 1) / (2 * h) for h in (3, 10, 25)}
    q = (1 - c[3]) / (1 - c[25])
    assert 0.02 < q < 0.03
    s = 0.05 + 0.45 * q if alpha == 9.0 else 0.05
    # the smoothed span is the constant s; below the midrange span the smooth
    # is (1 - f) midrange + f tweeter with f = (s - 0.2) / (0.05 - 0.2)
    f = (s - 0.2) / (0.05 - 0.2)
    v = y * ((1 - f) * m[10] + f * m[3])
    expected = v * m[3]                      # final tweeter smooth
    got = oracle.supsmu(x, y, w, iper=2, alpha=alpha)
    np.testing.assert_allclose(got, expected, rtol=0, atol=1e-13)


@pytest.mark.parametrize("alpha", [0.0, 9.0])
def test_midrange_wins_on_an_alternating_sequence(alpha):
    # y = (-1)^j, n = 100, half widths 3, 10, 25.  The leave-one-out mean of a
    # window of half width h is (-1)^j (S_h - 1) / (2h) with S_h the sum of
    # (-1)^k over k = -h..h: -1 for odd h, +1 for even h.  Residuals: 4/3
    # (h = 3), 1 (h = 10), 1.04 (h = 25): the midrange wins.  With alpha = 9
    # the span moves toward the woofer's by the residual ratio 1/1.04:
    # 0.2 + 0.3 / 1.04.  Window means: (-1)^j / 21 (h = 10), -(-1)^j / 51
    # (h = 25), -(-1)^j / 7 (h = 3).
    n = 100
    x, w = _grid(n)
    sgn = (-1.0) ** np.arange(n)
    if alpha == 0.0:
        v = sgn / 21.0                       # span 0.2: the midrange smooth
    else:
        f = (0.3 / 1.04) / 0.3               # (s - 0.2) / (0.5 - 0.2)
        v = (1 - f) * sgn / 21.0 + f * (-sgn / 51.0)
    expected = v * (-1.0 / 7.0)
    got = oracle.supsmu(x, sgn, w, iper=2, alpha=alpha)
    np.testing.assert_allclose(got, expected, rtol=0, atol=1e-15)


@pytest.mark.parametrize("alpha", [0.0, 9.0])
def test_woofer_wins_on_an_alternating_sequence(alpha):
    # n = 110, half widths 3, 11, 28: residuals 4/3, 1 + 1/11 and 1, so the
    # woofer wins; bass enhancement applies only below the woofer's residual,
    # so alpha changes nothing.  Smooth: woofer mean (-1)^j / 57, then the
    # final tweeter smooth multiplies by -1/7.
    n = 110
    x, w = _grid(n)
    sgn = (-1.0) ** np.arange(n)
    expected = -sgn / 399.0
    got = oracle.supsmu(x, sgn, w, iper=2, alpha=alpha)
    np.testing.assert_allclose(got, expected, rtol=0, atol=1e-15)


@pytest.mark.parametrize("alpha", [0.0, 9.0, 10.0])
def test_three_way_tie_keeps_the_tweeter(alpha):
    # n = 96, half widths 2, 10, 24, all even: every leave-one-out mean of
    # (-1)^j is 0, so all three residuals are exactly 1 at every centre.  The
    # span choice takes the first strict minimum (the tweeter), and since
    # that minimum is not below the woofer's residual no bass step applies,
    # for any alpha.  The tie is exact in binary64 as well: the residual is
    # |y_j - fit_j| / (1 - leverage_j) with fit_j = (-1)^j / m and leverage
    # 1/m, so numerator and denominator are the same rounded 1 - 1/m.
    # Smooth: tweeter mean (-1)^j / 5, then the final tweeter smooth, 1/25.
    # Taking the last minimum, or a bass step at equality, gives the woofer
    # instead: (-1)^j / 245.
    n = 96
    x, w = _grid(n)
    sgn = (-1.0) ** np.arange(n)
    got = oracle.supsmu(x, sgn, w, iper=2, alpha=alpha)
    np.testing.assert_allclose(got, sgn / 25.0, rtol=0, atol=1e-15)


def test_sp_reading_on_the_same_cases():
    # The SP reading (one sweep, generalized validation g = |y - s| / (1 - nu/m)
    # with nu = 2 where the line keeps its slope, as it does here): on the
    # alternating n = 110 sequence the fits at the centre are the window means
    # -(-1)^j / 7, -(-1)^j / 23 and (-1)^j / 57, so g is (8/7) / (5/7) = 1.6
    # (tweeter), (24/23) / (21/23) = 8/7 (midrange) and (56/57) / (55/57) =
    # 56/55 (woofer): the woofer wins, no bass applies, and the SP smooth is
    # the woofer's fit with no further smoothing.
    n = 110
    x, w = _grid(n)
    sgn = (-1.0) ** np.arange(n)
    got = oracle.supsmu_sp(x, sgn, w, iper=2, alpha=9.0)
    np.testing.assert_allclose(got, sgn / 57.0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n,span,fit", [(100, 1, 1.0 / 21.0), (110, 2, 1.0 / 57.0),
                                        (28, 2, -1.0 / 15.0)])
def test_spg_reading_on_alternating_sequences(n, span, fit):
    # The SPG reading (one span per frequency, least summed squared
    # generalized-validation residual, reading 15): on y = (-1)^j every point
    # has the same residual per span, |1 - fit_h| / (1 - 2/m) with the window
    # means fit_h = +-1/(2h+1) of the cases above: n = 100 gives 1.6, 20/19
    # and 52/49 (the midrange wins), n = 110 gives 1.6, 8/7 and 56/55 (the
    # woofer wins).  The smooth is that span's fit, (-1)^j / 21 or / 57.
    # n = 28 (half widths 2, 3, 7) gives 4/3, 1.6 and 16/13: the woofer wins
    # only through the denominator, since with m one larger in it (6 and 16)
    # the tweeter's 1.2 would beat the woofer's 1.22.  Its fit is -(-1)^j / 15.
    x, w = _grid(n)
    sgn = (-1.0) ** np.arange(n)
    got, k = oracle.supsmu_spg(x, sgn, w, iper=2)
    assert k == span
    np.testing.assert_allclose(got, sgn * fit, rtol=0, atol=1e-15)


def test_spg_reading_on_a_cosine():
    # On y = cos(2 pi x) the residual of span h is |cos(2 pi x_j)| (1 - m_h) /
    # (1 - 2/m): the same column times a constant per span, smallest for the
    # tweeter (the least curvature bias), so SPG takes the tweeter's fit,
    # cos(2 pi x) m_3.
    n = 100
    x, w = _grid(n)
    y = np.cos(2 * np.pi * x)
    got, k = oracle.supsmu_spg(x, y, w, iper=2)
    assert k == 0
    m3 = _cos_sum(3, n) / 7
    np.testing.assert_allclose(got, y * m3, rtol=0, atol=1e-13)
