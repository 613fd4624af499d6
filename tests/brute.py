"""Independent brute-force restatements used to pin the oracle.

Nothing here calls the oracle's arithmetic.  The running line is computed as
an explicit weighted least-squares problem (numpy ``lstsq`` on the window's
design matrix), leave-one-out residuals by refitting without the point, and
Listing 1 / the single-pass reading are re-walked on top of those fits.  They
are O(n^2) or worse and meant for n of a few dozen points.
"""
from __future__ import annotations

import numpy as np

SPANS = (0.05, 0.2, 0.5)


def half_width(n: int, span: float) -> int:
    ibw = int(np.floor(0.5 * span * n + 0.5))
    ibw = max(ibw, 2)
    return min(ibw, (n - 1) // 2)


def window(n: int, ibw: int, periodic: bool, j: int, x: np.ndarray):
    """(point indices, abscissae) of point j's window."""
    if periodic:
        slots = np.arange(j - ibw, j + ibw + 1)
        idx = np.mod(slots, n)
        xs = x[idx] + np.floor_divide(slots, n)  # -1 before 0, +1 past n-1
        return idx, xs
    lo = min(max(j - ibw, 0), n - 1 - 2 * ibw)
    idx = np.arange(lo, lo + 2 * ibw + 1)
    return idx, x[idx]


def wls_line(xs, vs, ws, x0, vsmlsq=0.0):
    """Weighted least-squares line through (xs, vs) evaluated at x0; a plain
    weighted mean when the weighted spread of xs does not exceed vsmlsq.  The
    spread of equal abscissae is 0 exactly (a computed mean of equal values
    may round off them and leave a spread of rounding noise)."""
    xm = np.sum(ws * xs) / np.sum(ws)
    sxx = 0.0 if np.all(xs == xs[0]) else np.sum(ws * (xs - xm) ** 2)
    if not sxx > vsmlsq:
        return np.sum(ws * vs) / np.sum(ws), False
    A = np.stack([np.ones_like(xs), xs], axis=1) * np.sqrt(ws)[:, None]
    coef, *_ = np.linalg.lstsq(A, vs * np.sqrt(ws), rcond=None)
    return coef[0] + coef[1] * x0, True


def runline(x, v, w, span, iper, vsmlsq=0.0, tie_average=True):
    n = x.size
    ibw = half_width(n, span)
    periodic = abs(iper) == 2
    smo = np.empty(n)
    acvr = np.zeros(n)
    for j in range(n):
        idx, xs = window(n, ibw, periodic, j, x)
        smo[j], _ = wls_line(xs, v[idx], w[idx], x[j], vsmlsq)
        if iper > 0:
            # explicit leave-one-out refit: drop point j's own slot
            keep = idx != j
            fit_loo, _ = wls_line(xs[keep], v[idx][keep], w[idx][keep], x[j], vsmlsq)
            acvr[j] = abs(v[j] - fit_loo)
    if tie_average:
        smo = tie_avg(x, w, smo)
    return smo, acvr


def tie_avg(x, w, s):
    s = s.copy()
    n = x.size
    j = 0
    while j < n:
        k = j
        while k + 1 < n and x[k + 1] == x[k]:
            k += 1
        if k > j:
            s[j:k + 1] = np.sum(w[j:k + 1] * s[j:k + 1]) / np.sum(w[j:k + 1])
        j = k + 1
    return s


def vsmlsq_of(x):
    n = x.size
    i = n // 4 - 1
    j = 3 * (n // 4) - 1
    return 1e-6 * (x[j] - x[i]) ** 2


def _select(res, res_woof, alpha, fallback, spans):
    best = None
    for i in range(3):
        if res[i] < 1e20 and (best is None or res[i] < res[best]):
            best = i
    s = fallback if best is None else spans[best]
    rmin = 1e20 if best is None else res[best]
    if 0 < alpha <= 10 and 0 < rmin < res_woof:
        s = s + (spans[2] - s) * max(rmin / res_woof, 1e-7) ** (10.0 - alpha)
    return s


def _interp(s, tw, mid, woof, spans):
    s = min(max(s, spans[0]), spans[2])
    f = s - spans[1]
    if f < 0:
        g = f / (spans[0] - spans[1])
        return (1 - g) * mid + g * tw
    g = f / (spans[2] - spans[1])
    return (1 - g) * mid + g * woof


def supsmu(x, y, w, alpha=9.0, iper=2, spans=SPANS, return_span=False):
    """Listing 1 on top of brute-force running lines (CV by explicit LOO).
    With return_span the smoothed span column (before its clamp) comes back
    as well, so that a test can show which clamp its input reaches."""
    n = x.size
    if x[-1] <= x[0]:
        out = np.full(n, np.sum(w * y) / np.sum(w))
        return (out, None) if return_span else out
    vs = vsmlsq_of(x)
    smo, res, raw = [], [], []
    for s in spans:
        sm, cv = runline(x, y, w, s, iper, vs)
        rr, _ = runline(x, cv, w, spans[1], -iper, vs)
        smo.append(sm)
        res.append(rr)
        raw.append(cv)
    chosen = np.array([_select([res[0][j], res[1][j], res[2][j]], res[2][j], alpha,
                                raw[2][j], spans) for j in range(n)])
    sm_span, _ = runline(x, chosen, w, spans[1], -iper, vs)
    v = np.array([_interp(sm_span[j], smo[0][j], smo[1][j], smo[2][j], spans)
                  for j in range(n)])
    out, _ = runline(x, v, w, spans[0], -iper, vs)
    return (out, sm_span) if return_span else out


def supsmu_sp(x, y, w, alpha=9.0, iper=2, spans=SPANS):
    """Single-pass generalized-validation reading on brute-force window fits."""
    n = x.size
    if x[-1] <= x[0]:
        return np.full(n, np.sum(w * y) / np.sum(w))
    vs = vsmlsq_of(x)
    periodic = abs(iper) == 2
    out = np.empty(n)
    for j in range(n):
        fits, g = [], []
        for s in spans:
            ibw = half_width(n, s)
            idx, xs = window(n, ibw, periodic, j, x)
            fit, sloped = wls_line(xs, y[idx], w[idx], x[j], vs)
            m = 2 * ibw + 1
            nu = 2.0 if sloped else 1.0
            fits.append(fit)
            g.append(abs(y[j] - fit) / (1.0 - nu / m))
        s = _select(g, g[2], alpha, spans[2], spans)
        out[j] = _interp(s, fits[0], fits[1], fits[2], spans)
    return tie_avg(x, w, out)


def supsmu_spg(x, y, w, iper=2, spans=SPANS):
    """Global generalized-validation reading: per span, the weighted sum of
    squared GCV residuals over all points; the least-score span's running
    line, tie-averaged.  Returns (smooth, chosen span index)."""
    n = x.size
    if x[-1] <= x[0]:
        return np.full(n, np.sum(w * y) / np.sum(w)), -1
    vs = vsmlsq_of(x)
    periodic = abs(iper) == 2
    fits, scores = [], []
    for s in spans:
        ibw = half_width(n, s)
        m = 2 * ibw + 1
        f = np.empty(n)
        score = 0.0
        for j in range(n):
            idx, xs = window(n, ibw, periodic, j, x)
            f[j], sloped = wls_line(xs, y[idx], w[idx], x[j], vs)
            nu = 2.0 if sloped else 1.0
            score += w[j] * (abs(y[j] - f[j]) / (1.0 - nu / m)) ** 2
        fits.append(f)
        scores.append(score)
    k = 0
    for i in (1, 2):
        if scores[i] < scores[k]:
            k = i
    return tie_avg(x, w, fits[k]), k
