"""Host model of the window initialisation in the periodic extension
(win_init_body, ext_prefix, chunk_lower, chunk_nearest and divn in
csrc/ssp_device.cuh).

The kernel gives each of its G threads a chunk of centres.  Chunk u starts at
floor(u n / G), moved forward past any run of tied phases it would split, and
the per-chunk raw moments (sum w, sum w x, sum w x^2, sum w v, sum w x v) are
prefix-summed.  The sums over a window [c - h, c + h] of the periodic
extension (slot e is point e mod n with x shifted by whole periods) are then
the difference of two prefixes taken at the chunk boundaries nearest to the
window's ends -- each moved to its period by the moment transforms of a
shift x -> x + k -- plus or minus the points between each end and its
boundary.  The model follows that index arithmetic step by step, on integer
data so every sum is exact, and checks that

- the fixed-point division that replaces integer division by n is exact over
  every dividend the kernel forms (objects of up to 65,535 points, CTAs of up
  to 512 threads);
- the first guess of chunk_lower is never below the answer (the kernel only
  walks down);
- every slot and chunk index stays in range;
- the decomposed sums equal the window sums taken point by point, for
  periodic and clamped windows, sparse and dense ties, and every CTA size.

The Super Smoother's running line (Sec. 2.2's cited smoother) is defined by
these window sums; the GPU parity tests check the kernel's results, this file
the bookkeeping that the kernel uses to reach them.
"""
import random

import numpy as np
import pytest

MAX_N = 65535          # largest object the library accepts
GROUP_SIZES = (32, 64, 128, 256, 512)


# ---- the kernel's fixed-point division by n ----
def divn_make(n):
    L = 0
    while (1 << L) < n:
        L += 1
    s = 26 + L
    m = (((1 << s) // n) + 1) & 0xFFFFFFFF       # uint32 multiplier
    return m, s


def divn(a, d):
    assert 0 <= a < (1 << 32)                    # the kernel passes a uint32
    return (a * d[0]) >> d[1]


def test_divn_is_exact_over_the_kernels_dividends():
    # chunk_lower divides p G + n - 1 with 0 <= p <= n.  The floor of a m / 2^s
    # drifts above floor(a / n) first just below a multiple of n, and the
    # drift grows with a, so the largest dividend congruent to n - 1 is the
    # worst case below the largest dividend; both are checked for every n.
    n = np.arange(1, MAX_N + 1, dtype=np.int64)
    L = np.ceil(np.log2(n)).astype(np.int64)     # smallest L with 2^L >= n
    for k in (1, 2, 3, 4, 5, 256, 257, MAX_N):
        assert divn_make(k)[1] == 26 + L[k - 1]
    s = 26 + L
    m = (np.left_shift(np.int64(1), s) // n) + 1
    assert m.max() < (1 << 32)
    G = max(GROUP_SIZES)
    amax = n * G + n - 1
    assert amax.max() < (1 << 31)                # p G fits the kernel's int
    worst = amax - ((amax + 1) % n)              # largest a = n - 1 (mod n), a <= amax
    for a in (amax, worst, n * (G // 2) + n - 1):
        got = (a * m) >> s                       # a m < 2^63: exact in int64
        np.testing.assert_array_equal(got, a // n)
    # and every dividend for a few small objects
    for k in (1, 2, 3, 5, 7, 31, 100, 257):
        d = divn_make(k)
        assert all(divn(a, d) == a // k for a in range(k * G + k))


# ---- chunk starts and boundary lookups, as the kernel forms them ----
def chunk_starts(n, G, tie):
    lg = G.bit_length() - 1
    cs = []
    for t in range(G):
        c = (t * n) >> lg                        # floor(t n / G)
        while 0 < c < n and tie[c - 1]:
            c += 1
        cs.append(c)
    cs.append(n)
    return cs


def chunk_lower(cs, G, n, dn, p):
    assert 0 <= p <= n
    u = divn(p * G + n - 1, dn)                  # ceil(p G / n)
    assert 0 <= u <= G and cs[u] >= p            # never too low: the kernel only walks down
    while u > 0 and cs[u - 1] >= p:
        u -= 1
    return u


def chunk_nearest(cs, G, n, dn, p):
    u = chunk_lower(cs, G, n, dn, p)
    return u - 1 if (u > 0 and p - cs[u - 1] < cs[u] - p) else u


# ---- moments and their transforms under a shift by k periods ----
def moments(w, x, v):
    return [w, w * x, w * x * x, w * v, w * x * v]


def add(a, b, sg=1):
    return [p + sg * q for p, q in zip(a, b)]


def shift(M, k, per):
    W, S1, S2, C, D = M
    return [W, S1 + k * per * W, S2 + 2 * k * per * S1 + k * k * per * per * W, C, D + k * per * C]


def check_case(rng, n, G, periodic, tie_span, trials):
    per = tie_span + 1                           # the period in the integer abscissa
    w = [rng.randint(1, 5) for _ in range(n)]
    X = sorted(rng.randint(0, tie_span) for _ in range(n))
    V = [rng.randint(-9, 9) for _ in range(n)]
    tie = [X[j] == X[j + 1] for j in range(n - 1)] + [False]
    cs = chunk_starts(n, G, tie)
    assert all(cs[u] <= cs[u + 1] for u in range(G))
    assert all(not tie[cs[u] - 1] for u in range(1, G) if 0 < cs[u] < n)   # no run split
    dn = divn_make(n)
    P = [[0] * 5]
    for u in range(G):
        acc = P[-1]
        for j in range(cs[u], cs[u + 1]):
            acc = add(acc, moments(w[j], X[j], V[j]))
        P.append(acc)
    T = P[G]

    def ext_prefix(u, k):
        # prefix before boundary u of period k of the periodic extension
        if k == 0:
            return P[u]
        if k < 0:
            return shift(add(P[u], T, -1), -1, per)
        return add(T, shift(P[u], 1, per))

    hmax = (n - 1) // 2
    for _ in range(trials):
        c = rng.randrange(n)
        h = rng.randint(1, hmax) if hmax >= 1 else 0
        if periodic:
            ea = c - h
        else:
            lo = c - h
            ea = 0 if lo < 0 else (n - 1 - 2 * h if lo > n - 1 - 2 * h else lo)
        eb = ea + 2 * h
        assert -n < ea and eb + 1 < 2 * n
        ka = -1 if ea < 0 else 0
        kb = 1 if eb + 1 > n else 0
        if not periodic:
            assert ka == 0 and kb == 0
        pa, pb = ea - ka * n, eb + 1 - kb * n
        assert 0 <= pa < n and 0 < pb <= n
        ua = chunk_nearest(cs, G, n, dn, pa)
        ub = chunk_nearest(cs, G, n, dn, pb)
        S = add(ext_prefix(ub, kb), ext_prefix(ua, ka), -1)
        qa, qb = cs[ua], cs[ub]
        la, nl, sl = (pa, qa - pa, 1) if qa >= pa else (qa, pa - qa, -1)
        lb, nr, sr = (qb, pb - qb, 1) if qb <= pb else (pb, qb - pb, -1)
        for k in range(max(nl, nr)):
            if k < nl:
                p = la + k
                assert 0 <= p < n
                S = add(S, shift(moments(w[p], X[p], V[p]), ka, per), sl)
            if k < nr:
                p = lb + k
                assert 0 <= p < n
                S = add(S, shift(moments(w[p], X[p], V[p]), kb, per), sr)
        ref = [0] * 5
        for e in range(ea, eb + 1):
            k = -1 if e < 0 else (1 if e >= n else 0)
            p = e - k * n
            ref = add(ref, shift(moments(w[p], X[p], V[p]), k, per))
        assert S == ref, (n, G, periodic, c, h)


SIZES = list(range(4, 40)) + [63, 64, 65, 100, 257, 1000, 1537, 3000, 4097]


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("G", GROUP_SIZES)
def test_window_sums_from_prefixes_equal_point_sums(G, periodic):
    rng = random.Random(1000 * G + periodic)
    for n in SIZES:
        trials = 12 if n < 1000 else 4
        check_case(rng, n, G, periodic, 10 * n, trials)       # few ties
        check_case(rng, n, G, periodic, max(1, n // 8), trials)  # runs of about 8 ties


def test_all_points_tied():
    # one run of ties: every chunk start but the first is pushed to n, so
    # every window comes from its ragged ends and boundary n is reached
    # from any p
    rng = random.Random(7)
    for n in (5, 33, 300):
        for G in (32, 512):
            check_case(rng, n, G, True, 0, 20)
            check_case(rng, n, G, False, 0, 20)
