"""Claims the paper makes about results, checked on synthetic data.

The SP reading against the one accuracy claim the paper makes for SP: the
single-pass variant finds correct periods about as often as the original
Super Smoother (Sec. 5.6: 84.6 % against 83.8 % of Stripe82 objects within
1 % of the catalogued period).  Stripe82 is not available; the check runs the
oracle on C3-shaped objects (sinusoids and box eclipses, n = 30..500) over a
100-day span, so that a 2,500-frequency grid resolves their peaks.  And the
choice of alpha for transits (Sec. 5.4).  Both are deterministic (seeded
inputs, thread-count-independent oracle)."""
import numpy as np

import oracle
from paper_2111_07396_gb300 import synth


def test_sp_reading_finds_periods_as_often_as_ss():
    cat = synth.config3(n_objects=230, n_freq=2500, t_span=100.0)
    keep = [o for o in range(cat.n_objects) if np.isfinite(cat.periods[o])][:160]
    sub = cat.subset(keep)
    period = cat.periods[keep]
    rate = {}
    for name, code in (("ss", oracle.SS), ("sp", oracle.SP)):
        _, best = oracle.periodogram(sub.t, sub.y, sub.dy, sub.n_per_object, sub.freq, code)
        rate[name] = float(np.mean(np.abs(best / period - 1.0) < 0.01))
    # both find most periods, and SP is not behind SS by more than a few
    # objects (on this sample it is ahead, as in the paper)
    assert rate["ss"] > 0.4 and rate["sp"] > 0.4, rate
    assert rate["sp"] >= rate["ss"] - 0.03, rate


def test_alpha_zero_finds_transit_periods():
    # Sec. 5.4: for transiting exoplanets the in-transit points are the
    # signal, so bass enhancement (which treats them as outliers) hurts and
    # alpha = 0 finds every period.  Synthetic transits on a 27-day span with
    # a 1-day gap (a TESS sector's shape): duty 2-5 %, depth 0.3-1 %, noise
    # 0.1 %, periods 1.5-8 d.
    g = np.random.default_rng(5)
    freq = np.linspace(0.05, 1.5, 1500)
    found = {0.0: 0, 9.0: 0}
    for _ in range(12):
        t = np.sort(g.uniform(0, 27, 800))
        t = t[(t < 13) | (t > 14)]
        period, duty, depth = g.uniform(1.5, 8.0), g.uniform(0.02, 0.05), g.uniform(0.003, 0.01)
        phase = ((t - g.uniform(0, period)) / period) % 1.0
        y = np.where(phase < duty, -depth, 0.0) + g.normal(0, 0.001, t.size)
        dy = np.full(t.size, 0.001)
        for alpha in found:
            _, best = oracle.periodogram(t, y, dy, [t.size], freq, oracle.SS, alpha=alpha)
            found[alpha] += abs(best[0] / period - 1.0) < 0.01
    assert found[0.0] == 12, found
    assert found[9.0] < found[0.0], found
