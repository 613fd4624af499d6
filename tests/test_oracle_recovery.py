"""The SP reading against the one accuracy claim the paper makes for SP: the
single-pass variant finds correct periods about as often as the original
Super Smoother (Sec. 5.6: 84.6 % against 83.8 % of Stripe82 objects within
1 % of the catalogued period).  Stripe82 is not available; the check runs the
oracle on C3-shaped objects (sinusoids and box eclipses, n = 30..500) over a
100-day span, so that a 2,500-frequency grid resolves their peaks.  It is
deterministic (seeded inputs, thread-count-independent oracle)."""
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
