"""Host logic of bench.py's accuracy checks, on the CPU: the serving run's
oracle check of a sample of requests reports a zero error for results equal
to the oracle's and catches a perturbed one."""
import numpy as np

import bench
import oracle
from paper_2111_07396_gb300 import synth


def _requests():
    # three requests of the serving mix's shape (n ~ logU(30, 3000)), both
    # variants, on a short grid
    arrivals, cat, variants = synth.config5_arrivals(200.0, 0.05, 64)
    objs = [cat.obj(k) for k in range(3)]
    return objs, variants[:3], cat.freq


def test_serve_check_of_oracle_results_is_exact():
    objs, variants, freq = _requests()
    codes = (oracle.SS, oracle.SP)
    served = {}
    for i, (t, y, dy) in enumerate(objs):
        p, _ = oracle.periodogram(t, y, dy, [t.size], freq, codes[variants[i]])
        served[i] = p[0]
    chk = bench.serve_oracle_check(objs, served, variants, freq, k=6)
    assert chk["requests"] == 3 and chk["frequencies"] >= 3 * 6
    assert chk["max_gate_err"] < 1e-12


def test_serve_check_catches_a_wrong_power():
    objs, variants, freq = _requests()
    codes = (oracle.SS, oracle.SP)
    t, y, dy = objs[0]
    p, _ = oracle.periodogram(t, y, dy, [t.size], freq, codes[variants[0]])
    bad = p[0].copy()
    bad[int(np.argmax(bad))] *= 1.01      # the best frequency is always sampled
    chk = bench.serve_oracle_check(objs[:1], {0: bad}, variants, freq, k=4)
    assert chk["max_gate_err"] > 5e-3
