"""The serving loop (ssp_server_*): every request's results equal
ssp_periodogram on that object alone, whatever shares its batch; tickets are
reported once; the in-flight cap and input checks hold."""
import numpy as np
import pytest

from oracle import oracle
from paper_2111_07396_gb300 import build as ssp_build
from paper_2111_07396_gb300 import ssp, synth
from tests.parity import TOL, gate_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ssp_build.build()
    ssp.lib()


def _objects(k, n_freq=300):
    cat = synth.config3(n_objects=k, n_freq=n_freq, n_hi=1600)
    out = []
    for o in range(k):
        a, b = cat.offsets[o], cat.offsets[o + 1]
        out.append((cat.t[a:b], cat.y[a:b], cat.dy[a:b]))
    return cat.freq, out


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("max_wait_ms", [0.0, 3.0])
def test_results_equal_single_object_calls(precision, max_wait_ms):
    freq, objs = _objects(24)
    variants = ["ss" if k % 3 else "sp" for k in range(len(objs))]
    with ssp.Server(freq, precision=precision, max_wait_ms=max_wait_ms,
                    max_batch_ptf=4e5) as srv:
        tickets = [srv.submit(t, y, dy, v) for (t, y, dy), v in zip(objs, variants)]
        assert tickets == list(range(1, len(objs) + 1))
        seen = []
        while len(seen) < len(tickets):
            tk = srv.next(wait_ms=20000)
            assert tk is not None
            seen.append(tk)
        assert sorted(seen) == tickets
        for tk, (t, y, dy), v in zip(tickets, objs, variants):
            power, best, lat = srv.poll(tk)
            ref, ref_best = ssp.ssp_periodogram(t, y, dy, [t.size], freq, variant=v,
                                                precision=precision)
            np.testing.assert_array_equal(power, ref[0])
            assert best == ref_best[0] and lat >= 0.0


def test_results_meet_oracle_tolerance():
    freq, objs = _objects(4, n_freq=200)
    with ssp.Server(freq) as srv:
        for v, code in (("ss", oracle.SS), ("sp", oracle.SP)):
            tks = [srv.submit(t, y, dy, v) for t, y, dy in objs]
            for tk, (t, y, dy) in zip(tks, objs):
                power, _, _ = srv.poll(tk, wait_ms=20000)
                ref, _ = oracle.periodogram(t, y, dy, [t.size], freq, code)
                assert gate_error(power[None, :], ref) <= TOL["fp32c"]


def test_in_flight_cap_and_ticket_rules():
    freq, objs = _objects(3)
    (t, y, dy) = objs[0]
    with ssp.Server(freq, max_in_flight=2) as srv:
        a = srv.submit(t, y, dy)
        b = srv.submit(t, y, dy, "sp")
        with pytest.raises(ssp.SSPError) as ei:
            srv.submit(t, y, dy)
        assert ei.value.status == ssp.SSP_ERR_BUSY
        assert srv.poll(a, wait_ms=20000) is not None
        c = srv.submit(t, y, dy)           # a is collected: room again
        assert c == 3
        with pytest.raises(ssp.SSPError) as ei:
            srv.poll(a)                    # retired
        assert ei.value.status == ssp.SSP_ERR_ARG
        assert srv.poll(b, wait_ms=20000) is not None
        assert srv.poll(c, wait_ms=20000) is not None
        assert srv.next(wait_ms=0) is None  # every finished ticket was collected


def test_submit_checks_inputs():
    freq, objs = _objects(1)
    t, y, dy = objs[0]
    with ssp.Server(freq) as srv:
        for bad in (dict(y=np.r_[y[:-1], np.nan]), dict(dy=np.r_[dy[:-1], 0.0]),
                    dict(t=t[:3], y=y[:3], dy=dy[:3])):
            args = dict(t=t, y=y, dy=dy)
            args.update(bad)
            with pytest.raises(ssp.SSPError) as ei:
                srv.submit(**args)
            assert ei.value.status == ssp.SSP_ERR_ARG
        assert srv.submit(t, y, dy) == 1


def test_destroy_with_requests_outstanding():
    freq, objs = _objects(8, n_freq=2000)
    srv = ssp.Server(freq)
    for t, y, dy in objs:
        srv.submit(t, y, dy)
    srv.close()                            # drops the queue, waits for the GPU
    srv.close()                            # idempotent in the binding


def test_request_arriving_during_a_batch_finishes_first():
    # Continuous batching: a short request submitted while a long batch is on
    # the GPU runs in another slot at once and finishes (and is reported)
    # first.  The long batch is one 65,535-point object in binary64 on a
    # 16-frequency grid: 16 CTAs for tens of milliseconds, which leaves SMs
    # free for the short one.
    import time
    g = np.random.default_rng(8)
    freq = synth.uniform_grid(0.05, 3.0, 16)
    tl = np.sort(g.uniform(0, 1000, 65535))
    long_obj = (tl, np.sin(tl) + g.normal(0, 0.1, tl.size), np.full(tl.size, 0.1))
    ts = np.sort(g.uniform(0, 100, 40))
    short_obj = (ts, np.cos(ts) + g.normal(0, 0.1, ts.size), np.full(ts.size, 0.1))
    with ssp.Server(freq, precision="fp64") as srv:
        a = srv.submit(*long_obj, "ss")
        time.sleep(0.005)                  # a's batch is on the GPU
        b = srv.submit(*short_obj, "sp")
        first = srv.next(wait_ms=60000)
        second = srv.next(wait_ms=60000)
        assert (first, second) == (b, a)
        pb, bb, _ = srv.poll(b)
        pa, ba, _ = srv.poll(a)
    ref_b, rb = ssp.ssp_periodogram(*short_obj, [ts.size], freq, variant="sp", precision="fp64")
    ref_a, ra = ssp.ssp_periodogram(*long_obj, [tl.size], freq, variant="ss", precision="fp64")
    np.testing.assert_array_equal(pb, ref_b[0])
    np.testing.assert_array_equal(pa, ref_a[0])
    assert (bb, ba) == (rb[0], ra[0])


def test_admission_waits_for_arena_room():
    # An arena of about 4,000 points per variant: requests beyond it wait on
    # the host until earlier ones finish, then run with the same results; an
    # object larger than the arena is refused at submission.
    freq, objs = _objects(24)
    with ssp.Server(freq, device_bytes=3 * 24 * 4000, slots=2) as srv:
        assert all(t.size <= 4000 for t, _, _ in objs)
        tks = [srv.submit(t, y, dy, "ss") for t, y, dy in objs]
        for tk, (t, y, dy) in zip(tks, objs):
            power, _, _ = srv.poll(tk, wait_ms=60000)
            ref, _ = ssp.ssp_periodogram(t, y, dy, [t.size], freq, variant="ss")
            np.testing.assert_array_equal(power, ref[0])
    with ssp.Server(freq, device_bytes=3 * 24 * 1000) as srv:
        k = np.arange(2000.0)
        with pytest.raises(ssp.SSPError) as ei:
            srv.submit(k * 0.37, np.sin(k), np.ones(k.size))
        assert ei.value.status == ssp.SSP_ERR_NOMEM
