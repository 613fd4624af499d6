"""Failure paths, reached from the host without faulting a GPU (fault
injection is test-only: ssp_test_fault with SSP_TESTING=1).

- A device allocation that fails returns SSP_ERR_NOMEM and leaves nothing
  behind: the next call gives the results of a clean run, bit for bit.
- A served batch that outlives the server's bounded wait (stall_ms) ends its
  requests with SSP_ERR_TIMEOUT while the server keeps serving; both a real
  expiry (a wait of microseconds) and an injected one are covered.
- A served batch whose allocation fails ends its requests with SSP_ERR_NOMEM.
- A served request whose upload fails ends with SSP_ERR_CUDA and never joins
  a batch, even one formed later from requests on both sides of it.
"""
import numpy as np
import pytest

from paper_2111_07396_gb300 import build as ssp_build
from paper_2111_07396_gb300 import ssp, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ssp_build.build()
    ssp.lib()


@pytest.fixture
def testing(monkeypatch):
    monkeypatch.setenv("SSP_TESTING", "1")
    yield
    ssp.ssp_test_fault(ssp.SSP_FAULT_ALLOC, 0)
    ssp.ssp_test_fault(ssp.SSP_FAULT_STALL, 0)
    ssp.ssp_test_fault(ssp.SSP_FAULT_UPLOAD, 0)


def _cat():
    return synth.config3(n_objects=6, n_freq=200)


def test_allocation_failure_is_nomem_and_leaves_a_clean_state(testing):
    import torch
    cat = _cat()
    ref, ref_best = ssp.ssp_periodogram(cat.t, cat.y, cat.dy, cat.n_per_object, cat.freq)
    # host entry point: its first allocation (the frequency grid) fails
    ssp.ssp_test_fault(ssp.SSP_FAULT_ALLOC, 1)
    with pytest.raises(ssp.SSPError) as ei:
        ssp.ssp_periodogram(cat.t, cat.y, cat.dy, cat.n_per_object, cat.freq)
    assert ei.value.status == ssp.SSP_ERR_NOMEM
    got, best = ssp.ssp_periodogram(cat.t, cat.y, cat.dy, cat.n_per_object, cat.freq)
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(best, ref_best)
    # device entry point: its workspace allocation fails, nothing is enqueued
    put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    t, y, dy, fq = put(cat.t), put(cat.y), put(cat.dy), put(cat.freq)
    pw = torch.full((cat.n_objects, cat.freq.size), -7.0, dtype=torch.float32, device="cuda")
    bp = torch.empty(cat.n_objects, dtype=torch.float64, device="cuda")
    ssp.ssp_test_fault(ssp.SSP_FAULT_ALLOC, 1)
    with pytest.raises(ssp.SSPError) as ei:
        ssp.ssp_periodogram_device(t, y, dy, cat.n_per_object, fq, pw, bp)
    assert ei.value.status == ssp.SSP_ERR_NOMEM
    torch.cuda.synchronize()
    assert np.all(pw.cpu().numpy() == -7.0)   # no kernel ran
    ssp.ssp_periodogram_device(t, y, dy, cat.n_per_object, fq, pw, bp)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(pw.cpu().numpy(), ref)


def test_server_batch_allocation_failure_then_recovery(testing):
    cat = _cat()
    ref, ref_best = ssp.ssp_periodogram(*cat.obj(0), [cat.n_per_object[0]], cat.freq)
    with ssp.Server(cat.freq) as srv:
        ssp.ssp_test_fault(ssp.SSP_FAULT_ALLOC, 1)
        tk = srv.submit(*cat.obj(0))
        with pytest.raises(ssp.SSPError) as ei:
            srv.poll(tk, wait_ms=60000)
        assert ei.value.status == ssp.SSP_ERR_NOMEM
        pw, best, _ = srv.poll(srv.submit(*cat.obj(0)), wait_ms=60000)
        np.testing.assert_array_equal(pw, ref[0])
        assert best == ref_best[0]


def test_server_injected_stall_times_out_then_serves(testing):
    cat = _cat()
    ref, _ = ssp.ssp_periodogram(*cat.obj(1), [cat.n_per_object[1]], cat.freq)
    with ssp.Server(cat.freq) as srv:
        ssp.ssp_test_fault(ssp.SSP_FAULT_STALL, 1)
        tk = srv.submit(*cat.obj(1))
        with pytest.raises(ssp.SSPError) as ei:
            srv.poll(tk, wait_ms=60000)
        assert ei.value.status == ssp.SSP_ERR_TIMEOUT
        pw, _, _ = srv.poll(srv.submit(*cat.obj(1)), wait_ms=60000)
        np.testing.assert_array_equal(pw, ref[0])


def test_server_failed_upload_is_answered_and_never_batched(testing):
    # With a two-second batching window, request B is admitted and waits for
    # company; request A's upload then fails (injected) and C follows.  A is
    # answered with SSP_ERR_CUDA at once and sits in the ring between B and
    # C: the batches formed at the end of the window must leave it out.  B
    # and C are collected first, so a batch that had taken A in would have
    # overwritten its answer before A is polled.
    import time
    cat = _cat()
    refs = [ssp.ssp_periodogram(*cat.obj(k), [cat.n_per_object[k]], cat.freq)[0][0]
            for k in range(3)]
    with ssp.Server(cat.freq, max_wait_ms=2000.0) as srv:
        tb = srv.submit(*cat.obj(0))
        time.sleep(0.5)                          # B admitted (uploaded), batch window open
        ssp.ssp_test_fault(ssp.SSP_FAULT_UPLOAD, 1)
        ta = srv.submit(*cat.obj(1))
        tc = srv.submit(*cat.obj(2))
        for tk, ref in ((tb, refs[0]), (tc, refs[2])):
            pw, _, _ = srv.poll(tk, wait_ms=60000)
            np.testing.assert_array_equal(pw, ref)
        with pytest.raises(ssp.SSPError) as ei:
            srv.poll(ta, wait_ms=60000)
        assert ei.value.status == ssp.SSP_ERR_CUDA
        # the ring space is reused: the server keeps serving
        pw, _, _ = srv.poll(srv.submit(*cat.obj(1)), wait_ms=60000)
        np.testing.assert_array_equal(pw, refs[1])


def test_server_bounded_wait_expires_on_a_real_batch():
    # A wait limit of 10 microseconds from launch: one batch of 3,000 points x
    # 20,000 frequencies takes milliseconds, so the watchdog fires on the
    # GPU's real timing.  (A batch found complete when the worker first looks
    # at it counts as finished in time, whatever the clock says: its results
    # are valid.)  The server shuts down cleanly, and a server with the
    # default limit serves the same object.
    cat = synth.config2(n_freq=20_000)
    with ssp.Server(cat.freq, stall_ms=0.01) as srv:
        with pytest.raises(ssp.SSPError) as ei:
            srv.poll(srv.submit(*cat.obj(0), variant="ss"), wait_ms=60000)
        assert ei.value.status == ssp.SSP_ERR_TIMEOUT
    with ssp.Server(cat.freq) as srv:
        pw, best, _ = srv.poll(srv.submit(*cat.obj(0), variant="ss"), wait_ms=60000)
        assert np.all(np.isfinite(pw)) and best > 0.0
