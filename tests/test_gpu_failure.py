"""Failure detection on the GPU without a GPU fault: a bounded device-side wait
that runs out is reported on the host as GP_ERR_TIMEOUT, and the handle and the
CUDA context stay usable afterwards."""
import numpy as np
import pytest

import oracle
from paper_2105_10517_gb300 import gpspin, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpspin.build()
    gpspin.load()


def test_bounded_wait_times_out_and_handle_stays_usable():
    p = dict(nx=48, ny=40, xlen=9.6, ylen=8.0, dt=0.004, c0=60.0, c2=-6.0, omeg=0.5, so_type=1, gamma=0.5,
             rabi=0.2)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=4)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        with pytest.raises(gpspin.GPError) as ei:
            s.check_wait_timeout(64)
        assert ei.value.status == 7  # GP_ERR_TIMEOUT
        # the state is untouched and the handle propagates normally
        s.propagate(5, gpspin.IMAG)
        got = s.get_state()
    want = oracle.propagate(p, psi, 5, oracle.IMAG)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def small(n=48, **kw):
    p = dict(nx=n, ny=n, xlen=0.2 * n, ylen=0.2 * n, dt=0.004, c0=60.0, c2=-6.0, omeg=0.5, so_type=1, gamma=0.5,
             rabi=0.2)
    p.update(kw)
    return p


def test_injected_allocation_failure_is_reported_and_recovers():
    gpspin.inject_alloc_failure(0)
    try:
        with pytest.raises(gpspin.GPError) as ei:
            gpspin.Solver(small())
        assert ei.value.status == 2  # GP_ERR_OOM, the partial allocations released
    finally:
        gpspin.inject_alloc_failure(-1)
    with gpspin.Solver(small()) as s:  # the next creation succeeds
        s.init_gaussian(seed=3)
        s.propagate(3, gpspin.IMAG)


def test_batch_admission_reports_oom_with_nothing_running():
    with gpspin.Batch(4 << 30, check_every=10) as b:
        rid = b.submit(small(), seed=1, tol=1e-300, cap=20)
        gpspin.inject_alloc_failure(0)  # the handle's first allocation fails
        try:
            b.step()
        finally:
            gpspin.inject_alloc_failure(-1)
        assert b.poll(rid)[0] == gpspin.REQ_FAILED and b.error(rid) == 2
        ok = b.submit(small(), seed=1, tol=1e-300, cap=20)
        for _ in range(5):
            b.step()
        assert b.poll(ok)[0] == gpspin.REQ_DONE


def test_cancel_queued_and_running_requests():
    p = small(64)
    one = gpspin.request_bytes(p)
    with gpspin.Batch(int(1.5 * one), check_every=10) as b:
        ids = [b.submit(p, seed=s, tol=1e-300, cap=50) for s in range(3)]
        nr, nq = b.step()
        assert (nr, nq) == (1, 2)
        b.cancel(ids[0])  # running: its memory is released at once
        b.cancel(ids[2])  # queued: leaves the queue
        assert b.poll(ids[0])[0] == gpspin.REQ_CANCELLED and b.poll(ids[2])[0] == gpspin.REQ_CANCELLED
        nr, nq = b.step()  # the freed memory admits the remaining request
        assert (nr, nq) == (1, 0)
        for _ in range(10):
            b.step()
        assert b.poll(ids[1])[0] == gpspin.REQ_DONE
        b.poll(ids[0], release=True)
        with pytest.raises(gpspin.GPError):
            b.cancel(ids[0])  # forgotten: unknown id


def test_queue_limit_refuses_submissions():
    p = small(64)
    with gpspin.Batch(int(1.5 * gpspin.request_bytes(p)), check_every=10) as b:
        b.set_queue_limit(2)
        b.submit(p, seed=1, tol=1e-300, cap=20)
        b.submit(p, seed=2, tol=1e-300, cap=20)
        with pytest.raises(gpspin.GPError) as ei:
            b.submit(p, seed=3, tol=1e-300, cap=20)
        assert ei.value.status == 8  # GP_ERR_QUEUE_FULL
        b.step()  # one admitted, one queued: room for one more
        b.submit(p, seed=3, tol=1e-300, cap=20)


def test_serving_deadline_cancels_late_requests():
    from paper_2105_10517_gb300 import serve
    trace = [dict(arrival=0.0, params=small(64), seed=s) for s in range(3)]
    summary, rec = serve.serve_batched(trace, policy=gpspin.POLICY_FP64, max_bytes=4 << 30, check_every=10,
                                       tol=1e-300, cap=10 ** 8, deadline_s=0.5)
    assert summary["cancelled"] == 3 and summary["solves"] == 0
    assert all(r["state"] == gpspin.REQ_CANCELLED for r in rec)
