"""Request-serving loop for parameter sweeps of the imaginary-time solve.

Requests arrive over wall-clock time (a trace from inputs.serving_trace); the
loop submits each one to a gp_batch as it arrives and keeps calling
gp_batch_step, which admits requests as memory frees up, advances every running
solve together and retires converged ones (continuous batching).  A solve is
done when its energy changes by less than `tol` between checks `check_every`
steps apart, or at `cap` steps.  The baseline serves the same trace one request
at a time with a plain FP64 handle.  Both report solves/s and the p50/p99 time
from arrival to converged state; the batched loop also reports the queue depth
and running count over its ticks.
"""
import time

import numpy as np

from . import gpspin


def _pct(v, q):
    return float(np.percentile(np.array(v), q)) if len(v) else None


def _summary(records, makespan):
    done = [r for r in records if r["state"] == gpspin.REQ_DONE]
    conv = [r["latency"] for r in done if r["steps"] < r["cap"]]
    cap = [r["latency"] for r in done if r["steps"] >= r["cap"]]
    lat = [r["latency"] for r in done]
    return dict(solves=len(done), makespan_s=makespan, solves_per_s=len(done) / makespan,
                p50_s=_pct(lat, 50), p99_s=_pct(lat, 99),
                converged=len(conv), p50_converged_s=_pct(conv, 50), p99_converged_s=_pct(conv, 99),
                capped=len(cap), p50_capped_s=_pct(cap, 50), p99_capped_s=_pct(cap, 99),
                failed=sum(1 for r in records if r["state"] == gpspin.REQ_FAILED),
                cancelled=sum(1 for r in records if r["state"] == gpspin.REQ_CANCELLED))


def serve_batched(trace, policy=gpspin.POLICY_FP32_REFINE, max_bytes=64 << 30, check_every=100, tol=1e-9,
                  tol32=1e-7, cap=20000, refine_steps=2000, stream=None, deadline_s=None, max_running_sites=0):
    """Continuous batching over the trace; returns (summary, per-request records).
    With deadline_s, a request still queued or running that long after its
    arrival is cancelled (its memory is released for the others) and recorded
    as REQ_CANCELLED."""
    pending = sorted(trace, key=lambda r: r["arrival"])
    records, live = [], {}
    depth = []  # (queued, running) after every tick
    with gpspin.Batch(max_bytes, check_every=check_every, stream=stream) as b:
        b.set_running_limit(max_running_sites)
        t0 = time.perf_counter()
        k = 0
        while k < len(pending) or live:
            now = time.perf_counter() - t0
            while k < len(pending) and pending[k]["arrival"] <= now:
                rq = pending[k]
                rid = b.submit(rq["params"], seed=rq["seed"], tol=tol, tol32=tol32, cap=cap, policy=policy,
                               refine_steps=refine_steps)
                live[rid] = rq
                k += 1
            if not live:
                time.sleep(max(0.0, pending[k]["arrival"] - (time.perf_counter() - t0)))
                continue
            depth.append(b.step()[::-1])
            done_t = time.perf_counter() - t0
            for rid in list(live):
                st, steps, obs, _ = b.poll(rid)
                if (deadline_s is not None and st in (gpspin.REQ_QUEUED, gpspin.REQ_RUNNING)
                        and done_t - live[rid]["arrival"] > deadline_s):
                    b.cancel(rid)
                    st = gpspin.REQ_CANCELLED
                if st in (gpspin.REQ_DONE, gpspin.REQ_FAILED, gpspin.REQ_CANCELLED):
                    rq = live.pop(rid)
                    b.poll(rid, release=True)
                    records.append(dict(arrival=rq["arrival"], done=done_t, latency=done_t - rq["arrival"],
                                        steps=steps, cap=cap, state=st, energy=obs["energy"], nx=rq["params"]["nx"]))
        makespan = time.perf_counter() - t0
    summary = _summary(records, makespan)
    if depth:
        q = np.array(depth, dtype=float)
        summary.update(ticks=len(depth), queue_depth_max=int(q[:, 0].max()), queue_depth_mean=float(q[:, 0].mean()),
                       running_max=int(q[:, 1].max()), running_mean=float(q[:, 1].mean()))
    return summary, records


def serve_one_at_a_time(trace, check_every=100, tol=1e-9, cap=20000, stream=None):
    """The plain FP64 path: requests in arrival order, one handle at a time."""
    pending = sorted(trace, key=lambda r: r["arrival"])
    records = []
    t0 = time.perf_counter()
    for rq in pending:
        wait = rq["arrival"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        p = dict(rq["params"], precision=gpspin.FP64)
        with gpspin.Solver(p, stream=stream) as s:
            s.init_gaussian((0.25, 0.5, 0.25), seed=rq["seed"], phase_noise=1e-3)
            steps, e_last = 0, None
            while True:
                s.propagate(check_every, gpspin.IMAG)
                steps += check_every
                e = s.observables()["energy"]
                if (e_last is not None and abs(e - e_last) < tol) or steps >= cap:
                    break
                e_last = e
        done_t = time.perf_counter() - t0
        records.append(dict(arrival=rq["arrival"], done=done_t, latency=done_t - rq["arrival"], steps=steps,
                            cap=cap, state=gpspin.REQ_DONE, energy=e, nx=rq["params"]["nx"]))
    return _summary(records, time.perf_counter() - t0), records
