"""The serving loop over a short seeded trace: every request completes, the
records and summary are consistent, and batched FP64 results equal the plain
one-at-a-time FP64 results to rounding (the batched and single-instance kernels
are separate instantiations of the same arithmetic; the compiler may fuse
multiply-adds differently in each, so the results agree to ~1e-15, not bitwise)."""
import pytest

from paper_2105_10517_gb300 import gpspin, inputs, serve

pytestmark = pytest.mark.gpu


def test_serving_trace_batched_and_one_at_a_time():
    gpspin.build()
    trace = inputs.serving_trace(n=6, rate=50.0, seed=4, sizes=(64, 96))
    sb, rb = serve.serve_batched(trace, policy=gpspin.POLICY_FP64, max_bytes=1 << 30, cap=300, tol=1e-9)
    sp, rp = serve.serve_one_at_a_time(trace, cap=300, tol=1e-9)
    assert sb["solves"] == sp["solves"] == 6 and sb["failed"] == 0
    assert sb["p50_s"] <= sb["p99_s"] and sp["p50_s"] <= sp["p99_s"]
    eb = {r["arrival"]: r for r in rb}
    for r in rp:
        q = eb[r["arrival"]]
        assert q["steps"] == r["steps"]
        assert abs(q["energy"] - r["energy"]) <= 1e-13 * abs(r["energy"])
