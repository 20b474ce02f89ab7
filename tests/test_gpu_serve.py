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


def test_bench_serving_line_reports_the_accuracy_bar():
    """bench.py --serve on a short trace: the line's value counts only results
    within |dE/E| <= 1e-6 of the plain FP64 result of the same request, and the
    latencies are split by converged and capped solves."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--serve", "--requests", "6", "--rate", "50", "--cap", "300"],
                       cwd=root, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    bar = d["at_1e-6"]
    assert d["value"] == bar[d["value_path"]]["solves_per_s"] > 0
    assert bar["plain_fp64_one_at_a_time"]["solves"] == 6
    assert bar["batched_fp64"]["solves"] == 6  # batched FP64 equals plain FP64 to rounding
    for k in ("batched_mixed", "batched_fp64", "plain_fp64_one_at_a_time"):
        assert {"p50_converged_s", "p99_capped_s", "capped", "converged"} <= set(d[k])
