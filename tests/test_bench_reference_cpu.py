"""The reference arm of bench.py (the FP64 oracle on the host cores) runs
without a GPU: one short invocation must print one JSON line with the keys the
benchmark contract asks of the reference arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_its_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Msite-steps/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["gpu_launches"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("quench1024: 1024x1024 real-time")


def test_cpu_baseline_has_single_thread_and_all_core_legs():
    """The CPU baseline times the oracle single-threaded and with its line loops
    on every host core; the all-cores leg is the reported value."""
    import bench
    from paper_2105_10517_gb300 import inputs
    p = inputs.physics(inputs.CONFIGS["small64"])
    b = bench.cpu_baseline(p, 0.3, 0)
    assert b["kind"] == "oracle" and b["legs"][0]["cores"] == 1
    assert b["cores"] == b["legs"][-1]["cores"] and b["value"] == b["legs"][-1]["value"]
    if bench.host_cores() > 1:
        assert len(b["legs"]) == 2 and b["legs"][1]["cores"] == bench.host_cores()
