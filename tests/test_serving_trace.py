"""The seeded request trace of the parameter-sweep serving workload (CPU): the
same seed gives the same trace; parameters stay in their stated ranges; the
arrivals are Poisson at the stated rate; and every request of the 256-request
trace has a valid default tiling in both precisions (gp_plan_tiling, no device),
so none is refused for being outside the tabulated solver's range."""
import numpy as np

from paper_2105_10517_gb300 import gpspin, inputs


def test_trace_is_seeded_and_in_range():
    a = inputs.serving_trace(n=256, rate=20.0, seed=4)
    b = inputs.serving_trace(n=256, rate=20.0, seed=4)
    assert a == b
    assert inputs.serving_trace(n=256, rate=20.0, seed=5) != a
    t = np.array([r["arrival"] for r in a])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 20.0) < 0.2 / 20.0
    sizes = {r["params"]["nx"] for r in a}
    assert sizes == {128, 256, 384, 512}
    for r in a:
        p = r["params"]
        dx = p["xlen"] / p["nx"]
        assert p["nx"] == p["ny"] and p["xlen"] == p["ylen"] == 32.0
        assert np.isclose(p["dt"], 0.1 * dx * dx)
        assert 0 <= p["omeg"] <= 0.9 and 0 <= p["gamma"] <= 2 and 0 <= p["rabi"] <= 1
        assert 100 <= p["c0"] <= 800 and -20 <= p["c2"] <= 20 and p["so_type"] in (1, 2)
    assert {r["params"]["so_type"] for r in a} == {1, 2}


def test_every_request_has_a_tiling():
    for r in inputs.serving_trace(n=256, rate=20.0, seed=4):
        for prec in (gpspin.FP64, gpspin.FP32_MIXED):
            plan = gpspin.plan_tiling(dict(r["params"], precision=prec), gpspin.IMAG)
            for t in plan.values():
                assert t["threads"] <= 512 and t["smem"] <= 227 * 1024 and t["fixup"] < t["chunk"]
