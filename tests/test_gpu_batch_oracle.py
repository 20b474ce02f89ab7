"""The batched and served forms against the FP64 oracle (not only against the
single-handle GPU path): every solve of a mixed batch -- FP64 and FP32-storage
policies, different grids and physics -- is compared element by element with
oracle.propagate of the same request.  FP64 solves agree to 1e-12 of max|psi|;
FP32-storage solves to the FP32 rounding accumulated over their steps."""
import numpy as np
import pytest

import oracle
from paper_2105_10517_gb300 import gpspin, inputs, serve

pytestmark = pytest.mark.gpu

CHECK = 20


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpspin.build()
    gpspin.load()


def req(n, **kw):
    box = 32.0 * n / 128
    p = dict(nx=n, ny=n, xlen=box, ylen=box, dt=0.1 * (32.0 / 128) ** 2, c0=200.0, c2=-5.0, omeg=0.5,
             so_type=1, gamma=0.6, rabi=0.2)
    p.update(kw)
    return p


def test_mixed_batch_matches_oracle():
    items = [
        (req(64, c2=12.0, so_type=2), dict(seed=3, cap=60)),
        (req(96), dict(seed=11, cap=120)),
        (req(80, omeg=0.8, rabi=0.0), dict(seed=5, cap=80, policy=gpspin.POLICY_FP32_REFINE)),
        (req(72, so_type=2, gamma=1.2), dict(seed=7, cap=40)),
        (req(128, c0=500.0), dict(seed=9, cap=60, policy=gpspin.POLICY_FP32_REFINE)),
    ]
    with gpspin.Batch(8 << 30, check_every=CHECK) as b:
        # FP32-policy solves stay in FP32 until the cap: no early hand-over
        ids = [b.submit(p, tol=1e-300, tol32=0.0, refine_steps=0, **kw) for p, kw in items]
        for _ in range(100):
            nr, nq = b.step()
            if nr == 0 and nq == 0:
                break
        got = [b.poll(i, fetch=True, release=True) for i in ids]
    for (p, kw), (st, steps, obs, psi) in zip(items, got):
        assert st == gpspin.REQ_DONE and steps == kw["cap"]
        psi0 = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=kw["seed"])
        want = oracle.propagate(p, psi0, steps, oracle.IMAG)
        eo = oracle.observables(p, want)["energy"]
        scale = np.max(np.abs(want))
        if kw.get("policy", gpspin.POLICY_FP64) == gpspin.POLICY_FP64:
            assert np.max(np.abs(psi - want)) <= 1e-12 * scale
            assert abs(obs["energy"] - eo) <= 1e-12 * abs(eo)
        else:
            # complex64 storage: a few FP32 roundings per step, damped in imaginary time
            assert np.max(np.abs(psi - want)) <= 1e-5 * scale
            assert abs(obs["energy"] - eo) <= 1e-5 * abs(eo)


def test_served_request_matches_oracle():
    """One request through the serving loop (Poisson trace of length one, FP64
    policy): its energy after the capped solve equals the oracle's."""
    p = req(64, c0=150.0, omeg=0.3)
    trace = [dict(arrival=0.0, params=p, seed=21)]
    summary, rec = serve.serve_batched(trace, policy=gpspin.POLICY_FP64, max_bytes=4 << 30, check_every=CHECK,
                                       tol=1e-300, cap=100)
    assert summary["solves"] == 1 and rec[0]["steps"] == 100
    psi0 = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=21)
    eo = oracle.observables(p, oracle.propagate(p, psi0, 100, oracle.IMAG))["energy"]
    assert abs(rec[0]["energy"] - eo) <= 1e-12 * abs(eo)
