"""The Omega-continuation of the Fig. S1 procedure (text after Fig. S1): an
Omega = 0 imaginary-time run from the centre-vortex guess, continued at
Omega = 0.3 from its state (`gp_set_params` rebuilds the tables), then real time
from the result with the real-time DT.  A short version of each stage on a small
grid against the oracle running the same sequence."""
import numpy as np
import pytest

from oracle import oracle
from paper_2105_10517_gb300 import gpspin, inputs, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpspin.build()
    gpspin.load()
    oracle.build()


@pytest.mark.parametrize("kind,so", [("ferro", 1), ("antiferro", 2)])
def test_continuation_stages_match_oracle(kind, so):
    cfg = workloads.FIGS1[kind]
    n, dx = 40, 0.25
    length = n * dx
    om = 0.3 if so == 1 else -0.3
    p = dict(nx=n, ny=n, xlen=length, ylen=length, dt=0.1 * dx * dx, c0=cfg["c0"] / 10, c2=cfg["c2"] / 10,
             omeg=0.0, so_type=so, gamma=0.5, rabi=0.0)
    stages = [(dict(p), 120, gpspin.IMAG), (dict(p, omeg=om), 120, gpspin.IMAG),
              (dict(p, omeg=om, dt=0.025 * dx * dx), 120, gpspin.REAL)]
    psi0 = inputs.winding_state(n, n, length, length, frac=(1 / 3, 1 / 3, 1 / 3), winding=cfg["winding"][so],
                                seed=3, phase_noise=1e-3)
    want = psi0
    with gpspin.Solver(p) as s:
        s.set_state(psi0)
        for q, steps, mode in stages:
            s.set_params(q)
            s.propagate(steps, mode)
            want = oracle.propagate(q, want, steps, mode)
            got = s.get_state()
            assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want))
