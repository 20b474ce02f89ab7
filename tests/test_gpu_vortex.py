"""Initial states with built-in centre vortices and the qualitative statement
about SO-coupled, non-rotating ground states (text after Fig. S1): centre
vortices of type (-+1, 0, +-1) for the antiferromagnetic and (0, +-1, +-2) for
the ferromagnetic condensate, upper sign Rashba, lower sign Dresselhaus.
Qualitative only: the test checks that imaginary time keeps those charges."""
import numpy as np
import pytest

from paper_2105_10517_gb300 import diagnostics, gpspin, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpspin.build()
    gpspin.load()


def test_init_winding_matches_input_generator():
    p = dict(nx=96, ny=80, xlen=12.0, ylen=10.0, dt=0.01)
    w = (-1, 2, 1)
    want = inputs.winding_state(96, 80, 12.0, 10.0, frac=(0.3, 0.4, 0.3), winding=w, seed=9, phase_noise=1e-3)
    with gpspin.Solver(p) as s:
        s.init_winding((0.3, 0.4, 0.3), winding=w, seed=9, phase_noise=1e-3)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(want))


@pytest.mark.parametrize("case", [
    ("antiferro", 1, (-1, 0, 1)), ("antiferro", 2, (1, 0, -1)),
    ("ferro", 1, (0, 1, 2)), ("ferro", 2, (0, -1, -2)),
])
def test_so_coupled_ground_state_keeps_centre_vortices(case):
    kind, so, w = case
    c0, c2 = (482.0, 15.0) if kind == "antiferro" else (669.0, -3.1)
    n, length = 128, 20.0
    dx = length / n
    p = dict(nx=n, ny=n, xlen=length, ylen=length, dt=0.1 * dx * dx, c0=c0, c2=c2, omeg=0.0, so_type=so,
             gamma=0.5, rabi=0.0)
    with gpspin.Solver(p) as s:
        s.init_winding((1 / 3, 1 / 3, 1 / 3), winding=w, seed=3, phase_noise=1e-3)
        s.propagate(4000, gpspin.IMAG)
        psi = s.get_state()
    x, y = inputs.grid(n, n, length, length)
    got = tuple(diagnostics.central_winding(psi[c], x, y, 1.5) for c in range(3))
    assert got == w
