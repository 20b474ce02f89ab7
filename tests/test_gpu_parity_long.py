"""The parity contract of the FP64 path over long runs and at full size: after
1000 steps the CUDA path (through the C ABI) agrees with the FP64 oracle to
max|dpsi| <= 1e-10 and |dE/E| <= 1e-12, at 128^2 and 256^2, in imaginary and
in real time with every term of the step switched on (rotation, Rashba or
Dresselhaus SO coupling, Rabi coupling, both interaction signs).

The two sides differ only in rounding order (3x3-block Thomas in the original
spin basis against scalar channel solves; divisions against reciprocals; libm
against short polynomials), so what is compared is accumulated rounding.
"""
import numpy as np
import pytest

import oracle
from paper_2105_10517_gb300 import gpspin, inputs

pytestmark = pytest.mark.gpu

IMAG, REAL = gpspin.IMAG, gpspin.REAL


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpspin.build()
    gpspin.load()


def case(name):
    """Shrunk copies of the workloads: the physics of the 512^2 vortex-lattice run
    (imaginary time) and of the 1024^2 Omega-quench run (real time after the
    quench, Omega = 0.9), on the same boxes with fewer points."""
    if name == "imag128":
        return dict(nx=128, ny=128, xlen=16.0, ylen=16.0, dt=0.002, c0=500.0, c2=-10.0, omeg=0.8, so_type=1,
                    gamma=1.0, rabi=0.3), IMAG
    if name == "imag256":
        return dict(nx=256, ny=256, xlen=32.0, ylen=32.0, dt=0.001, c0=500.0, c2=-10.0, omeg=0.8, so_type=1,
                    gamma=1.0, rabi=0.0), IMAG
    if name == "real128":
        return dict(nx=128, ny=128, xlen=20.0, ylen=20.0, dt=0.0005, c0=800.0, c2=15.0, omeg=0.9, so_type=2,
                    gamma=0.75, rabi=0.5), REAL
    if name == "real256":
        return dict(nx=256, ny=256, xlen=40.0, ylen=40.0, dt=0.0005, c0=800.0, c2=15.0, omeg=0.9, so_type=2,
                    gamma=0.75, rabi=0.5), REAL
    raise KeyError(name)


@pytest.mark.parametrize("name", ["imag128", "imag256", "real128", "real256"])
def test_thousand_step_parity(name):
    p, mode = case(name)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=17)
    want = oracle.propagate(p, psi, 1000, mode)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.propagate(1000, mode)
        got = s.get_state()
        obs = s.observables()
    o = oracle.observables(p, want)
    assert np.max(np.abs(got - want)) <= 1e-10
    assert abs(obs["energy"] - o["energy"]) <= 1e-12 * abs(o["energy"])
    if mode == REAL:
        assert abs(obs["norm_total"] - 1.0) <= 1e-12


@pytest.mark.parametrize("mode", [IMAG, REAL])
def test_full_size_1024_autotuned(mode):
    """The 1024^2 workload in the launch configuration bench.py times (autotuned
    tiling): three steps compared everywhere with the oracle."""
    c = inputs.CONFIGS["quench1024"]
    p = dict(inputs.physics(c), omeg=0.9)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=c["seed"])
    want = oracle.propagate(p, psi, 3, mode)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.autotune(mode)
        s.propagate(3, mode)
        got = s.get_state()
        e = s.observables()["energy"]
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    assert abs(e - oracle.observables(p, want)["energy"]) <= 1e-12 * abs(e)


@pytest.mark.parametrize("name", ["imag256", "real256"])
def test_thousand_step_parity_register_solve(name):
    """The 1000-step contract with the register-resident complex128 solve in both
    passes (the solve the autotuner picks for the 1024^2 y-pass), over 2-CTA
    clusters: the chunk carries cross distributed shared memory every step."""
    p, mode = case(name)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=19)
    want = oracle.propagate(p, psi, 1000, mode)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        for d in (0, 1):
            s.set_tiling(d, cluster=2, lines_per_cta=2, chunk=32, mode=mode, register_solve=True)
        t = s.tiling(mode)
        assert t["xpass"]["register_solve"] and t["ypass"]["register_solve"] and t["ypass"]["cluster"] == 2
        s.propagate(1000, mode)
        got = s.get_state()
        obs = s.observables()
    o = oracle.observables(p, want)
    assert np.max(np.abs(got - want)) <= 1e-10
    assert abs(obs["energy"] - o["energy"]) <= 1e-12 * abs(o["energy"])
