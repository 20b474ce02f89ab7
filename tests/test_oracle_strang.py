"""Pins of the oracle's second-order (Strang) step P(dt/2) X(dt/2) Y(dt) X(dt/2)
P(dt/2), an extension: the paper names a split-step scheme without its order.

* Order: in real time the error against a fine-step solution falls about 4x
  when dt halves (about 2x for the first-order Lie step, which the same test
  measures, so a composition that is not symmetric fails).
* Real time conserves the norm.
* Without trap, interactions, Rabi coupling, rotation and SO coupling the
  pointwise substep is the identity, so one Strang step must equal
  X(dt/2) X(dt/2) Y(dt) exactly (the two axes commute then).
* Imaginary time reaches the same ground-state energy as the Lie step, to
  O(dt)."""
import numpy as np
import pytest

import oracle
from paper_2105_10517_gb300 import inputs

REAL, IMAG = oracle.REAL, oracle.IMAG


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def base(**kw):
    p = dict(nx=20, ny=18, xlen=8.0, ylen=7.2, dt=0.02, wx=1.0, wy=1.2, c0=8.0, c2=-1.5, omeg=0.4, so_type=1,
             gamma=0.6, rabi=0.3)
    p.update(kw)
    return p


def state(p, seed=3):
    return inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=seed, phase_noise=0.2)


def run(p, psi, dt, t, strang):
    q = dict(p, dt=dt)
    n = int(round(t / dt))
    f = oracle.propagate_strang if strang else oracle.propagate
    return f(q, psi, n, REAL)


def test_second_order_in_real_time():
    p = base()
    psi = state(p)
    t = 0.32
    ref = run(p, psi, 0.0025, t, True)
    e_s = [np.max(np.abs(run(p, psi, dt, t, True) - ref)) for dt in (0.04, 0.02)]
    e_l = [np.max(np.abs(run(p, psi, dt, t, False) - ref)) for dt in (0.04, 0.02)]
    assert 3.3 < e_s[0] / e_s[1] < 4.7
    assert 1.6 < e_l[0] / e_l[1] < 3.0
    assert e_s[1] < e_l[1]


def test_real_time_norm():
    p = base()
    psi = state(p)
    n0 = oracle.observables(p, psi)["norm_total"]
    out = oracle.propagate_strang(p, psi, 50, REAL)
    assert abs(oracle.observables(p, out)["norm_total"] - n0) <= 1e-12 * n0


def test_reduces_to_lie_when_the_pointwise_substep_is_a_global_phase():
    # P is the identity; with no rotation or SO coupling the x- and y-sweeps act
    # on separate axes and commute, so X(dt/2) Y(dt) X(dt/2) = X(dt/2) X(dt/2) Y(dt)
    p = base(wx=0.0, wy=0.0, c0=0.0, c2=0.0, rabi=0.0, omeg=0.0, gamma=0.0, so_type=0)
    psi = state(p)
    half = dict(p, dt=p["dt"] / 2)
    want = oracle.substep(half, oracle.substep(half, oracle.substep(p, psi, "Y", REAL), "X", REAL), "X", REAL)
    got = oracle.propagate_strang(p, psi, 1, REAL)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_imaginary_time_ground_state_agrees_with_lie():
    p = base(dt=0.01)
    psi = state(p)
    es = oracle.observables(p, oracle.propagate_strang(p, psi, 600, IMAG))["energy"]
    el = oracle.observables(p, oracle.propagate(p, psi, 600, IMAG))["energy"]
    assert abs(es - el) <= 5e-3 * abs(el)
