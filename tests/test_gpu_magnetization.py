"""Magnetisation-constrained imaginary time on the GPU against the oracle
(both conditions below Eq. S.5, gamma = R = 0)."""
import numpy as np
import pytest

import oracle
from paper_2105_10517_gb300 import gpspin, inputs

pytestmark = pytest.mark.gpu


def params(**kw):
    p = dict(nx=72, ny=45, xlen=14.4, ylen=9.9, dt=0.004, c0=60.0, c2=-6.0, omeg=0.7, so_type=0, gamma=0.0,
             rabi=0.0)
    p.update(kw)
    return p


@pytest.mark.parametrize("m", [0.3, -0.15])
def test_constrained_imaginary_time_matches_oracle(m):
    gpspin.build()
    p = params()
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], frac=(0.5, 0.3, 0.2), seed=6)
    want = oracle.propagate_m(p, psi, 30, m)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.set_magnetization(m)
        s.propagate(30, gpspin.IMAG)
        got = s.get_state()
        o = s.observables()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    assert abs(o["norm_total"] - 1) <= 1e-13 and abs(o["magnetization"] - m) <= 1e-13


def test_constrained_fp32_storage_keeps_both_conditions():
    p = params(precision=gpspin.FP32_MIXED)
    with gpspin.Solver(p) as s:
        s.init_gaussian((0.5, 0.3, 0.2), seed=2)
        s.set_magnetization(0.2)
        s.propagate(40, gpspin.IMAG)
        o = s.observables()
    assert abs(o["norm_total"] - 1) <= 2e-6 and abs(o["magnetization"] - 0.2) <= 2e-6


def test_constraint_needs_gamma_and_rabi_zero():
    with gpspin.Solver(params(so_type=1, gamma=0.5)) as s:
        with pytest.raises(gpspin.GPError):
            s.set_magnetization(0.1)
    with gpspin.Solver(params(rabi=0.2)) as s:
        with pytest.raises(gpspin.GPError):
            s.set_magnetization(0.1)
