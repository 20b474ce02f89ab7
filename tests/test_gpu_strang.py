"""Second-order (Strang) steps on the GPU, an extension with no counterpart in
the paper: P(dt/2) X(dt/2) Y(dt) X(dt/2) P(dt/2) [+ renormalisation in imaginary
time] against the oracle's Strang step, on a ragged grid and on lines long
enough to span clusters of CTAs."""
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
    oracle.build()


def params(**kw):
    p = dict(nx=72, ny=45, xlen=14.4, ylen=9.9, dt=0.004, wx=1.0, wy=1.2, c0=60.0, c2=-6.0, omeg=0.7,
             so_type=1, gamma=0.8, rabi=0.35)
    p.update(kw)
    return p


def start(p, seed):
    return inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=seed, phase_noise=0.3) \
        + inputs.random_state(p["nx"], p["ny"], seed=seed + 100, scale=0.05)


@pytest.mark.parametrize("mode", [IMAG, REAL])
@pytest.mark.parametrize("so_type", [1, 2])
def test_strang_matches_oracle(mode, so_type):
    p = params(so_type=so_type)
    psi = start(p, 21)
    want = oracle.propagate_strang(p, psi, 4, mode)
    with gpspin.Solver(p) as s:
        s.set_splitting(gpspin.SPLIT_STRANG)
        s.set_state(psi)
        s.propagate(4, mode)
        got = s.get_state()
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
        # the one-call host path follows the setting
        assert np.array_equal(s.propagate_host(psi, 4, mode), got)


def test_strang_on_clustered_lines():
    p = params(nx=320, ny=288, xlen=0.05 * 320, ylen=0.05 * 288, dt=0.0005)
    psi = start(p, 23)
    want = oracle.propagate_strang(p, psi, 2, IMAG)
    with gpspin.Solver(p) as s:
        assert s.tiling(IMAG)["xpass"]["cluster"] > 1
        s.set_splitting(gpspin.SPLIT_STRANG)
        s.set_state(psi)
        s.propagate(2, IMAG)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_strang_differs_from_lie_and_switches_back():
    p = params()
    psi = start(p, 25)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.set_splitting(gpspin.SPLIT_STRANG)
        s.propagate(3, REAL)
        strang = s.get_state()
        s.set_splitting(gpspin.SPLIT_LIE)
        s.set_state(psi)
        s.propagate(3, REAL)
        lie = s.get_state()
    assert np.max(np.abs(strang - lie)) > 1e-6 * np.max(np.abs(lie))
    assert np.max(np.abs(lie - oracle.propagate(p, psi, 3, REAL))) <= 1e-12 * np.max(np.abs(lie))


def test_strang_unsupported_for_complex64_storage():
    with gpspin.Solver(params(precision=gpspin.FP32_MIXED)) as s:
        with pytest.raises(gpspin.GPError):
            s.set_splitting(gpspin.SPLIT_STRANG)
