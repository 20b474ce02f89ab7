"""gp_propagate_host: host state in, host state out in one call.  It must give
exactly what gp_set_state + gp_propagate + gp_get_state give, whether the first
x-pass reads the caller's buffer directly (pinned or device-readable pageable
memory, complex128 handle) or the call falls back to the copies."""
import numpy as np
import pytest
import torch

from paper_2105_10517_gb300 import gpspin, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpspin.build()
    gpspin.load()


def params(**kw):
    p = dict(nx=96, ny=70, xlen=19.2, ylen=14.0, dt=0.003, wx=1.0, wy=1.1, c0=80.0, c2=-4.0, omeg=0.6,
             so_type=1, gamma=0.7, rabi=0.3)
    p.update(kw)
    return p


def reference(p, psi, n, mode):
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.propagate(n, mode)
        return s.get_state()


@pytest.mark.parametrize("mode", [gpspin.IMAG, gpspin.REAL])
@pytest.mark.parametrize("buffers", ["pinned", "pageable"])
def test_matches_the_three_calls(mode, buffers):
    p = params()
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=11, phase_noise=0.1)
    want = reference(p, psi, 5, mode)
    if buffers == "pinned":
        hin = torch.from_numpy(psi.copy()).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
    else:
        hin, hout = psi.copy(), np.empty_like(psi)
    with gpspin.Solver(p) as s:
        for _ in range(2):  # two calls in a row on one handle
            got = s.propagate_host(hin, 5, mode, out=hout)
            got = got.numpy() if hasattr(got, "numpy") else got
            assert np.array_equal(got, want)
        assert np.array_equal(s.get_state(), want)  # the handle holds the new state


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("in_place", [False, True])
def test_real_time_calls_of_few_steps(n, in_place):
    """Real-time calls of one, two and three steps with pinned buffers (the first
    x-pass reads the input buffer, one kernel writes the output): bitwise the
    three-call result and the handle's state, also in place."""
    p = params(so_type=2, rabi=0.5)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=23, phase_noise=0.1)
    want = reference(p, psi, n, gpspin.REAL)
    hin = torch.from_numpy(psi.copy()).pin_memory()
    hout = hin if in_place else torch.empty_like(hin).pin_memory()
    with gpspin.Solver(p) as s:
        s.propagate_host(hin, n, gpspin.REAL, out=hout)
        assert np.array_equal(hout.numpy(), want)
        assert np.array_equal(s.get_state(), want)
        assert s.observables()["steps"] == n


def test_in_place_and_zero_steps():
    p = params(so_type=2, omeg=-0.4)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=5, phase_noise=0.1)
    want = reference(p, psi, 3, gpspin.IMAG)
    buf = torch.from_numpy(psi.copy()).pin_memory()
    with gpspin.Solver(p) as s:
        s.propagate_host(buf, 3, gpspin.IMAG, out=buf)
        assert np.array_equal(buf.numpy(), want)
        out = s.propagate_host(psi, 0, gpspin.IMAG)
        assert np.array_equal(out, psi)


def test_complex64_handle_and_magnetisation_constraint_fall_back_or_match():
    p = params(precision=gpspin.FP32_MIXED)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=3, phase_noise=0.1)
    want = reference(p, psi, 4, gpspin.IMAG)
    with gpspin.Solver(p) as s:
        assert np.array_equal(s.propagate_host(psi, 4, gpspin.IMAG), want)
    q = params(gamma=0.0, rabi=0.0)
    with gpspin.Solver(q) as s:
        s.set_magnetization(0.1)
        s.set_state(psi)
        s.propagate(4, gpspin.IMAG)
        want_m = s.get_state()
    with gpspin.Solver(q) as s:
        s.set_magnetization(0.1)
        assert np.array_equal(s.propagate_host(psi, 4, gpspin.IMAG), want_m)
