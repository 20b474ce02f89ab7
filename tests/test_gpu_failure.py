"""Failure detection on the GPU without a GPU fault: a bounded device-side wait
that runs out is reported on the host as GP_ERR_TIMEOUT, and the handle and the
CUDA context stay usable afterwards."""
import numpy as np
import pytest

import oracle
from paper_2105_10517_gb300 import gpspin, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpspin.build()
    gpspin.load()


def test_bounded_wait_times_out_and_handle_stays_usable():
    p = dict(nx=48, ny=40, xlen=9.6, ylen=8.0, dt=0.004, c0=60.0, c2=-6.0, omeg=0.5, so_type=1, gamma=0.5,
             rabi=0.2)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=4)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        with pytest.raises(gpspin.GPError) as ei:
            s.check_wait_timeout(64)
        assert ei.value.status == 7  # GP_ERR_TIMEOUT
        # the state is untouched and the handle propagates normally
        s.propagate(5, gpspin.IMAG)
        got = s.get_state()
    want = oracle.propagate(p, psi, 5, oracle.IMAG)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
