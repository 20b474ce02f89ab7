"""Checkpoint and resume: a run interrupted by gp_checkpoint_save and continued
from gp_checkpoint_load in a fresh handle gives bitwise the uninterrupted
result, in both modes and both storage precisions (the paper reuses converged
wave functions as the initial states of later runs; this is its exact form)."""
import numpy as np
import pytest

from paper_2105_10517_gb300 import gpspin

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpspin.build()
    gpspin.load()


def params(**kw):
    p = dict(nx=72, ny=45, xlen=14.4, ylen=9.9, dt=0.004, c0=60.0, c2=-6.0, omeg=0.7, so_type=1, gamma=0.8,
             rabi=0.35)
    p.update(kw)
    return p


@pytest.mark.parametrize("precision", [gpspin.FP64, gpspin.FP32_MIXED])
@pytest.mark.parametrize("mode", [gpspin.IMAG, gpspin.REAL])
def test_resume_is_bitwise(tmp_path, precision, mode):
    p = params(precision=precision)
    with gpspin.Solver(p) as a:
        a.init_gaussian(seed=5)
        a.propagate(40, mode)
        want = a.get_state()
        ea = a.observables()
    with gpspin.Solver(p) as b:
        b.init_gaussian(seed=5)
        b.propagate(20, mode)
        b.save_checkpoint(tmp_path / "ck.bin")
    with gpspin.Solver(p) as c:
        c.load_checkpoint(tmp_path / "ck.bin")
        assert c.observables()["steps"] == 20
        c.propagate(20, mode)
        got = c.get_state()
        ec = c.observables()
    assert np.array_equal(got, want)
    assert ec["energy"] == ea["energy"] and ec["steps"] == 40


def test_refined_state_resumes_in_fp64():
    p = params(precision=gpspin.FP32_MIXED)
    with gpspin.Solver(p) as a:
        a.init_gaussian(seed=6)
        a.propagate(10, gpspin.IMAG)
        a.refine_fp64(10, gpspin.IMAG)
        ck = a.checkpoint()
        a.propagate(10, gpspin.IMAG)
        want = a.get_state()
    with gpspin.Solver(p) as b:
        b.restore(ck)
        b.propagate(10, gpspin.IMAG)
        assert np.array_equal(b.get_state(), want)


def test_load_rejects_foreign_buffers():
    p = params()
    with gpspin.Solver(p) as a:
        a.init_gaussian(seed=7)
        ck = a.checkpoint()
        before = a.get_state()
    with gpspin.Solver(params(nx=64)) as other:
        with pytest.raises(gpspin.GPError) as ei:
            other.restore(ck)  # another grid
        assert ei.value.status == 1
    with gpspin.Solver(p) as b:
        b.init_gaussian(seed=7)
        bad = b"XXXXXXXX" + ck[8:]
        for data in (bad, ck[:100], ck[:-8]):
            with pytest.raises(gpspin.GPError):
                b.restore(data)
        assert np.array_equal(b.get_state(), before)  # nothing changed
