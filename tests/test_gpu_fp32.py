"""The FP32-storage precision form (GP_FP32_MIXED): psi stored and propagated as
complex64, Thomas coefficient tables computed in FP64, norms and observables
reduced in FP64, and gp_refine_fp64 continuing in FP64.  Errors are stated
against the FP64 oracle: single substeps within a few FP32 roundings, runs
within |dE/E| <= 1e-6 after the FP64 refinement block."""
import numpy as np
import pytest

import oracle
from paper_2105_10517_gb300 import gpspin, inputs

pytestmark = pytest.mark.gpu

IMAG, REAL = gpspin.IMAG, gpspin.REAL
F32 = gpspin.FP32_MIXED


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpspin.build()
    gpspin.load()


def ragged(**kw):
    p = dict(nx=72, ny=45, xlen=14.4, ylen=9.9, dt=0.004, wx=1.0, wy=1.2, c0=60.0, c2=-6.0, omeg=0.7,
             so_type=1, gamma=0.8, rabi=0.35, precision=F32)
    p.update(kw)
    return p


@pytest.mark.parametrize("mode", [IMAG, REAL])
@pytest.mark.parametrize("which", ["P", "X", "Y"])
@pytest.mark.parametrize("so_type", [1, 2])
def test_fp32_substep_parity(which, mode, so_type):
    p = ragged(so_type=so_type)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=3, phase_noise=0.3) \
        + inputs.random_state(p["nx"], p["ny"], seed=103, scale=0.05)
    want = oracle.substep(p, psi, which, mode)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.apply_substep(which, mode)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 2e-6 * np.max(np.abs(want))


@pytest.mark.parametrize("which", ["P", "X", "Y"])
def test_fp32_substeps_on_clustered_tilings(which):
    """Lines of 320 and 288 points: the default tilings split each line group
    over a cluster of CTAs, including the substeps that skip the solve."""
    p = ragged(nx=320, ny=288, xlen=0.05 * 320, ylen=0.05 * 288, dt=0.0005)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=4, phase_noise=0.3) \
        + inputs.random_state(p["nx"], p["ny"], seed=104, scale=0.05)
    want = oracle.substep(p, psi, which, IMAG)
    with gpspin.Solver(p) as s:
        t = s.tiling(IMAG)
        assert t["xpass"]["cluster"] > 1 and t["ypass"]["cluster"] > 1
        s.set_state(psi)
        s.apply_substep(which, IMAG)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 2e-6 * np.max(np.abs(want))


def test_fp32_then_fp64_refinement_matches_oracle_energy():
    """1000 FP32 steps then 1000 FP64 refinement steps versus 2000 FP64 oracle steps
    of the 64 x 64 workload: |dE/E| <= 1e-6 and the density error stated."""
    c = inputs.CONFIGS["small64"]
    p = dict(inputs.physics(c), precision=F32)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=c["seed"])
    half = oracle.propagate(p, psi, 1000, IMAG)
    want = oracle.propagate(p, half, 1000, IMAG)
    eo = oracle.observables(p, want)
    with gpspin.Solver(p) as s:
        s.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
        s.propagate(1000, IMAG)
        e32 = s.observables()["energy"]
        s.refine_fp64(1000, IMAG)
        got = s.get_state()
        o = s.observables()
    assert abs(o["energy"] - eo["energy"]) <= 1e-6 * abs(eo["energy"])
    rho_err = np.sqrt(np.sum((np.abs(got) ** 2 - np.abs(want) ** 2) ** 2)) / np.sqrt(np.sum(np.abs(want) ** 4))
    assert rho_err < 1e-4
    # the FP32 phase alone, against the oracle at the same step
    e_half = oracle.observables(p, half)["energy"]
    assert abs(e32 - e_half) <= 1e-5 * abs(e_half)


def test_refine_switches_to_fp64_bitwise():
    """After gp_refine_fp64 the handle propagates exactly like an FP64 handle fed the
    widened state."""
    p = ragged()
    with gpspin.Solver(p) as s:
        s.init_gaussian(seed=5)
        s.propagate(30, IMAG)
        s.refine_fp64(0, IMAG)
        mid = s.get_state()
        s.propagate(20, IMAG)
        a = s.get_state()
    with gpspin.Solver(dict(p, precision=gpspin.FP64)) as t:
        t.set_state(mid)
        t.propagate(20, IMAG)
        b = t.get_state()
    assert np.max(np.abs(a - b)) <= 1e-14


def test_fp32_observables_are_fp64_reductions_of_the_widened_state():
    p = ragged()
    with gpspin.Solver(p) as s:
        s.init_gaussian(seed=8)
        s.propagate(17, IMAG)
        st = s.get_state()
        o = s.observables()
    q = dict(p, precision=gpspin.FP64)
    oo = oracle.observables(q, st)
    for k in ("norm_total", "magnetization", "energy", "mu"):
        assert abs(o[k] - oo[k]) <= 1e-12 * max(1.0, abs(oo[k])), k


def test_fp32_real_time_norm_drift():
    p = ragged(so_type=2, dt=0.002)
    with gpspin.Solver(p) as s:
        s.init_gaussian(seed=9)
        s.propagate(1, IMAG)
        n0 = s.observables()["norm_total"]
        s.propagate(500, REAL)
        n1 = s.observables()["norm_total"]
    assert abs(n1 - n0) <= 1e-4


def test_fp32_full_size_vortex512_step_parity():
    c = inputs.CONFIGS["vortex512"]
    p = dict(inputs.physics(c), precision=F32)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=c["seed"])
    want = oracle.propagate(p, psi, 2, IMAG)
    with gpspin.Solver(p) as s:
        s.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
        s.propagate(2, IMAG)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 2e-6 * np.max(np.abs(want))


def test_fp32_full_size_precision2048_autotuned_step_parity():
    """The 2048^2 complex64 step in the launch configuration bench.py times
    (autotuned: register-resident solves, clusters of CTAs) against the oracle."""
    c = inputs.CONFIGS["precision2048"]
    p = dict(inputs.physics(c), precision=F32)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=c["seed"])
    want = oracle.propagate(p, psi, 2, IMAG)
    with gpspin.Solver(p) as s:
        s.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
        s.autotune(IMAG)
        t = s.tiling(IMAG)
        assert t["xpass"]["register_solve"] and t["ypass"]["register_solve"]
        s.propagate(2, IMAG)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 2e-6 * np.max(np.abs(want))
