"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: single substeps and short runs agree to 1e-12 (rounding order only:
the oracle solves 3x3-block systems in the original spin basis, the GPU solves
scalar systems per eigen-channel); after 1000 steps max|dpsi| <= 1e-10 and
|dE/E| <= 1e-12.
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


def ragged(**kw):
    # 72 x 45: several chunks per line plus a ragged last chunk in both directions
    p = dict(nx=72, ny=45, xlen=14.4, ylen=9.9, dt=0.004, wx=1.0, wy=1.2, c0=60.0, c2=-6.0, omeg=0.7,
             so_type=1, gamma=0.8, rabi=0.35)
    p.update(kw)
    return p


def smooth_plus_rough(p, seed):
    g = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=seed, phase_noise=0.3)
    return g + inputs.random_state(p["nx"], p["ny"], seed=seed + 100, scale=0.05)


@pytest.mark.parametrize("mode", [IMAG, REAL])
@pytest.mark.parametrize("so_type", [0, 1, 2])
@pytest.mark.parametrize("which", ["P", "X", "Y"])
def test_substep_parity(which, so_type, mode):
    p = ragged(so_type=so_type)
    psi = smooth_plus_rough(p, 3 + so_type)
    want = oracle.substep(p, psi, which, mode)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.apply_substep(which, mode)
        got = s.get_state()
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got - want)) <= 1e-13 * scale


@pytest.mark.parametrize("mode", [IMAG, REAL])
def test_substep_parity_large_arguments(mode):
    # dt c0 rho > 1/8 and dt |B| > 0.1: the library-function branches of P
    p = ragged(c0=4000.0, c2=-900.0, rabi=40.0, dt=0.01)
    psi = smooth_plus_rough(p, 9)
    want = oracle.substep(p, psi, "P", mode)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.apply_substep("P", mode)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("mode", [IMAG, REAL])
@pytest.mark.parametrize("c0", [-3.0, -25.0, -300.0])
def test_substep_parity_attractive_contact(c0, mode):
    # c0 < 0 (attractive): dt c0 rho is negative, and its magnitude falls in each
    # tier of the scalar factor in turn (|x| <= 1/64, <= 1/8, beyond) somewhere on the grid
    p = ragged(c0=c0, dt=0.01)
    psi = smooth_plus_rough(p, 13)
    want = oracle.substep(p, psi, "P", mode)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.apply_substep("P", mode)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("mode", [IMAG, REAL])
def test_short_run_parity(mode):
    p = ragged()
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=5)
    want = oracle.propagate(p, psi, 20, mode)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.propagate(20, mode)
        got = s.get_state()
        obs = s.observables()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    o = oracle.observables(p, want)
    assert abs(obs["energy"] - o["energy"]) <= 1e-12 * abs(o["energy"])


def test_observables_parity():
    for so_type in (0, 1, 2):
        p = ragged(so_type=so_type)
        psi = smooth_plus_rough(p, 21 + so_type)
        o = oracle.observables(p, psi)
        with gpspin.Solver(p) as s:
            s.set_state(psi)
            g = s.observables()
        for k in ("norm_total", "magnetization", "energy", "mu"):
            assert abs(g[k] - o[k]) <= 1e-12 * max(1.0, abs(o[k])), k
        assert np.allclose(g["norm"], o["norm"], rtol=1e-13, atol=0)


def test_init_gaussian_matches_input_generator():
    p = ragged()
    want = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], frac=(0.25, 0.5, 0.25), seed=77,
                                 phase_noise=1e-3)
    with gpspin.Solver(p) as s:
        s.init_gaussian((0.25, 0.5, 0.25), seed=77, phase_noise=1e-3)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 1e-15


def test_thousand_step_parity_small64():
    """The 64 x 64 imaginary-time workload: 1000 steps, max|dpsi| <= 1e-10, |dE/E| <= 1e-12."""
    c = inputs.CONFIGS["small64"]
    p = inputs.physics(c)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=c["seed"])
    want = oracle.propagate(p, psi, 1000, IMAG)
    with gpspin.Solver(p) as s:
        s.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
        s.propagate(1000, IMAG)
        got = s.get_state()
        e = s.observables()["energy"]
    eo = oracle.observables(p, want)["energy"]
    assert np.max(np.abs(got - want)) <= 1e-10
    assert abs(e - eo) <= 1e-12 * abs(eo)


def test_real_time_parity_and_norm():
    p = ragged(so_type=2, nx=48, ny=40, xlen=12.0, ylen=10.0, dt=0.002)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=8)
    want = oracle.propagate(p, psi, 300, REAL)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.propagate(300, REAL)
        got = s.get_state()
        obs = s.observables()
    assert np.max(np.abs(got - want)) <= 1e-11
    assert abs(obs["norm_total"] - 1.0) <= 1e-12


def test_rashba_dresselhaus_mirror_on_gpu():
    p = ragged(nx=40, ny=36, xlen=10.0, ylen=9.0)
    psi = smooth_plus_rough(p, 31)
    with gpspin.Solver(dict(p, so_type=1, omeg=0.6)) as a, gpspin.Solver(dict(p, so_type=2, omeg=-0.6)) as b:
        a.set_state(psi)
        b.set_state(psi[:, ::-1, :].copy())
        a.propagate(50, IMAG)
        b.propagate(50, IMAG)
        ga, gb = a.get_state(), b.get_state()
        ea, eb = a.observables()["energy"], b.observables()["energy"]
    assert np.max(np.abs(ga[:, ::-1, :] - gb)) <= 1e-12
    assert abs(ea - eb) <= 1e-12 * abs(ea)


@pytest.mark.parametrize("shape", [(4, 4), (5, 9), (130, 17), (17, 130)])
def test_edge_shapes(shape):
    nx, ny = shape
    p = ragged(nx=nx, ny=ny, xlen=0.2 * nx, ylen=0.2 * ny)
    psi = smooth_plus_rough(p, 41)
    want = oracle.propagate(p, psi, 3, IMAG)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.propagate(3, IMAG)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_full_size_vortex512_sampled():
    """The 512 x 512 workload in the launch configuration the benchmark times:
    two steps compared everywhere (the oracle finishes them in seconds)."""
    c = inputs.CONFIGS["vortex512"]
    p = inputs.physics(c)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=c["seed"])
    want = oracle.propagate(p, psi, 2, IMAG)
    with gpspin.Solver(p) as s:
        s.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
        s.propagate(2, IMAG)
        got = s.get_state()
        e = s.observables()["energy"]
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    assert abs(e - oracle.observables(p, want)["energy"]) <= 1e-12 * abs(e)


def test_determinism_bitwise():
    p = ragged()
    out = []
    for _ in range(2):
        with gpspin.Solver(p) as s:
            s.init_gaussian(seed=3)
            s.propagate(25, IMAG)
            out.append((s.get_state(), s.observables()["energy"]))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_errors_are_reported():
    p = ragged()
    with gpspin.Solver(p) as s:
        bad = smooth_plus_rough(p, 1)
        bad[1, 3, 4] = np.nan
        with pytest.raises(gpspin.GPError) as ei:
            s.set_state(bad, normalize=True)
        assert ei.value.status == 4
        with pytest.raises(gpspin.GPError):
            s.propagate(-1)
        with pytest.raises(gpspin.GPError):
            s.set_params(dict(p, nx=10))
    # dt far beyond the tabulated factorisation's range
    with gpspin.Solver(ragged(dt=50.0)) as s:
        s.init_gaussian()
        with pytest.raises(gpspin.GPError) as ei:
            s.propagate(1)
        assert ei.value.status == 5


def test_omega_quench_rebuilds_coefficients():
    p = ragged()
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=12)
    q = dict(p, omeg=0.9)
    want = oracle.propagate(q, oracle.propagate(p, psi, 5, REAL), 5, REAL)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.propagate(5, REAL)
        s.set_params(q)
        s.propagate(5, REAL)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("mode", [IMAG, REAL])
def test_graph_replay_matches_direct_launches(mode):
    """gp_propagate replays a captured CUDA graph for blocks of steps; the result
    is bitwise the same as one direct step at a time."""
    p = ragged()
    out = []
    for chunks in ([37], [1] * 37):
        with gpspin.Solver(p) as s:
            s.init_gaussian(seed=4)
            for n in chunks:
                s.propagate(n, mode)
            out.append(s.get_state())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("mode", [IMAG, REAL])
@pytest.mark.parametrize("shape", [(300, 270), (301, 257)])
def test_long_lines_split_over_a_cluster(shape, mode):
    """Lines of >= 256 points span a 2-CTA cluster (carries through distributed
    shared memory); odd lengths also take the unstaged load path."""
    nx, ny = shape
    p = ragged(nx=nx, ny=ny, xlen=0.05 * nx, ylen=0.05 * ny, dt=0.0005)
    psi = smooth_plus_rough(p, 51)
    want = oracle.propagate(p, psi, 2, mode)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        s.propagate(2, mode)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    with gpspin.Solver(dict(p, precision=gpspin.FP32_MIXED)) as s:
        s.set_state(psi)
        s.propagate(2, mode)
        got32 = s.get_state()
    assert np.max(np.abs(got32 - want)) <= 4e-6 * np.max(np.abs(want))


@pytest.mark.parametrize("precision", [gpspin.FP64, gpspin.FP32_MIXED])
def test_autotune_keeps_state_and_results(precision):
    """gp_autotune times candidate tilings without changing the state; propagation
    with the tuned tilings agrees with the oracle."""
    p = ragged(nx=288, ny=264, xlen=0.05 * 288, ylen=0.05 * 264, dt=0.0005, precision=precision)
    psi = smooth_plus_rough(p, 61)
    want = oracle.propagate(p, psi, 3, IMAG)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        before = s.get_state()
        ms = s.autotune(IMAG)
        assert ms > 0
        assert np.array_equal(s.get_state(), before)
        s.propagate(3, IMAG)
        got = s.get_state()
    tol = 1e-12 if precision == gpspin.FP64 else 4e-6
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
@pytest.mark.parametrize("precision", [gpspin.FP64, gpspin.FP32_MIXED])
def test_every_cluster_size(cluster, precision):
    """Line groups spread over 1, 2, 4 or 8 CTAs of a cluster (carries through
    distributed shared memory) all give the oracle's result."""
    # 16 chunks per line at the least for a cluster of 8 (two per CTA)
    p = ragged(nx=640, ny=608, xlen=0.05 * 640, ylen=0.05 * 608, dt=0.0005, precision=precision)
    psi = smooth_plus_rough(p, 71)
    want = oracle.propagate(p, psi, 2, IMAG)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        for d in (0, 1):
            s.set_tiling(d, cluster=cluster, lines_per_cta=2 if cluster < 8 else 1, chunk=24)
        t = s.tiling()
        assert t["xpass"]["cluster"] == cluster and t["ypass"]["cluster"] == cluster
        s.propagate(2, IMAG)
        got = s.get_state()
    tol = 1e-12 if precision == gpspin.FP64 else 4e-6
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


@pytest.mark.parametrize("mode", [IMAG, REAL])
@pytest.mark.parametrize("cluster,lines", [(1, 1), (1, 3), (2, 2), (4, 1), (8, 1)])
def test_register_solve_complex128(cluster, lines, mode):
    """The complex128 register-resident solve (chunk length 32 held in registers,
    one line array in shared memory) gives the oracle's result on every cluster
    size, with ragged last chunks shorter than the fixup length (650 = 20 x 32
    + 10 and 610 = 19 x 32 + 2 points) and in both modes."""
    p = ragged(nx=650, ny=610, xlen=0.05 * 650, ylen=0.05 * 610, dt=0.0005)
    psi = smooth_plus_rough(p, 73)
    want = oracle.propagate(p, psi, 2, mode)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        for d in (0, 1):
            s.set_tiling(d, cluster=cluster, lines_per_cta=lines, chunk=32, mode=mode, register_solve=True)
        t = s.tiling(mode)
        assert t["xpass"]["register_solve"] and t["ypass"]["register_solve"]
        assert t["xpass"]["cluster"] == cluster and t["xpass"]["chunk"] == 32
        s.propagate(2, mode)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("mode", [IMAG, REAL])
@pytest.mark.parametrize("which", ["X", "Y"])
def test_register_solve_complex128_substeps(which, mode):
    """Single X and Y substeps with the complex128 register-resident solve on the
    72 x 45 grid (chunks of 32, 32, 8 and 32, 13 points)."""
    p = ragged()
    psi = smooth_plus_rough(p, 5)
    want = oracle.substep(p, psi, which, mode)
    with gpspin.Solver(p) as s:
        s.set_state(psi)
        for d in (0, 1):
            s.set_tiling(d, cluster=1, lines_per_cta=2, chunk=32, mode=mode, register_solve=True)
        s.apply_substep(which, mode)
        got = s.get_state()
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


POISON_TILINGS = [
    (gpspin.FP64, None),                            # the default tiling
    (gpspin.FP64, (2, 2, 32, False)),               # a 2-CTA cluster, shared-memory solve
    (gpspin.FP64, (2, 2, 32, True)),                # the register-resident complex128 solve
    (gpspin.FP64, (8, 1, 32, True)),
    (gpspin.FP32_MIXED, None),
    (gpspin.FP32_MIXED, (4, 2, 24, True)),          # complex64 register-resident solve
    (gpspin.FP32_MIXED, (2, 1, 40, False)),         # complex64 shared-memory solve
]


@pytest.mark.parametrize("mode", [IMAG, REAL])
@pytest.mark.parametrize("precision,tiling", POISON_TILINGS)
def test_every_element_written_each_step(precision, tiling, mode):
    """With the poison check on, every byte a pass must write is first set to a
    NaN pattern: the results stay bitwise those of a run without the check, so
    no pass leaves an element of the intermediate or of the state unwritten
    (ragged 650 x 610 grid; clusters, lines per CTA and both solve forms)."""
    p = ragged(nx=650, ny=610, xlen=0.05 * 650, ylen=0.05 * 610, dt=0.0005, precision=precision)
    psi = smooth_plus_rough(p, 79)
    out = []
    for debug in (False, True):
        with gpspin.Solver(p) as s:
            s.set_state(psi)
            if tiling:
                S, R, m, reg = tiling
                for d in (0, 1):
                    s.set_tiling(d, cluster=S, lines_per_cta=R, chunk=m, mode=mode, register_solve=reg)
            s.set_debug(debug)
            s.propagate(20, mode)  # one captured graph of 16 steps and 4 direct steps
            out.append((s.get_state(), s.observables()))
    assert np.all(np.isfinite(out[1][0]))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1]["energy"] == out[1][1]["energy"]
