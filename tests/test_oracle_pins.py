"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics,
not by the oracle itself (CPU only).

Each test names the passage of arXiv 2105.10517 (Supplementary Material) it
rests on.  The dense operators come from tests/dense.py, built with numpy from
the operator form of Eqs. (S.1)-(S.5); the oracle solves block-tridiagonal
systems line by line and evaluates Eq. (S.6) with the explicit SO terms, so a
dropped term, a sign or an index slip on either side fails here.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2105_10517_gb300 import inputs
from tests import dense

IMAG, REAL = oracle.IMAG, oracle.REAL


def tiny(**kw):
    p = dict(nx=7, ny=6, xlen=5.6, ylen=4.2, dt=0.03, wx=1.0, wy=1.3, c0=3.0, c2=-1.5, omeg=0.7,
             so_type=1, gamma=0.9, rabi=0.4)
    p.update(kw)
    return p


# ---------------------------------------------------------------------------
# P4: every directional substep equals the dense Crank-Nicolson solve built in
# the ORIGINAL spin basis (Eq. S.3 rotation term, SO term below Eq. S.4, Eq. S.5).
@pytest.mark.parametrize("mode", [IMAG, REAL])
@pytest.mark.parametrize("so_type", [0, 1, 2])
@pytest.mark.parametrize("which", ["X", "Y"])
def test_directional_substep_matches_dense_cn(mode, so_type, which):
    p = tiny(so_type=so_type)
    psi = inputs.random_state(p["nx"], p["ny"], seed=11 + so_type)
    a = dense.a_x(p) if which == "X" else dense.a_y(p)
    want = dense.cn(a, psi, p["dt"], mode)
    got = oracle.substep(p, psi, which, mode)
    assert np.max(np.abs(got - want)) < 1e-13


def test_directional_operators_are_hermitian():
    # -1/2 d_xx, -Omega L_z and the SO term are Hermitian (p = -i grad, Sigma Hermitian):
    # this is what makes real-time CN unitary.
    p = tiny(so_type=2)
    for a in (dense.a_x(p), dense.a_y(p), dense.h_linear(p)):
        assert np.max(np.abs(a - a.conj().T)) < 1e-12


# P11: at Omega = gamma = 0 the X substep on a sine mode of the discrete Laplacian
# multiplies it by the Cayley factor (1 - tau k)/(1 + tau k) exactly.
@pytest.mark.parametrize("mode", [IMAG, REAL])
def test_cayley_factor_on_laplacian_eigenmode(mode):
    nx, ny = 9, 4
    p = dict(nx=nx, ny=ny, xlen=4.5, ylen=2.0, dt=0.07, omeg=0.0, so_type=0)
    dx = p["xlen"] / nx
    n = 3
    i = np.arange(nx)
    mode_x = np.sin(n * math.pi * (i + 1) / (nx + 1))
    k = (1 - math.cos(n * math.pi / (nx + 1))) / dx ** 2  # eigenvalue of -1/2 D2
    rng = np.random.default_rng(3)
    amp = rng.normal(size=(3, ny)) + 1j * rng.normal(size=(3, ny))
    psi = amp[:, :, None] * mode_x[None, None, :]
    tau = 0.5 * p["dt"] * (1j if mode == REAL else 1.0)
    got = oracle.substep(p, psi, "X", mode)
    assert np.max(np.abs(got - psi * (1 - tau * k) / (1 + tau * k))) < 1e-14


# ---------------------------------------------------------------------------
# The c2 terms of Eqs. (S.1)-(S.2) equal c2 (F . Sigma) psi with F = psi^dagger Sigma psi,
# and the Rabi terms equal R Sigma_x psi: this is the form the pointwise substep uses.
def test_spin_exchange_and_rabi_terms_match_component_form():
    rng = np.random.default_rng(5)
    c2, r = -2.7, 0.6
    for _ in range(20):
        ps, p0, pm = rng.normal(size=3) + 1j * rng.normal(size=3)
        rp, r0, rm = abs(ps) ** 2, abs(p0) ** 2, abs(pm) ** 2
        paper = np.array([
            c2 * (rp - rm + r0) * ps + c2 * p0 ** 2 * np.conj(pm) + r / math.sqrt(2) * p0,
            c2 * (rp + rm) * p0 + 2 * c2 * ps * pm * np.conj(p0) + r / math.sqrt(2) * (ps + pm),
            c2 * (rm - rp + r0) * pm + c2 * p0 ** 2 * np.conj(ps) + r / math.sqrt(2) * p0,
        ])
        v = np.array([ps, p0, pm])
        f = [np.real(np.vdot(v, s @ v)) for s in (dense.SX, dense.SY, dense.SZ)]
        mat = c2 * (f[0] * dense.SX + f[1] * dense.SY + f[2] * dense.SZ) + r * dense.SX
        assert np.max(np.abs(mat @ v - paper)) < 1e-12


# P5: the pointwise substep equals expm(-tau' H_loc) psi per site, H_loc frozen at
# the start of the substep (scipy's Pade expm is independent of the oracle's series).
@pytest.mark.parametrize("mode", [IMAG, REAL])
def test_pointwise_substep_matches_expm(mode):
    p = tiny(c0=40.0, c2=-25.0, rabi=3.0, dt=0.05)
    psi = inputs.random_state(p["nx"], p["ny"], seed=21)
    got = oracle.substep(p, psi, "P", mode)
    x, y, _, _ = dense.axes(p)
    v = dense.trap(p)
    tau = p["dt"] * (1j if mode == REAL else 1.0)
    for j in range(p["ny"]):
        for i in range(p["nx"]):
            s = psi[:, j, i]
            rho = np.sum(np.abs(s) ** 2)
            f = [np.real(np.vdot(s, m @ s)) for m in (dense.SX, dense.SY, dense.SZ)]
            h = (v[j, i] + p["c0"] * rho) * np.eye(3) + p["c2"] * (
                f[0] * dense.SX + f[1] * dense.SY + f[2] * dense.SZ) + p["rabi"] * dense.SX
            want = scipy.linalg.expm(-tau * h) @ s
            assert np.max(np.abs(got[:, j, i] - want)) < 2e-14 * max(1.0, np.max(np.abs(want)))


def test_pointwise_substep_real_time_is_unitary_per_site():
    p = tiny(c0=40.0, c2=-25.0, rabi=3.0, dt=0.05)
    psi = inputs.random_state(p["nx"], p["ny"], seed=22)
    got = oracle.substep(p, psi, "P", REAL)
    assert np.max(np.abs(np.sum(np.abs(got) ** 2, 0) - np.sum(np.abs(psi) ** 2, 0))) < 1e-13


# ---------------------------------------------------------------------------
# Energy functional (S.6) with the explicit SO terms f_{+-1}, f_0 equals the
# expectation of the operator form plus the nonlinear terms; mu = <H_GP>/N.
@pytest.mark.parametrize("so_type", [0, 1, 2])
def test_energy_functional_matches_operator_form(so_type):
    p = tiny(so_type=so_type)
    psi = inputs.random_state(p["nx"], p["ny"], seed=31 + so_type)
    obs = oracle.observables(p, psi)
    e, mu = dense.energy(p, psi)
    assert abs(obs["energy"] - e) < 1e-12 * max(1, abs(e))
    assert abs(obs["mu"] - mu) < 1e-12 * max(1, abs(mu))
    _, _, dx, dy = dense.axes(p)
    nc = np.sum(np.abs(psi) ** 2, axis=(1, 2)) * dx * dy
    assert np.allclose(obs["norm"], nc, rtol=1e-14, atol=0)
    assert abs(obs["magnetization"] - (nc[0] - nc[2])) < 1e-13


def _ho_ground_1d(n, length):
    """Lowest eigenpair of the 1D discrete -1/2 D2 + x^2/2 on the cell-centred grid."""
    h = length / n
    x = -0.5 * length + (np.arange(n) + 0.5) * h
    m = -0.5 * dense.d2(n, h) + np.diag(0.5 * x ** 2)
    w, v = np.linalg.eigh(m)
    g = v[:, 0] * np.sign(v[n // 2, 0])
    return w[0], g / math.sqrt(np.sum(g ** 2) * h)


# P1: non-interacting, isotropic: the discrete ground state is the product of the
# 1D discrete ground states and its energy is exactly 2 e0.
def test_energy_of_discrete_ho_ground_state_is_twice_1d():
    n, length = 20, 10.0
    e0, g = _ho_ground_1d(n, length)
    p = dict(nx=n, ny=n, xlen=length, ylen=length, dt=0.01)
    frac = np.array([0.2, 0.5, 0.3])
    psi = np.sqrt(frac)[:, None, None] * np.outer(g, g)[None].astype(complex)
    obs = oracle.observables(p, psi)
    assert abs(obs["energy"] - 2 * e0) < 1e-12
    # rotation energy of a real state vanishes, whatever Omega (L_z is imaginary)
    obs_rot = oracle.observables(dict(p, omeg=0.8), psi)
    assert abs(obs_rot["energy"] - 2 * e0) < 1e-12


# P2: Rabi only: the ground state is the HO ground state times the Sigma_x
# eigenvector with eigenvalue -1, with energy 2 e0 - R.
def test_energy_of_rabi_ground_state():
    n, length, r = 20, 10.0, 0.7
    e0, g = _ho_ground_1d(n, length)
    p = dict(nx=n, ny=n, xlen=length, ylen=length, dt=0.01, rabi=r)
    spinor = np.array([1.0, -math.sqrt(2.0), 1.0]) / 2
    psi = spinor[:, None, None] * np.outer(g, g)[None].astype(complex)
    obs = oracle.observables(p, psi)
    assert abs(obs["energy"] - (2 * e0 - r)) < 1e-12


# P1/P2 dynamics: imaginary-time propagation converges to those ground states;
# the Lie-split fixed point differs from the exact one by O(dt), its energy by O(dt^2).
@pytest.mark.parametrize("rabi", [0.0, 0.7])
def test_imaginary_time_converges_to_ho_ground_energy(rabi):
    n, length = 16, 8.0
    e0, g = _ho_ground_1d(n, length)
    errs = []
    for dt in (0.04, 0.02):
        p = dict(nx=n, ny=n, xlen=length, ylen=length, dt=dt, rabi=rabi)
        psi = inputs.gaussian_state(n, n, length, length, frac=(0.3, 0.3, 0.4), seed=4, phase_noise=0.0)
        psi = oracle.propagate(p, psi, int(round(16.0 / dt)), IMAG)
        errs.append(oracle.observables(p, psi)["energy"] - (2 * e0 - rabi))
    assert 0 <= errs[1] < errs[0] < 5e-3
    assert errs[0] / errs[1] > 3.0  # second order in dt


# P3: with 0 < Omega < 1 the non-interacting ground energy is still the Omega = 0 one.
def test_rotation_does_not_lower_noninteracting_ground_energy():
    n, length, dt = 16, 8.0, 0.02
    e0, _ = _ho_ground_1d(n, length)
    p = dict(nx=n, ny=n, xlen=length, ylen=length, dt=dt, omeg=0.5)
    psi = inputs.gaussian_state(n, n, length, length, seed=6, phase_noise=1e-2)
    psi = oracle.propagate(p, psi, 800, IMAG)
    e = oracle.observables(p, psi)["energy"]
    assert abs(e - 2 * e0) < 2e-3


# ---------------------------------------------------------------------------
# P6: real time conserves the norm (H Hermitian, CN a Cayley transform, P unitary),
# and the magnetisation when gamma = R = 0 (c2 F.Sigma commutes with total F_z).
def test_real_time_conserves_norm_and_magnetisation():
    p = inputs.physics(inputs.CONFIGS["small64"])
    p.update(nx=32, ny=32, xlen=16.0, ylen=16.0, dt=0.002, so_type=0, rabi=0.0)
    psi = inputs.gaussian_state(32, 32, 16.0, 16.0, frac=(0.5, 0.2, 0.3), seed=9)
    o0 = oracle.observables(p, psi)
    psi2 = oracle.propagate(p, psi, 100, REAL)
    o1 = oracle.observables(p, psi2)
    assert abs(o1["norm_total"] - o0["norm_total"]) < 1e-13
    assert abs(o1["magnetization"] - o0["magnetization"]) < 1e-13
    # with SO and Rabi on, the norm is still conserved
    q = dict(p, so_type=2, gamma=0.8, rabi=0.5)
    o2 = oracle.observables(q, oracle.propagate(q, psi, 100, REAL))
    assert abs(o2["norm_total"] - o0["norm_total"]) < 1e-13


# P7: imaginary time lowers the energy monotonically (after the first step).
def test_imaginary_time_energy_is_non_increasing():
    p = inputs.physics(inputs.CONFIGS["small64"])
    p.update(nx=32, ny=32, xlen=16.0, ylen=16.0, dt=0.01)
    psi = inputs.gaussian_state(32, 32, 16.0, 16.0, seed=1)
    psi = oracle.step(p, psi, IMAG)
    es = []
    for _ in range(60):
        psi = oracle.step(p, psi, IMAG)
        es.append(oracle.observables(p, psi)["energy"])
    d = np.diff(es)
    assert np.all(d <= 1e-12 * abs(es[0]))
    assert es[-1] < es[0]


# P8: Rashba at +Omega from psi(x, y) equals Dresselhaus at -Omega from psi(x, -y)
# mirrored (the paper's statement that the two give identical structure once the
# sign of the rotation is changed).
@pytest.mark.parametrize("mode", [IMAG, REAL])
def test_rashba_dresselhaus_mirror_symmetry(mode):
    p = inputs.physics(inputs.CONFIGS["small64"])
    p.update(nx=24, ny=24, xlen=12.0, ylen=12.0, dt=0.005, rabi=0.3)
    psi = inputs.random_state(24, 24, seed=17, scale=0.1) + inputs.gaussian_state(24, 24, 12.0, 12.0, seed=2)
    pr = dict(p, so_type=1, omeg=0.6)
    pd = dict(p, so_type=2, omeg=-0.6)
    a = oracle.propagate(pr, psi, 20, mode)
    b = oracle.propagate(pd, psi[:, ::-1, :], 20, mode)
    assert np.max(np.abs(a[:, ::-1, :] - b)) < 1e-13
    ea, eb = oracle.observables(pr, a)["energy"], oracle.observables(pd, b)["energy"]
    assert abs(ea - eb) < 1e-12 * abs(ea)


# ---------------------------------------------------------------------------
# P10: Thomas-Fermi trend: for large c0 and no spin terms, mu ~ sqrt(c0/pi) (2D, N = 1).
def test_thomas_fermi_chemical_potential():
    c0 = 200.0
    p = dict(nx=32, ny=32, xlen=16.0, ylen=16.0, dt=0.02, c0=c0)
    psi = inputs.gaussian_state(32, 32, 16.0, 16.0, seed=3, phase_noise=0.0)
    psi = oracle.propagate(p, psi, 600, IMAG)
    mu = oracle.observables(p, psi)["mu"]
    assert abs(mu / math.sqrt(c0 / math.pi) - 1) < 0.06


# P9: c0 and c2 of Eq. (S.4) for the paper's 87Rb and 23Na parameters are
# checked against the printed values stored in tests/golden/ (tests/test_golden.py).


def test_normalisation_after_imaginary_step():
    p = inputs.physics(inputs.CONFIGS["small64"])
    p.update(nx=16, ny=16)
    psi = 2.0 * inputs.gaussian_state(16, 16, 16.0, 16.0, seed=1)
    out = oracle.step(p, psi, IMAG)
    assert abs(oracle.observables(p, out)["norm_total"] - 1.0) < 1e-14


def test_oracle_rejects_bad_parameters():
    p = tiny(dt=-1.0)
    with pytest.raises(oracle.OracleError):
        oracle.step(p, inputs.random_state(7, 6), IMAG)


# ---------------------------------------------------------------------------
# Magnetisation-constrained normalisation (both conditions below Eq. S.5).
def _norms(p, psi):
    _, _, dx, dy = dense.axes(p)
    return np.sum(np.abs(psi) ** 2, axis=(1, 2)) * dx * dy


@pytest.mark.parametrize("m", [-0.4, 0.0, 0.3])
def test_constrained_normalisation_meets_both_conditions(m):
    p = tiny(so_type=0, rabi=0.0)
    psi = inputs.random_state(p["nx"], p["ny"], seed=71)
    before = _norms(p, psi)
    out = oracle.normalize_m(p, psi, m)
    after = _norms(p, out)
    assert abs(after.sum() - 1) < 1e-14 and abs(after[0] - after[2] - m) < 1e-14
    sig = np.sqrt(after / before)
    assert abs(sig[0] * sig[2] - sig[1] ** 2) < 1e-14  # the flow's extra condition


def test_constrained_normalisation_maps_the_rotated_ferromagnetic_populations():
    # populations (1/4, 1/2, 1/4) -> ((1+m)^2/4, (1-m^2)/2, (1-m)^2/4): the spin-rotated
    # fully polarised family, closed under the projection
    p = dict(nx=8, ny=8, xlen=4.0, ylen=4.0, dt=0.01)
    g = inputs.gaussian_state(8, 8, 4.0, 4.0, frac=(0.25, 0.5, 0.25), seed=3, phase_noise=0.0)
    for m in (-0.5, 0.2, 0.7):
        n = _norms(p, oracle.normalize_m(p, g, m))
        assert np.allclose(n, [(1 + m) ** 2 / 4, (1 - m * m) / 2, (1 - m) ** 2 / 4], atol=1e-14)


def test_constrained_imaginary_time_keeps_m_and_lowers_energy():
    p = dict(nx=24, ny=24, xlen=12.0, ylen=12.0, dt=0.01, c0=40.0, c2=-3.0, omeg=0.3)
    psi = inputs.gaussian_state(24, 24, 12.0, 12.0, frac=(0.5, 0.3, 0.2), seed=8)
    es = []
    for _ in range(40):
        psi = oracle.propagate_m(p, psi, 1, 0.25)
        o = oracle.observables(p, psi)
        assert abs(o["norm_total"] - 1) < 1e-13 and abs(o["magnetization"] - 0.25) < 1e-13
        es.append(o["energy"])
    assert np.all(np.diff(es[1:]) <= 1e-12 * abs(es[0]))
    # SO or Rabi coupling does not conserve m: the constrained flow is rejected there
    with pytest.raises(oracle.OracleError):
        oracle.propagate_m(dict(p, rabi=0.1), psi, 1, 0.25)


# ---------------------------------------------------------------------------
# The composition of one step (reading of the paper's split-step scheme, program
# summary "Solution method", and of the normalisation condition below Eq. S.5):
# P(dt), then X(dt), then Y(dt), then in imaginary time the rescaling to N = 1.
# Built here from scipy's expm per site and the dense CN solves of tests/dense.py,
# in that order; swapping X and Y, or normalising before Y, or applying P last
# must each miss, so the pin fixes the order and not only the pieces.
def _dense_p(p, psi, mode):
    v = dense.trap(p)
    tau = p["dt"] * (1j if mode == REAL else 1.0)
    out = np.empty_like(psi)
    for j in range(p["ny"]):
        for i in range(p["nx"]):
            s = psi[:, j, i]
            rho = np.sum(np.abs(s) ** 2)
            f = [np.real(np.vdot(s, m @ s)) for m in (dense.SX, dense.SY, dense.SZ)]
            h = (v[j, i] + p["c0"] * rho) * np.eye(3) + p["c2"] * (
                f[0] * dense.SX + f[1] * dense.SY + f[2] * dense.SZ) + p["rabi"] * dense.SX
            out[:, j, i] = scipy.linalg.expm(-tau * h) @ s
    return out


def _dense_norm(p, psi):
    da = (p["xlen"] / p["nx"]) * (p["ylen"] / p["ny"])
    return psi / math.sqrt(da * np.sum(np.abs(psi) ** 2))


def _dense_step(p, psi, mode, order="PXYN"):
    for s in order:
        if s == "P":
            psi = _dense_p(p, psi, mode)
        elif s == "X":
            psi = dense.cn(dense.a_x(p), psi, p["dt"], mode)
        elif s == "Y":
            psi = dense.cn(dense.a_y(p), psi, p["dt"], mode)
        elif s == "N" and mode == IMAG:
            psi = _dense_norm(p, psi)
    return psi


@pytest.mark.parametrize("mode", [IMAG, REAL])
@pytest.mark.parametrize("so_type", [1, 2])
def test_step_is_p_then_x_then_y_then_normalise(mode, so_type):
    p = tiny(so_type=so_type, c0=30.0, c2=-12.0, rabi=1.5, dt=0.04)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=61, phase_noise=0.5) \
        + inputs.random_state(p["nx"], p["ny"], seed=62, scale=0.1)
    got = oracle.step(p, psi, mode)
    want = _dense_step(p, psi, mode)
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got - want)) <= 1e-13 * scale
    # negative controls: each plausible misordering misses by far more than rounding
    wrong = ["PYXN", "XPYN", "PXNY" if mode == IMAG else "XYP"]
    for order in wrong:
        assert np.max(np.abs(_dense_step(p, psi, mode, order) - want)) > 1e-6 * scale, order


# The oracle spreads independent lines over threads (the paper's program runs its
# line loops under OpenMP); the result must not depend on the thread count.
@pytest.mark.parametrize("mode", [IMAG, REAL])
def test_oracle_threads_give_bitwise_identical_steps(mode):
    p = tiny(nx=40, ny=33, xlen=8.0, ylen=6.6, so_type=2)
    psi = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=63, phase_noise=0.3)
    keep = oracle.set_threads(0)
    try:
        oracle.set_threads(1)
        one = oracle.propagate(p, psi, 5, mode)
        n = oracle.set_threads(4)
        many = oracle.propagate(p, psi, 5, mode)
    finally:
        oracle.set_threads(keep)
    assert np.array_equal(one, many), n
