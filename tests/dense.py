"""Dense reference operators for tiny grids, built with numpy straight from the
operator form of the paper's equations (Supplementary Material, Eqs. S.1-S.5):

  H = -1/2 (d_xx + d_yy) + V - Omega L_z + gamma (eta p_y Sigma_x - p_x Sigma_y)
      + R Sigma_x,   L_z = -i (x d_y - y d_x),  p = -i grad,

on the cell-centred grid with zero Dirichlet data and central differences.  The
state vector index is (c, j, i) flattened as psi[c][j][i].  These builders share
nothing with the oracle's line solver; they are how the tests pin it.
"""
import numpy as np

SQ2 = np.sqrt(2.0)
SX = np.array([[0, 1, 0], [1, 0, 1], [0, 1, 0]], dtype=complex) / SQ2
SY = 1j * np.array([[0, -1, 0], [1, 0, -1], [0, 1, 0]], dtype=complex) / SQ2
SZ = np.diag([1.0, 0.0, -1.0]).astype(complex)


def axes(p):
    nx, ny = int(p["nx"]), int(p["ny"])
    dx, dy = p["xlen"] / nx, p["ylen"] / ny
    x = -0.5 * p["xlen"] + (np.arange(nx) + 0.5) * dx
    y = -0.5 * p["ylen"] + (np.arange(ny) + 0.5) * dy
    return x, y, dx, dy


def d1(n, h):
    m = np.zeros((n, n))
    for k in range(n):
        if k + 1 < n:
            m[k, k + 1] = 1 / (2 * h)
        if k > 0:
            m[k, k - 1] = -1 / (2 * h)
    return m


def d2(n, h):
    m = np.zeros((n, n))
    for k in range(n):
        m[k, k] = -2 / h ** 2
        if k + 1 < n:
            m[k, k + 1] = 1 / h ** 2
        if k > 0:
            m[k, k - 1] = 1 / h ** 2
    return m


def eta_gamma(p):
    so = int(p.get("so_type", 0))
    eta = {0: 0, 1: 1, 2: -1}[so]
    return eta, (float(p.get("gamma", 0.0)) if so else 0.0)


def a_x(p):
    """X-direction operator: -1/2 d_xx - i Omega y d_x + i gamma Sigma_y d_x."""
    x, y, dx, dy = axes(p)
    nx, ny = len(x), len(y)
    eta, g = eta_gamma(p)
    om = float(p.get("omeg", 0.0))
    ix, iy, i3 = np.eye(nx), np.eye(ny), np.eye(3)
    kin = np.kron(i3, np.kron(iy, -0.5 * d2(nx, dx)))
    rot = -1j * om * np.kron(i3, np.kron(np.diag(y), d1(nx, dx)))
    so = 1j * g * np.kron(SY, np.kron(iy, d1(nx, dx)))
    return kin + rot + so


def a_y(p):
    """Y-direction operator: -1/2 d_yy + i Omega x d_y - i eta gamma Sigma_x d_y."""
    x, y, dx, dy = axes(p)
    nx, ny = len(x), len(y)
    eta, g = eta_gamma(p)
    om = float(p.get("omeg", 0.0))
    ix, i3 = np.eye(nx), np.eye(3)
    kin = np.kron(i3, np.kron(-0.5 * d2(ny, dy), ix))
    rot = 1j * om * np.kron(i3, np.kron(d1(ny, dy), np.diag(x)))
    so = -1j * eta * g * np.kron(SX, np.kron(d1(ny, dy), ix))
    return kin + rot + so


def trap(p):
    x, y, dx, dy = axes(p)
    wx, wy = float(p.get("wx", 1.0)), float(p.get("wy", 1.0))
    v = 0.5 * (wx ** 2 * x[None, :] ** 2 + wy ** 2 * y[:, None] ** 2)
    return v


def h_linear(p):
    """Full linear Hamiltonian: A_x + A_y + V + R Sigma_x."""
    x, y, dx, dy = axes(p)
    n = len(x) * len(y)
    v = np.kron(np.eye(3), np.diag(trap(p).ravel()))
    rabi = float(p.get("rabi", 0.0)) * np.kron(SX, np.eye(n))
    return a_x(p) + a_y(p) + v + rabi


def cn(a, psi, dt, mode):
    """Crank-Nicolson: (I + tau A) psi' = (I - tau A) psi, tau = dt/2 (imag) or i dt/2 (real)."""
    tau = 0.5 * dt * (1j if mode == 1 else 1.0)
    n = a.shape[0]
    rhs = (np.eye(n) - tau * a) @ psi.ravel()
    return np.linalg.solve(np.eye(n) + tau * a, rhs).reshape(psi.shape)


def spin_density(psi):
    """F_k = psi^dagger Sigma_k psi per site, shape (3, ny, nx)."""
    out = []
    for s in (SX, SY, SZ):
        out.append(np.real(np.einsum("cji,cd,dji->ji", psi.conj(), s, psi)))
    return np.array(out)


def energy(p, psi):
    """E = dA [psi^dagger H_lin psi + sum (c0 rho^2/2 + c2 |F|^2/2)] and mu = <H_GP>/N."""
    x, y, dx, dy = axes(p)
    da = dx * dy
    h = h_linear(p)
    lin = np.real(np.vdot(psi.ravel(), h @ psi.ravel()))
    rho = np.sum(np.abs(psi) ** 2, axis=0)
    f = spin_density(psi)
    f2 = np.sum(f ** 2, axis=0)
    nl = np.sum(0.5 * p.get("c0", 0.0) * rho ** 2 + 0.5 * p.get("c2", 0.0) * f2)
    e = da * (lin + nl)
    n = da * np.sum(rho)
    mu = (e + da * nl) / n
    return e, mu
