"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no step of the method: it only builds initial wave functions
and parameter sets.  The counter-based generator is splitmix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): state
z = x + 0x9E3779B97F4A7C15, then z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9,
z = (z ^ (z >> 27)) * 0x94D049BB133111EB, z ^ (z >> 31); the top 53 bits times
2^-53 give u in [0, 1).
"""
import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x):
    """splitmix64 output for an array of uint64 counters."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform01(seed, n):
    """u_k = top 53 bits of splitmix64(seed ^ k) * 2^-53, k = 0..n-1."""
    k = np.arange(n, dtype=np.uint64) ^ np.uint64(seed)
    return (splitmix64(k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def grid(nx, ny, xlen, ylen):
    dx, dy = xlen / nx, ylen / ny
    x = -0.5 * xlen + (np.arange(nx) + 0.5) * dx
    y = -0.5 * ylen + (np.arange(ny) + 0.5) * dy
    return x, y


def gaussian_state(nx, ny, xlen, ylen, frac=(0.25, 0.5, 0.25), seed=1, phase_noise=1e-3, normalize=True):
    """psi_c = sqrt(frac_c) pi^-1/2 exp(-(x^2+y^2)/2) exp(i phase_noise (2u-1)),
    u from splitmix64(seed ^ ((c ny + j) nx + i)); normalised to dx dy sum |psi|^2 = 1."""
    x, y = grid(nx, ny, xlen, ylen)
    g = np.exp(-0.5 * (x[None, :] ** 2 + y[:, None] ** 2)) / math.sqrt(math.pi)
    u = uniform01(seed, 3 * nx * ny).reshape(3, ny, nx)
    phase = phase_noise * (2.0 * u - 1.0)
    psi = np.sqrt(np.asarray(frac, dtype=np.float64))[:, None, None] * g[None] * np.exp(1j * phase)
    if normalize:
        n = np.sum(np.abs(psi) ** 2) * (xlen / nx) * (ylen / ny)
        psi = psi / math.sqrt(n)
    return psi.astype(np.complex128)


def winding_state(nx, ny, xlen, ylen, frac=(0.25, 0.5, 0.25), winding=(0, 0, 0), seed=1, phase_noise=1e-3,
                  normalize=True):
    """gaussian_state times (x + i sgn(l_c) y)^|l_c| per component: centre vortices
    of charge l_c built into the initial guess (normalised to 1)."""
    x, y = grid(nx, ny, xlen, ylen)
    psi = gaussian_state(nx, ny, xlen, ylen, frac, seed, phase_noise, normalize=False)
    X, Y = np.meshgrid(x, y)
    for c, l in enumerate(winding):
        if l:
            psi[c] = psi[c] * (X + 1j * np.sign(l) * Y) ** abs(int(l))
    if normalize:
        n = np.sum(np.abs(psi) ** 2) * (xlen / nx) * (ylen / ny)
        psi = psi / math.sqrt(n)
    return psi.astype(np.complex128)


def random_state(nx, ny, seed=7, scale=1.0):
    """A rough complex field (splitmix64 real and imaginary parts in [-1, 1)) for
    substep tests that must exercise every coefficient, not just smooth data."""
    u = uniform01(seed, 6 * nx * ny).reshape(2, 3, ny, nx)
    return (scale * ((2 * u[0] - 1) + 1j * (2 * u[1] - 1))).astype(np.complex128)


# Workloads of the benchmark and the parity tests (grid, box, time step, physics).
CONFIGS = {
    "small64": dict(nx=64, ny=64, xlen=16.0, ylen=16.0, dt=0.005, c0=50.0, c2=-2.0, omeg=0.5,
                    so_type=1, gamma=0.5, rabi=0.0, mode=0, steps=2000, seed=1),
    "vortex512": dict(nx=512, ny=512, xlen=32.0, ylen=32.0, dt=0.001, c0=500.0, c2=-10.0, omeg=0.8,
                      so_type=1, gamma=1.0, rabi=0.0, mode=0, steps=20000, seed=2),
    "quench1024": dict(nx=1024, ny=1024, xlen=40.0, ylen=40.0, dt=0.0005, c0=800.0, c2=15.0, omeg=0.6,
                       so_type=2, gamma=0.75, rabi=0.5, mode=1, steps=10000, seed=3),
    "precision2048": dict(nx=2048, ny=2048, xlen=48.0, ylen=48.0, dt=0.0005, c0=1500.0, c2=-25.0, omeg=0.85,
                          so_type=1, gamma=1.5, rabi=0.25, mode=0, steps=40000, seed=5),
}


def physics(cfg):
    """The parameter keys of a workload, without its run-control keys."""
    return {k: v for k, v in cfg.items() if k not in ("mode", "steps", "seed")}


def serving_trace(n=256, rate=20.0, seed=4, sizes=(128, 256, 384, 512), box=32.0):
    """Seeded request trace of the parameter-sweep serving workload: Poisson
    arrivals at `rate` per second; grids drawn uniformly from `sizes` on a box of
    side `box` (DX = box/N) with the imaginary-time step DT = 0.1 DX^2; Omega ~
    U[0, 0.9], gamma ~ U[0, 2] (Rashba or Dresselhaus 50/50), R ~ U[0, 1],
    c0 ~ U[100, 800], c2 ~ U[-20, 20]; each request starts from the seeded
    Gaussian state with its own seed."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for k in range(n):
        nx = int(rng.choice(sizes))
        dx = box / nx
        out.append(dict(
            arrival=float(t[k]),
            params=dict(nx=nx, ny=nx, xlen=box, ylen=box, dt=0.1 * dx * dx, omeg=float(rng.uniform(0, 0.9)),
                        gamma=float(rng.uniform(0, 2)), so_type=int(rng.integers(1, 3)),
                        rabi=float(rng.uniform(0, 1)), c0=float(rng.uniform(100, 800)),
                        c2=float(rng.uniform(-20, 20))),
            seed=1000 + k))
    return out
