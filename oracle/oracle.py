"""ctypes front end of the plain-C FP64 oracle in ``gp_oracle.c``.

TEST INFRASTRUCTURE: the checker the GPU library is compared against.  It shares
no code with the CUDA path.  Only tests, the smoke check and the CPU-baseline leg
of the benchmark use it.

Every function takes a parameter dict with the problem statement of the paper's
Supplementary Material (Eqs. S.1-S.4): nx, ny, xlen, ylen, dt, wx, wy, c0, c2,
omeg, so_type (0 none, 1 Rashba, 2 Dresselhaus), gamma, rabi; and psi as a
complex128 array of shape (3, ny, nx) (components m_F = +1, 0, -1).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_LIB = os.path.join(_HERE, "libgporacle.so")

IMAG, REAL = 0, 1


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("xlen", ctypes.c_double), ("ylen", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("wx", ctypes.c_double), ("wy", ctypes.c_double),
        ("c0", ctypes.c_double), ("c2", ctypes.c_double), ("omeg", ctypes.c_double),
        ("so_type", ctypes.c_int),
        ("gamma", ctypes.c_double), ("rabi", ctypes.c_double),
    ]


def build(force=False):
    """Compile gp_oracle.c with gcc (plain C99, no fast-math, no FMA contraction),
    with OpenMP over grid lines where the compiler supports it."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-o", _LIB + ".tmp", _SRC, "-lm"]
    if subprocess.run(base + ["-fopenmp"], capture_output=True).returncode != 0:
        subprocess.run(base, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        cp = ctypes.POINTER(_Params)
        dp = ctypes.POINTER(ctypes.c_double)
        for name in ("orc_substep_p", "orc_substep_x", "orc_substep_y", "orc_step"):
            fn = getattr(lib, name)
            fn.argtypes = [cp, dp, ctypes.c_int]
            fn.restype = ctypes.c_int
        lib.orc_propagate.argtypes = [cp, dp, ctypes.c_longlong, ctypes.c_int]
        lib.orc_propagate.restype = ctypes.c_int
        lib.orc_propagate_strang.argtypes = [cp, dp, ctypes.c_longlong, ctypes.c_int]
        lib.orc_propagate_strang.restype = ctypes.c_int
        lib.orc_normalize_m.argtypes = [cp, dp, ctypes.c_double]
        lib.orc_normalize_m.restype = ctypes.c_int
        lib.orc_step_m.argtypes = [cp, dp, ctypes.c_double]
        lib.orc_step_m.restype = ctypes.c_int
        lib.orc_normalize.argtypes = [cp, dp]
        lib.orc_normalize.restype = ctypes.c_int
        lib.orc_norm.argtypes = [cp, dp]
        lib.orc_norm.restype = ctypes.c_double
        lib.orc_observables.argtypes = [cp, dp, dp]
        lib.orc_observables.restype = ctypes.c_int
        lib.orc_interaction_constants.argtypes = [ctypes.c_double] * 4 + [dp]
        lib.orc_interaction_constants.restype = None
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def set_threads(n):
    """Threads over grid lines in the substeps (results are bitwise the same for
    every count); returns the count in effect.  n <= 0 only queries it."""
    return int(_load().orc_set_threads(int(n)))


DEFAULTS = dict(wx=1.0, wy=1.0, c0=0.0, c2=0.0, omeg=0.0, so_type=0, gamma=0.0, rabi=0.0)


def _params(p):
    q = dict(DEFAULTS)
    q.update(p)
    return _Params(int(q["nx"]), int(q["ny"]), float(q["xlen"]), float(q["ylen"]), float(q["dt"]),
                   float(q["wx"]), float(q["wy"]), float(q["c0"]), float(q["c2"]), float(q["omeg"]),
                   int(q["so_type"]), float(q["gamma"]), float(q["rabi"]))


def _buf(psi, p):
    a = np.ascontiguousarray(psi, dtype=np.complex128)
    if a.shape != (3, int(p["ny"]), int(p["nx"])):
        raise ValueError(f"psi must have shape (3, ny, nx), got {a.shape}")
    return a.copy()


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != 0:
        raise OracleError(f"{what} failed with status {st}")


def substep(p, psi, which, mode):
    """Apply one substep ('P', 'X' or 'Y') and return the new psi."""
    a = _buf(psi, p)
    fn = {"P": "orc_substep_p", "X": "orc_substep_x", "Y": "orc_substep_y"}[which]
    _check(getattr(_load(), fn)(ctypes.byref(_params(p)), _ptr(a), int(mode)), fn)
    return a


def step(p, psi, mode):
    a = _buf(psi, p)
    _check(_load().orc_step(ctypes.byref(_params(p)), _ptr(a), int(mode)), "orc_step")
    return a


def propagate(p, psi, nsteps, mode):
    a = _buf(psi, p)
    _check(_load().orc_propagate(ctypes.byref(_params(p)), _ptr(a), int(nsteps), int(mode)), "orc_propagate")
    return a


def propagate_strang(p, psi, nsteps, mode):
    """nsteps second-order (Strang) steps: P(dt/2) X(dt/2) Y(dt) X(dt/2) P(dt/2)."""
    a = _buf(psi, p)
    _check(_load().orc_propagate_strang(ctypes.byref(_params(p)), _ptr(a), int(nsteps), int(mode)),
           "orc_propagate_strang")
    return a


def normalize(p, psi):
    a = _buf(psi, p)
    _check(_load().orc_normalize(ctypes.byref(_params(p)), _ptr(a)), "orc_normalize")
    return a


def normalize_m(p, psi, m):
    """Magnetisation-constrained normalisation: N = 1 and N+ - N- = m."""
    a = _buf(psi, p)
    _check(_load().orc_normalize_m(ctypes.byref(_params(p)), _ptr(a), float(m)), "orc_normalize_m")
    return a


def propagate_m(p, psi, nsteps, m):
    """Imaginary-time steps with the magnetisation-constrained normalisation (gamma = R = 0)."""
    a = _buf(psi, p)
    for _ in range(int(nsteps)):
        _check(_load().orc_step_m(ctypes.byref(_params(p)), _ptr(a), float(m)), "orc_step_m")
    return a


def observables(p, psi):
    """dict with norm (3,), norm_total, magnetization, energy, mu."""
    a = _buf(psi, p)
    out = np.zeros(7)
    _check(_load().orc_observables(ctypes.byref(_params(p)), _ptr(a), _ptr(out)), "orc_observables")
    return dict(norm=out[:3].copy(), norm_total=out[3], magnetization=out[4], energy=out[5], mu=out[6])


def interaction_constants(natoms, a0, a2, l0_over_sqrt_kappa):
    """(c0, c2) of Eq. (S.4) for lengths given in one common unit."""
    out = np.zeros(2)
    _load().orc_interaction_constants(float(natoms), float(a0), float(a2), float(l0_over_sqrt_kappa), _ptr(out))
    return float(out[0]), float(out[1])


def grid(p):
    """Cell-centred coordinates (x, y) of the grid reading."""
    nx, ny = int(p["nx"]), int(p["ny"])
    dx, dy = p["xlen"] / nx, p["ylen"] / ny
    x = -0.5 * p["xlen"] + (np.arange(nx) + 0.5) * dx
    y = -0.5 * p["ylen"] + (np.arange(ny) + 0.5) * dy
    return x, y
