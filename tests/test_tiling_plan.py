"""Host logic of the line-pass tilings, checked on the CPU through gp_plan_tiling
(no device needed).

* The fixup length F: the Thomas recurrence c'_k = gamma' / (beta - alpha c'_{k-1})
  of every line and spin channel is iterated here to its limit.  F must make
  |c'_inf|^F reach the precision's threshold (2^-60 for complex128, 2^-26 for
  complex64) and be the smallest such length plus one row of margin.
* The recurrence must have converged, to the precision's rounding, within the
  first chunk, so later chunks may use the converged coefficients.
* The launch shape fits the hardware: threads a multiple of 32 and at most 512
  covering one thread per chunk and line-channel; shared memory within 227 KB; the
  chunks cover the line; the one-array (register-resident) layout only for
  complex64 chunk lengths 16, 24, 32 with 16-byte aligned strides.
* The bank-conflict count that the library reports for the solve's
  chunk-parallel accesses is recounted here from the addresses."""
import numpy as np
import pytest

from paper_2105_10517_gb300 import gpspin, inputs

CASES = [(wl, prec, mode) for wl in ("small64", "vortex512", "quench1024", "precision2048")
         for prec in (gpspin.FP64, gpspin.FP32_MIXED) for mode in (gpspin.IMAG, gpspin.REAL)]
CASES += [("serve", prec, gpspin.IMAG) for prec in (gpspin.FP64, gpspin.FP32_MIXED)]


def case_params(wl, prec):
    if wl == "serve":  # a serving-trace-like request: 384^2, DX = 32/N, DT = 0.1 DX^2
        n = 384
        dx = 32.0 / n
        return dict(nx=n, ny=n, xlen=32.0, ylen=32.0, dt=0.1 * dx * dx, c0=400.0, c2=12.0, omeg=0.7, so_type=2,
                    gamma=1.6, rabi=0.8, precision=prec)
    return dict(inputs.physics(inputs.CONFIGS[wl]), precision=prec)


def line_systems(p, d, mode):
    """alpha, beta, gamma' of I + tau A for every line and channel of direction d
    (reading 4-6: A = -1/2 D2 + i kb D1, central differences)."""
    nx, ny = p["nx"], p["ny"]
    h = p["xlen"] / nx if d == 0 else p["ylen"] / ny
    nl, length = (ny, p["ylen"]) if d == 0 else (nx, p["xlen"])
    pos = -0.5 * length + (np.arange(nl) + 0.5) * length / nl
    lam = np.array([1.0, 0.0, -1.0])
    gam = p.get("gamma", 0.0) if p.get("so_type", 0) else 0.0
    eta = {1: 1.0, 2: -1.0}.get(p.get("so_type", 0), 0.0)
    om = p.get("omeg", 0.0)
    kb = (gam * lam[None, :] - om * pos[:, None]) if d == 0 else (om * pos[:, None] - eta * gam * lam[None, :])
    tau = 0.5j * p["dt"] if mode == gpspin.REAL else 0.5 * p["dt"]
    a = tau * (-0.5 / h**2 - 1j * kb / (2 * h))
    c = tau * (-0.5 / h**2 + 1j * kb / (2 * h))
    b = 1.0 + tau / h**2 + 0 * kb
    return a.ravel(), np.broadcast_to(b, kb.shape).ravel(), c.ravel()


def recurrence(a, b, c, rows):
    cp = np.zeros_like(a)
    out = []
    for _ in range(rows):
        cp = c / (b - a * cp)
        out.append(cp.copy())
    return np.array(out)


@pytest.mark.parametrize("wl,prec,mode", CASES)
def test_plan_tiling(wl, prec, mode):
    p = case_params(wl, prec)
    plan = gpspin.plan_tiling(p, mode)
    bits = 26 if prec == gpspin.FP32_MIXED else 60
    for d, name in ((0, "xpass"), (1, "ypass")):
        t = plan[name]
        L, nl = (p["nx"], p["ny"]) if d == 0 else (p["ny"], p["nx"])
        a, b, c = line_systems(p, d, mode)
        seq = recurrence(a, b, c, 400)
        cinf = seq[-1]
        r = np.max(np.abs(cinf))
        # fixup length: sufficient, and minimal up to one row of margin
        F, m = t["fixup"], t["chunk"]
        assert r ** F <= 2.0 ** -bits
        assert F < 3 or r ** (F - 2) > 2.0 ** -bits
        # the factorisation has converged to rounding by row m - F (>= H rows),
        # so the chunks after the first may use the converged coefficients; the
        # FP64 floor is the rounding noise of the iteration itself (a few ulps)
        err = np.max(np.abs(seq[m - F] - cinf) / np.abs(cinf))
        assert err <= max(2.0 ** -bits, 8 * 2.0 ** -53)
        # launch shape
        S, R, Q = t["cluster"], t["lines_per_cta"], t["chunks"]
        Qc = -(-Q // S)
        assert Q == -(-L // m) and m >= 16
        assert t["threads"] % 32 == 0 and 3 * R * Qc <= t["threads"] <= 512
        assert t["smem"] <= 227 * 1024 and 1 <= R <= nl
        assert t["ctas"] == -(-nl // R) * S
        assert S == (2 if (L >= 256 and Q >= 8) else 1)
        cs, Lp = t["chunk_stride"], t["line_stride"]
        assert cs >= m and Lp >= Qc * cs
        if t["register_solve"]:
            assert prec == gpspin.FP32_MIXED and m in (16, 24, 32)
            assert cs % 2 == 0 and Lp % 2 == 0  # chunk slots start on 16-byte boundaries
        # bank conflicts of one round of chunk-parallel accesses (thread tid =
        # chunk * 3R + line-channel at element lc Lp + chunk cs), recounted
        unit, G = (2, 8) if t["register_solve"] else (1, 8 if prec == gpspin.FP64 else 16)
        n = 3 * R * Qc
        tid = np.arange(n)
        ql, lc = tid // (3 * R), tid % (3 * R)
        bank = ((lc * Lp + ql * cs) // unit) % G
        extra = sum(np.bincount(bank[g:g + G], minlength=G).max() - 1 for g in range(0, n, G))
        assert extra == t["bank_conflicts"]


def test_plan_rejects_what_create_rejects():
    p = dict(nx=16, ny=16, xlen=8.0, ylen=8.0, dt=0.01)
    with pytest.raises(gpspin.GPError):
        gpspin.plan_tiling(dict(p, nx=3))
    # |c'_inf| >= 1/2 (dt/h^2 far beyond the workloads): outside the tabulated solver
    with pytest.raises(gpspin.GPError):
        gpspin.plan_tiling(dict(p, dt=50.0))


@pytest.mark.parametrize("mode", [gpspin.IMAG, gpspin.REAL])
def test_supported_range_boundary(mode):
    """The tabulated solver supports the systems whose Thomas recurrence contracts
    by |c'_inf| < 1/2 (the chunk fixups then reach the rounding level within the
    fixup table); beyond it gp_plan_tiling, like gp_create's first propagate,
    refuses with GP_ERR_UNSUPPORTED.  The limit |c'_inf| is computed here
    independently, by iterating the recurrence, on both sides of the boundary
    in dt/h^2."""
    base = dict(nx=64, ny=64, xlen=16.0, ylen=16.0, c0=50.0, c2=-2.0, omeg=0.3, so_type=1, gamma=0.4, rabi=0.1)
    h2 = (16.0 / 64) ** 2
    seen = set()
    for r in np.geomspace(0.5, 40.0, 60):  # dt / h^2
        p = dict(base, dt=r * h2)
        cmax = 0.0
        for d in (0, 1):
            a, b, c = line_systems(p, d, mode)
            cmax = max(cmax, float(np.max(np.abs(recurrence(a, b, c, 2000)[-1]))))
        try:
            gpspin.plan_tiling(p, mode)
            ok = True
        except gpspin.GPError as e:
            assert e.status == 5  # GP_ERR_UNSUPPORTED
            ok = False
        if abs(cmax - 0.5) > 1e-3:  # away from the boundary itself, where rounding may decide
            assert ok == (cmax < 0.5), (r, cmax, ok)
        seen.add(ok)
    assert seen == {True, False}  # the sweep crosses the boundary
