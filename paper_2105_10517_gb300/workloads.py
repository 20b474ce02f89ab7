"""Full-size runs of the synthetic workloads, each printing one JSON report.

  python -m paper_2105_10517_gb300.workloads vortex512      # 512^2, 20000 imaginary-time steps, Rashba at +Omega
                                                            # and Dresselhaus at -Omega from the mirrored state
  python -m paper_2105_10517_gb300.workloads quench1024     # 1024^2 ground state, then an Omega quench and
                                                            # 10000 real-time steps: norm and magnetisation drift
  python -m paper_2105_10517_gb300.workloads precision2048  # 2048^2: FP32 storage then an FP64 refinement block
                                                            # against an all-FP64 run from the same seed
  python -m paper_2105_10517_gb300.workloads figs1_ferro    # the Fig. S1 procedure: Omega = 0 ground state from the
  python -m paper_2105_10517_gb300.workloads figs1_antiferro  # centre-vortex guess, continued to Omega = 0.3, then
                                                            # 50 time units of real time from that ground state

Every step runs in the CUDA library; this module only sequences the calls and
computes summary numbers of the fetched states (vortex counts, errors).
"""
import argparse
import json
import sys
import time

import numpy as np

from . import diagnostics, gpspin, inputs


def _obs(s):
    o = s.observables()
    return {k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in o.items()}


def vortex512(steps=None):
    c = inputs.CONFIGS["vortex512"]
    p = inputs.physics(c)
    n = steps or c["steps"]
    psi0 = inputs.gaussian_state(p["nx"], p["ny"], p["xlen"], p["ylen"], seed=c["seed"])
    out = {"workload": "vortex512", "steps": n}
    t = time.perf_counter()
    with gpspin.Solver(dict(p, so_type=1, omeg=0.8)) as r, gpspin.Solver(dict(p, so_type=2, omeg=-0.8)) as d:
        r.set_state(psi0)
        d.set_state(psi0[:, ::-1, :].copy())
        r.propagate(n, gpspin.IMAG)
        d.propagate(n, gpspin.IMAG)
        pr, pd = r.get_state(), d.get_state()
        out["rashba"] = _obs(r)
        out["dresselhaus_mirrored"] = _obs(d)
    out["wall_s"] = time.perf_counter() - t
    out["max_abs_psiD_minus_mirror_psiR"] = float(np.max(np.abs(pd - pr[:, ::-1, :])))
    out["rel_dE_R_vs_D"] = abs(out["rashba"]["energy"] - out["dresselhaus_mirrored"]["energy"]) / \
        abs(out["rashba"]["energy"])
    out["vortices_rashba"] = diagnostics.vortex_counts(pr)
    out["vortices_dresselhaus"] = diagnostics.vortex_counts(pd)
    return out


def imag_to_convergence(s, cap, tol=1e-9, block=100):
    """Imaginary time in blocks until |E_k - E_{k-1}| < tol between blocks or
    `cap` steps; returns (steps, converged)."""
    e_last, k = None, 0
    while k < cap:
        s.propagate(block, gpspin.IMAG)
        k += block
        e = s.observables()["energy"]
        if e_last is not None and abs(e - e_last) < tol:
            return k, True
        e_last = e
    return k, False


# Fig. S1 (Supplementary Material) and the text after it: gamma = 0.5, Omega = 0.3,
# the two condensates of the interaction-constant paragraph (labels as in that
# paragraph: 87Rb c2 < 0 ferromagnetic, 23Na c2 > 0 antiferromagnetic), DX = 0.1,
# DT = 0.1 DX^2 in imaginary and 0.025 DX^2 in real time, 50 time units of real
# time.  Centre charges of the non-rotating SO-coupled ground states, upper sign
# Rashba: (-+1, 0, +-1) antiferromagnetic, (0, +-1, +-2) ferromagnetic.
FIGS1 = {
    "ferro": dict(c0=669.0, c2=-3.1, winding={1: (0, 1, 2), 2: (0, -1, -2)}),
    "antiferro": dict(c0=482.0, c2=15.0, winding={1: (-1, 0, 1), 2: (1, 0, -1)}),
}


def figs1(kind="ferro", so_type=1, n=256, dx=0.1, omega=0.3, gamma=0.5, imag_cap=100000, tol=1e-9,
          real_time=50.0, report_every=10.0):
    """The Fig. S1 procedure, Omega-continuation included.

    1. Imaginary time at Omega = 0 from the centre-vortex initial guess, to
       convergence.
    2. Imaginary time at Omega = 0.3 (-0.3 for Dresselhaus, the mirror
       statement), continued from stage 1's state.
    3. Real time for `real_time` units from stage 2's ground state.

    Reports E, mu, the centre charges and the vortex counts of every stage, and
    the norm and magnetisation drift of stage 3.  Qualitative: the figure's
    densities are not in the paper text."""
    cfg = FIGS1[kind]
    length = n * dx
    dt_imag, dt_real = 0.1 * dx * dx, 0.025 * dx * dx
    om = omega if so_type == 1 else -omega
    p = dict(nx=n, ny=n, xlen=length, ylen=length, dt=dt_imag, c0=cfg["c0"], c2=cfg["c2"], omeg=0.0,
             so_type=so_type, gamma=gamma, rabi=0.0)
    x, y = inputs.grid(n, n, length, length)
    out = {"workload": "figs1_" + kind, "so_type": so_type, "n": n, "dx": dx, "gamma": gamma, "omega": om}

    def stage(s):
        psi = s.get_state()
        return dict(_obs(s), centre_charges=[diagnostics.central_winding(psi[c], x, y, 1.5) for c in range(3)],
                    vortices=diagnostics.vortex_counts(psi))

    t = time.perf_counter()
    with gpspin.Solver(p) as s:
        s.init_winding((1 / 3, 1 / 3, 1 / 3), winding=cfg["winding"][so_type], seed=3, phase_noise=1e-3)
        k, conv = imag_to_convergence(s, imag_cap, tol)
        out["omega0"] = dict(stage(s), imag_steps=k, converged=conv)
        s.set_params(dict(p, omeg=om))
        k, conv = imag_to_convergence(s, imag_cap, tol)
        out["omega_rot"] = dict(stage(s), imag_steps=k, converged=conv)
        s.set_params(dict(p, omeg=om, dt=dt_real))
        o0 = s.observables()
        blk = int(round(report_every / dt_real))
        drift = []
        for b in range(int(round(real_time / report_every))):
            s.propagate(blk, gpspin.REAL)
            o = s.observables()
            drift.append(dict(time=(b + 1) * report_every, norm_drift=o["norm_total"] - o0["norm_total"],
                              magnetization=o["magnetization"], energy=o["energy"]))
        out["real_time"] = drift
        out["real_final"] = stage(s)
    out["wall_s"] = time.perf_counter() - t
    return out


def quench1024(imag_cap=20000, tol=1e-9, real_steps=None):
    c = inputs.CONFIGS["quench1024"]
    p = inputs.physics(c)
    n_real = real_steps or c["steps"]
    out = {"workload": "quench1024"}
    t = time.perf_counter()
    with gpspin.Solver(p) as s:
        s.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
        k, conv = imag_to_convergence(s, imag_cap, tol)
        out["ground_state"] = dict(_obs(s), imag_steps=k, converged=conv)
        s.set_params(dict(p, omeg=0.9))  # the quench: tables are rebuilt
        o0 = s.observables()
        drift = []
        for blk in range(n_real // 1000):
            s.propagate(1000, gpspin.REAL)
            o = s.observables()
            drift.append(dict(step=(blk + 1) * 1000, norm_drift=o["norm_total"] - o0["norm_total"],
                              magnetization=o["magnetization"], energy=o["energy"]))
        out["real_time"] = drift
        out["max_abs_norm_drift"] = max(abs(d["norm_drift"]) for d in drift) if drift else 0.0
        out["vortices_final"] = diagnostics.vortex_counts(s.get_state())
    out["wall_s"] = time.perf_counter() - t
    return out


def precision2048(fp32_steps=38000, fp64_steps=2000, checkpoint=4000):
    c = inputs.CONFIGS["precision2048"]
    p = inputs.physics(c)
    out = {"workload": "precision2048", "fp32_steps": fp32_steps, "fp64_refine_steps": fp64_steps}

    def run(solver, steps, energies, refine=0):
        # checkpoints every `checkpoint` steps: where the two trajectories part
        done = 0
        while done < steps:
            k = min(checkpoint, steps - done)
            solver.propagate(k, gpspin.IMAG)
            done += k
            energies.append(solver.observables()["energy"])
        if refine:
            solver.refine_fp64(refine, gpspin.IMAG)
            energies.append(solver.observables()["energy"])

    em, ef = [], []
    t = time.perf_counter()
    with gpspin.Solver(dict(p, precision=gpspin.FP32_MIXED)) as m:
        m.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
        run(m, fp32_steps, em, refine=fp64_steps)
        pm = m.get_state()
        out["mixed"] = _obs(m)
    out["mixed_wall_s"] = time.perf_counter() - t
    t = time.perf_counter()
    with gpspin.Solver(dict(p, precision=gpspin.FP64)) as f:
        f.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
        run(f, fp32_steps, ef)
        f.propagate(fp64_steps, gpspin.IMAG)
        ef.append(f.observables()["energy"])
        pf = f.get_state()
        out["fp64"] = _obs(f)
    out["fp64_wall_s"] = time.perf_counter() - t
    steps = [min((i + 1) * checkpoint, fp32_steps) for i in range(len(em) - 1)] + [fp32_steps + fp64_steps]
    out["rel_dE_by_step"] = [dict(step=k, rel_dE=abs(a - b) / abs(b)) for k, a, b in zip(steps, em, ef)]
    # Control: FP64 again, from the initial state rounded to complex64 (the
    # only difference the FP32 run starts with).  If its energy parts from the
    # FP64 run as the mixed run's does, the gap comes from the sensitivity of the
    # vortex nucleation to the initial state, not from error in the FP32 steps.
    ep = []
    with gpspin.Solver(dict(p, precision=gpspin.FP64)) as g:
        g.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
        psi0 = g.get_state()
        g.set_state(psi0.astype(np.complex64).astype(np.complex128), normalize=True)
        run(g, 2 * checkpoint, ep)
    out["fp64_from_fp32_rounded_state_rel_dE_by_step"] = [
        dict(step=(i + 1) * checkpoint, rel_dE=abs(a - b) / abs(b)) for i, (a, b) in enumerate(zip(ep, ef))]
    # Control without rotation (Omega = 0: no vortex nucleation to amplify the
    # rounding of every step): the FP32 steps against FP64 on the same grid.
    e32, e64 = [], []
    for prec, acc in ((gpspin.FP32_MIXED, e32), (gpspin.FP64, e64)):
        with gpspin.Solver(dict(p, omeg=0.0, precision=prec)) as g:
            g.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
            run(g, 2 * checkpoint, acc)
    out["no_rotation_fp32_vs_fp64_rel_dE_by_step"] = [
        dict(step=(i + 1) * checkpoint, rel_dE=abs(a - b) / abs(b)) for i, (a, b) in enumerate(zip(e32, e64))]
    out["rel_dE"] = abs(out["mixed"]["energy"] - out["fp64"]["energy"]) / abs(out["fp64"]["energy"])
    out["rel_dmu"] = abs(out["mixed"]["mu"] - out["fp64"]["mu"]) / abs(out["fp64"]["mu"])
    rm, rf = np.abs(pm) ** 2, np.abs(pf) ** 2
    out["density_rel_l2_error"] = [float(np.linalg.norm(rm[c_] - rf[c_]) / np.linalg.norm(rf[c_])) for c_ in range(3)]
    out["vortices_mixed"] = diagnostics.vortex_counts(pm)
    out["vortices_fp64"] = diagnostics.vortex_counts(pf)
    return out


RUNS = {"vortex512": vortex512, "quench1024": quench1024, "precision2048": precision2048,
        "figs1_ferro": lambda: figs1("ferro"), "figs1_antiferro": lambda: figs1("antiferro")}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("workload", choices=sorted(RUNS))
    args = ap.parse_args(argv)
    gpspin.build()
    print(json.dumps(RUNS[args.workload]()))


if __name__ == "__main__":
    sys.exit(main())
