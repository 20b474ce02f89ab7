"""Full-size runs of the synthetic workloads, each printing one JSON report.

  python -m paper_2105_10517_gb300.workloads vortex512      # 512^2, 20000 imaginary-time steps, Rashba at +Omega
                                                            # and Dresselhaus at -Omega from the mirrored state
  python -m paper_2105_10517_gb300.workloads quench1024     # 1024^2 ground state, then an Omega quench and
                                                            # 10000 real-time steps: norm and magnetisation drift
  python -m paper_2105_10517_gb300.workloads precision2048  # 2048^2: FP32 storage then an FP64 refinement block
                                                            # against an all-FP64 run from the same seed

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


def quench1024(imag_cap=20000, tol=1e-9, real_steps=None):
    c = inputs.CONFIGS["quench1024"]
    p = inputs.physics(c)
    n_real = real_steps or c["steps"]
    out = {"workload": "quench1024"}
    t = time.perf_counter()
    with gpspin.Solver(p) as s:
        s.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
        e_last, k = None, 0
        while k < imag_cap:
            s.propagate(100, gpspin.IMAG)
            k += 100
            e = s.observables()["energy"]
            if e_last is not None and abs(e - e_last) < tol:
                break
            e_last = e
        out["ground_state"] = dict(_obs(s), imag_steps=k, converged=k < imag_cap)
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


def precision2048(fp32_steps=38000, fp64_steps=2000):
    c = inputs.CONFIGS["precision2048"]
    p = inputs.physics(c)
    out = {"workload": "precision2048", "fp32_steps": fp32_steps, "fp64_refine_steps": fp64_steps}
    t = time.perf_counter()
    with gpspin.Solver(dict(p, precision=gpspin.FP32_MIXED)) as m:
        m.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
        m.propagate(fp32_steps, gpspin.IMAG)
        m.refine_fp64(fp64_steps, gpspin.IMAG)
        pm = m.get_state()
        out["mixed"] = _obs(m)
    out["mixed_wall_s"] = time.perf_counter() - t
    t = time.perf_counter()
    with gpspin.Solver(dict(p, precision=gpspin.FP64)) as f:
        f.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
        f.propagate(fp32_steps + fp64_steps, gpspin.IMAG)
        pf = f.get_state()
        out["fp64"] = _obs(f)
    out["fp64_wall_s"] = time.perf_counter() - t
    out["rel_dE"] = abs(out["mixed"]["energy"] - out["fp64"]["energy"]) / abs(out["fp64"]["energy"])
    out["rel_dmu"] = abs(out["mixed"]["mu"] - out["fp64"]["mu"]) / abs(out["fp64"]["mu"])
    rm, rf = np.abs(pm) ** 2, np.abs(pf) ** 2
    out["density_rel_l2_error"] = [float(np.linalg.norm(rm[c_] - rf[c_]) / np.linalg.norm(rf[c_])) for c_ in range(3)]
    out["vortices_mixed"] = diagnostics.vortex_counts(pm)
    out["vortices_fp64"] = diagnostics.vortex_counts(pf)
    return out


RUNS = {"vortex512": vortex512, "quench1024": quench1024, "precision2048": precision2048}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("workload", choices=sorted(RUNS))
    args = ap.parse_args(argv)
    gpspin.build()
    print(json.dumps(RUNS[args.workload]()))


if __name__ == "__main__":
    sys.exit(main())
