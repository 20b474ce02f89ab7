#!/usr/bin/env python3
"""Benchmark of the split-step Crank-Nicolson step (one JSON line on rank 0).

A bench step is one time step of the whole hot path.  The default workload is
the 1024 x 1024 real-time run ([-20,20]^2, dt = 5e-4, c0 = 800, c2 = 15,
Dresselhaus gamma = 0.75, R = 0.5): the seeded Gaussian initial state is first
relaxed by imaginary-time steps at Omega = 0.6 (untimed), Omega is then quenched
to 0.9 (the tables are rebuilt) and the real-time steps -- pointwise substep P,
X sweep, Y sweep -- are timed in FP64.  The metric is site-steps per second (one
grid point advanced one full step, all three components).  The same line carries
the 2048 x 2048 FP32-storage step (the HBM-bound form) and the 512 x 512 FP64
imaginary-time step as extra keys.

  python bench.py [--gpus N --steps K --warmup W]   the CUDA path (C ABI)
  python bench.py --impl reference ...              the FP64 CPU oracle

Under torchrun (N > 1) the path does not shard: every rank advances its own
replica (weak scaling), and the value is all ranks' site-steps over the slowest
rank's time.  The reference arm runs on rank 0 only.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Msite-steps/s & %HBM peak; served solves/s, p50/p99 vs plain FP64 at ΔE/E≤1e-6"
UNIT = "Msite-steps/s"
WORKLOAD = "quench1024"
# Workloads whose timed steps follow an untimed preparation: imaginary-time steps
# from the seeded Gaussian state, then new parameters (the Omega quench).
PREP = {"quench1024": dict(imag_steps=4000, quench=dict(omeg=0.9))}
# Extra lines measured after the main one (N = 1 only): workload, storage, steps.
EXTRAS = (("precision2048", "fp32", 1500), ("vortex512", "fp64", 1500))

# Roofline of the FP64 path: it is bound by FP64 issue, not HBM.  GB300 retires
# 2 FP64 FMA lanes per SM per clock (measured 1.2 TFLOP/s, rate independent of
# how many lanes of a warp are active): 2 lanes x 2 flop x 152 SMs x 2.07 GHz.
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12
# Algorithmic FP64 flops per site (FMA = 2) of the two line passes in imaginary
# time, small-argument branches (dt^2|B|^2 <= 1e-4, dt c0 rho <= 1/64), counted
# from the kernel arithmetic, without the chunk fixups of the parallel solve.
# In imaginary time the Thomas pivots are real, so a channel point costs 22 flops:
# forward 2 (real scaling) + 8, back substitution 8, psi' = 2w - phi 4.
#   x-pass: P 156 (63 FMA, 27 MUL, 3 ADD) + U_y^dag 16 + Thomas 3 x 22 + U_x^dag U_y 14
#   y-pass: Thomas 3 x 22 + U_x 16 + |psi|^2 partial sums 12
FLOPS_PER_SITE = {"xpass": 252, "ypass": 94}
INST_PER_SITE = {"xpass": 155, "ypass": 57}
# Real time, same counting (dt c0 rho <= 1/64): the Thomas pivots are complex (26
# flops, 14 instructions per channel point: forward cmul + cfnma, back cfnma,
# 2w - phi), and P applies exp(-i dt (V + c0 rho)) as a complex phase (cis
# series of four terms each, trap factor product, three complex products) and
# has no partial norms.
#   x-pass: P 182 (73 FMA, 33 MUL, 3 ADD; 109 instructions) + U_y^dag 16 (12)
#           + Thomas 3 x 26 (3 x 14) + U_x^dag U_y 14 (14)
#   y-pass: Thomas 3 x 26 (3 x 14) + U_x 16 (12)
FLOPS_PER_SITE_REAL = {"xpass": 290, "ypass": 94}
INST_PER_SITE_REAL = {"xpass": 177, "ypass": 54}
# Closing x-pass of a second-order (Strang) step, same counting: U_y^dag with the
# scale 18 + Thomas 3 x 22 + U_y 14 + P 160 (applied after the solve, with its
# scale) + |psi|^2 partial sums 12.
FLOPS_XTAIL = 270
# Algorithmic HBM bytes per site and pass: read and write 3 complex128 values.
BYTES_PER_SITE_PASS = 96
# DRAM traffic of one launch (dram__bytes_read.sum + dram__bytes_write.sum from
# one ncu capture of that kernel), keyed by kernel and workload and valid only
# while the kernel source is unchanged (sha256 prefix).
NCU_TRAFFIC = {
    "xpass_kernel<1, double2> quench1024": (57513728 + 9970688, "9cd44b01d8d15a4c"),
    "ypass_kernel_reg<1, double2, 32> quench1024": (57548800 + 6869760, "9cd44b01d8d15a4c"),
    "xpass_kernel<0, double2> vortex512": (16203264 + 0, "9cd44b01d8d15a4c"),
    "ypass_kernel<0, double2> vortex512": (16172288 + 0, "9cd44b01d8d15a4c"),
    "xpass_kernel_reg<0, float2, 32> precision2048": (105457664 + 56003072, "9cd44b01d8d15a4c"),
    "ypass_kernel_reg<0, float2, 32> precision2048": (105457920 + 57491456, "9cd44b01d8d15a4c"),
}

L2_FLUSH_BYTES = 256 << 20


def sha_kernels():
    h = hashlib.sha256()
    for f in ("gp_sweeps.cu", "gp_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2105_10517_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="seconds of oracle work per CPU-baseline leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the extra workload lines")
    ap.add_argument("--workload", default=WORKLOAD, help="quench1024 (default), vortex512, precision2048, small64")
    ap.add_argument("--prep-steps", type=int, default=None,
                    help="imaginary-time steps before the timed real-time steps (quench1024; default 4000)")
    ap.add_argument("--serve", action="store_true",
                    help="serving benchmark: the seeded request trace through the batched server and one at a time")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--cap", type=int, default=20000)
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--no-plain", action="store_true", help="serving: skip the one-at-a-time FP64 baseline")
    ap.add_argument("--max-running-sites", type=int, default=1 << 22,
                    help="serving: grid points of the solves running at once (0: admit by memory only)")
    ap.add_argument("--no-autotune", action="store_true", help="time the default tiling instead of the tuned one")
    ap.add_argument("--tiling", default=None,
                    help="S,R,m[,reg|smem]: cluster size, lines per CTA, chunk length and solve kind of both passes "
                         "(instead of autotuning); X:Y gives the x-pass and the y-pass their own")
    ap.add_argument("--substeps", action="store_true",
                    help="time split of the passes: the x- and y-pass with only P, only the X solve, only the Y "
                         "solve, then one full step (NVTX range 'substeps'); prints one JSON line")
    ap.add_argument("--splitting", default="lie", choices=["lie", "strang"],
                    help="lie: the first-order step (default); strang: the second-order extension (fp64)")
    ap.add_argument("--magnetization", type=float, default=None,
                    help="imaginary time with N+ - N- held at this value (the workload without SO and Rabi coupling)")
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32"],
                    help="storage precision (default: fp64; precision2048 defaults to fp32)")
    return ap.parse_args()


def workload(name=WORKLOAD):
    """(run-control dict, physics of the timed steps): for a prepared workload the
    physics after the quench."""
    from paper_2105_10517_gb300 import inputs
    c = dict(inputs.CONFIGS[name])
    p = inputs.physics(c)
    if name in PREP:
        p.update(PREP[name]["quench"])
    return c, p


def config_dict(c, p, name=WORKLOAD, precision="fp64", prep_steps=None):
    so = {0: "no SO", 1: "Rashba", 2: "Dresselhaus"}[p["so_type"]]
    mode = "imaginary" if c["mode"] == 0 else "real"
    half = c["xlen"] / 2
    om = f"Omega={c['omeg']}->{p['omeg']} (quench)" if p["omeg"] != c["omeg"] else f"Omega={p['omeg']}"
    out = {
        "workload": f"{name}: {c['nx']}x{c['ny']} {mode}-time, [-{half:g},{half:g}]^2, dt={c['dt']}, "
                    f"c0={p['c0']}, c2={p['c2']}, {om}, {so} gamma={p['gamma']}, R={p['rabi']}",
        "nx": c["nx"], "ny": c["ny"], "dt": c["dt"], "mode": mode, "storage": precision,
        "step": "one split-step CN time step: " + ("normalise, " if mode == "imaginary" else "")
                + "P, X sweep, Y sweep" + (", norm" if mode == "imaginary" else ""),
        "l2": "flushed by a 256 MiB device write before every timed step",
        "parallelism": "replicas",
    }
    if prep_steps:
        out["prep"] = (f"{prep_steps} untimed imaginary-time steps at Omega={c['omeg']} from the seeded Gaussian "
                       f"state, then the quench")
    return out


# ----------------------------------------------------------- rank logic ----
def max_over_ranks(x, dist, device):
    """Max of a float over all ranks (the slowest rank sets the job's time)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, sites, steps, t_max_ms):
    """Site-steps of all ranks (each advances its own replica) over the slowest
    rank's time, in Msite-steps/s."""
    return world * sites * steps / (t_max_ms / 1e3) / 1e6


# --------------------------------------------------------------- clocks ----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ our arm -----
def kernel_name(dom, mode, prec, tiles, strang):
    td = tiles[dom]
    if strang and dom == "xpass":
        return f"xpass_kernel<{mode}, double2> + xtail_kernel<{mode}> (both x-passes of a second-order step)"
    if td.get("register_solve"):
        return f"{dom}_kernel_reg<{mode}, {'float2' if prec == 'fp32' else 'double2'}, {td['chunk']}>"
    return f"{dom}_kernel<{mode}, {'float2' if prec == 'fp32' else 'double2'}>"


def roofline_of(name, prec, mode, sites, ms_x, ms_y, ms_n, ms_step, tiles, strang):
    """Roofline of the dominant kernel: FP64 ALU for complex128 storage (bound by
    FP64 issue on GB300), HBM for complex64 storage."""
    dom = "xpass" if ms_x >= ms_y else "ypass"
    ms_dom = ms_x if dom == "xpass" else ms_y
    kname = kernel_name(dom, mode, prec, tiles, strang)
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm = float(peaks["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        hbm, peaks = 6800.0, None
    tr = NCU_TRAFFIC.get(f"{kname} {name}")
    traffic = tr[0] if tr and tr[1] == sha_kernels() else None
    if prec == "fp64":
        fl = FLOPS_PER_SITE_REAL if mode == 1 else FLOPS_PER_SITE
        ins = INST_PER_SITE_REAL if mode == 1 else INST_PER_SITE
        flops = fl[dom] + (FLOPS_XTAIL if strang and dom == "xpass" else 0)
        achieved = flops * sites / (ms_dom / 1e3) / 1e12
        r = {
            "bound": "alu", "kernel": kname, "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "peak_source": "derived: 2 FP64 FMA lanes/SM/clk x 152 SMs x 2.07 GHz x 2 flop",
            "fp64_issue_frac": (None if strang and dom == "xpass" else
                                ins[dom] * sites / (ms_dom / 1e3) / (FP64_PEAK_TFLOPS / 2 * 1e12)),
            "flops_per_site": flops, "flops_per_launch": flops * sites,
        }
        bytes_site_pass = BYTES_PER_SITE_PASS
    else:
        bytes_site_pass = BYTES_PER_SITE_PASS // 2
        achieved = bytes_site_pass * sites / (ms_dom / 1e3) / 1e9
        r = {
            "bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm,
            "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "of fallback",
            "bytes_per_site": bytes_site_pass, "bytes_per_launch": bytes_site_pass * sites,
        }
    r["traffic"] = traffic
    r["kernel_ms"] = {"xpass": ms_x, "ypass": ms_y, "normalise": ms_n}
    r["step_hbm_frac_of_measured"] = bytes_site_pass * 2 * sites / (ms_step / 1e3) / 1e9 / hbm
    r["hbm_peak_gbs"] = hbm
    return r


def prepare(name, prec, stream, args, main=True):
    """A Solver on the workload's initial state, prepared and tuned (untimed)."""
    from paper_2105_10517_gb300 import gpspin
    c, p = workload(name)
    p["precision"] = gpspin.FP32_MIXED if prec == "fp32" else gpspin.FP64
    if main and args.magnetization is not None:  # m is conserved only without SO and Rabi coupling
        p.update(so_type=0, gamma=0.0, rabi=0.0)
    mode = c["mode"]
    prep_steps = None
    if name in PREP:
        prep_steps = PREP[name]["imag_steps"] if args.prep_steps is None else args.prep_steps
        s = gpspin.Solver(dict(p, omeg=c["omeg"]), stream=stream)
        s.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
        if prep_steps:
            s.propagate(prep_steps, gpspin.IMAG)
        s.set_params(p)  # the quench: tables are rebuilt for the timed physics
    else:
        s = gpspin.Solver(p, stream=stream)
        s.init_gaussian((0.25, 0.5, 0.25), seed=c["seed"], phase_noise=1e-3)
    if main and args.splitting == "strang":
        s.set_splitting(gpspin.SPLIT_STRANG)
    if main and args.magnetization is not None:
        s.set_magnetization(args.magnetization)
    tuned_ms = None
    if args.tiling:
        specs = args.tiling.split(":")
        for d in (0, 1):
            f = specs[min(d, len(specs) - 1)].split(",")
            kind = {"reg": True, "smem": False}[f[3]] if len(f) > 3 else None
            s.set_tiling(d, cluster=int(f[0]), lines_per_cta=int(f[1]), chunk=int(f[2]), mode=mode,
                         register_solve=kind)
    elif not args.no_autotune:
        tuned_ms = s.autotune(mode)  # the state is unchanged
    return s, c, p, mode, prep_steps, tuned_ms


def run_substeps(args):
    """Device time of the pass pair with only P, only the X solve or only the Y
    solve applied (gp_apply_substep), and of one full step (gp_profile_step): the
    split of a step between data movement, the pointwise substep and the solves.
    Each is the median of 30 launches after 3 warm-up ones, timed with CUDA
    events on the handle's stream; then one of each runs inside the NVTX range
    'substeps' for profilers."""
    import torch
    from paper_2105_10517_gb300 import gpspin
    gpspin.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    name = args.workload
    prec = args.precision or ("fp32" if name == "precision2048" else "fp64")
    stream = torch.cuda.Stream()
    s, c, p, mode, _, _ = prepare(name, prec, stream.cuda_stream, args)
    s.apply_substep("P", mode)  # applies a pending normalisation once
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def med(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(30):
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    out = {w: med(lambda: s.apply_substep(w, mode)) for w in ("P", "X", "Y")}
    prof = [s.profile_step(mode) for _ in range(30)]
    out["x_full"] = statistics.median(q[0] for q in prof)
    out["y_full"] = statistics.median(q[1] for q in prof)
    out["step"] = statistics.median(q[3] for q in prof)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("substeps")
    for w in ("P", "X", "Y"):
        s.apply_substep(w, mode)
    s.profile_step(mode)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    tiles = s.tiling(mode)
    s.close()
    return {"mode": "substeps", "workload": name, "storage": prec, "unit": "ms", "substep_ms": out, "tiles": tiles,
            "note": "P/X/Y: the x-pass and y-pass with only that substep applied (the others pass through)"}


def timed_steps(s, mode, steps, warmup, stream, flush, barrier, clocks=None):
    """Per-step device times (x-pass, y-pass, normalisation, step) of `steps`
    steps after `warmup` untimed ones, the L2 flushed before every step."""
    import torch
    for _ in range(max(3, warmup)):
        s.profile_step(mode)
    if clocks:
        clocks.start()
    barrier()
    t0 = time.perf_counter()
    per = []
    torch.cuda.nvtx.range_push("bench_timed")  # ncu --nvtx --nvtx-include "bench_timed/"
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        per.append(s.profile_step(mode))
    torch.cuda.nvtx.range_pop()
    barrier()
    wall = time.perf_counter() - t0
    if clocks:
        # keep the GPU busy until the sampler has seen the load a few times
        t1 = time.perf_counter()
        while len(clocks.lines) < 5 and time.perf_counter() - t1 < 3.0:
            s.propagate(20, mode)
        clocks.stop()
    return per, wall


def run_ours(args):
    import numpy as np
    import torch
    from paper_2105_10517_gb300 import gpspin, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    gpspin.build()
    name = args.workload
    prec = args.precision or ("fp32" if name == "precision2048" else "fp64")
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
            torch.cuda.synchronize()

    s, c, p, mode, prep_steps, tuned_ms = prepare(name, prec, stream.cuda_stream, args)
    sites = c["nx"] * c["ny"]
    tiles = s.tiling(mode)
    clocks = ClockSampler(local)
    per, wall = timed_steps(s, mode, args.steps, args.warmup, stream, flush, barrier, clocks)
    ms_x = statistics.fmean(q[0] for q in per)
    ms_y = statistics.fmean(q[1] for q in per)
    ms_n = statistics.fmean(q[2] for q in per)
    ms_step = statistics.fmean(q[3] for q in per)
    t_max = max_over_ranks(ms_step * args.steps, dist, "cuda")
    value = whole_job_value(world, sites, args.steps, t_max)
    strang = args.splitting == "strang"
    roofline = roofline_of(name, prec, mode, sites, ms_x, ms_y, ms_n, ms_step, tiles, strang)

    # end to end through the public API with pinned host buffers (the timed
    # physics, starting from the prepared state)
    e2e = None
    if args.e2e_steps > 0:
        hin = torch.from_numpy(s.get_state()).pin_memory()
        hout = torch.empty_like(hin).pin_memory()

        def one_call(a, b):
            s.propagate_host(a, 1, mode, out=b)

        def three_calls(a, b):
            s.set_state(a)
            s.propagate(1, mode)
            s.get_state(b)

        def timed(step):
            for _ in range(3):
                step(hin, hout)
            barrier()
            te = time.perf_counter()
            a, b = hin, hout
            for _ in range(args.e2e_steps):
                step(a, b)  # each step starts from the previous step's host result
                a, b = b, a
            barrier()
            return world * sites * args.e2e_steps / max_over_ranks(time.perf_counter() - te, dist, "cuda") / 1e6

        nbytes = 3 * sites * 16
        e2e = {"value": timed(one_call), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": args.e2e_steps,
               "path": "gp_propagate_host(pinned in, 1 step, pinned out) per step",
               "three_calls_value": timed(three_calls),
               "three_calls_path": "gp_set_state + gp_propagate(1) + gp_get_state per step"}
    s.close()

    # kernels of one step: x-pass, y-pass (+ the closing x-pass of a second-order
    # step) and in imaginary time the normalisation (two kernels when m is held)
    launches_per_step = 2 + (1 if strang else 0)
    if mode == gpspin.IMAG:
        launches_per_step += 2 if args.magnetization is not None else 1

    # extra lines: other workloads, each timed the same way (N = 1 only)
    extras = {}
    if world == 1 and not args.no_extras:
        for xname, xprec, xsteps in EXTRAS:
            if xname == name and xprec == prec:
                continue
            xs, xc, xp, xmode, xprep, _ = prepare(xname, xprec, stream.cuda_stream, args, main=False)
            xsites = xc["nx"] * xc["ny"]
            xtiles = xs.tiling(xmode)
            xclocks = ClockSampler(local)
            xper, _ = timed_steps(xs, xmode, xsteps, args.warmup, stream, flush, barrier, xclocks)
            xs.close()
            f = [statistics.fmean(q[k] for q in xper) for k in range(4)]
            extras[f"{xname}_{xprec}"] = {
                "value": xsites / (f[3] / 1e3) / 1e6, "unit": UNIT, "ms_per_step": f[3], "steps": xsteps,
                "dtype": "f32" if xprec == "fp32" else "f64",
                "config": dict(config_dict(xc, xp, xname, xprec, xprep), tiles=xtiles),
                "roofline": roofline_of(xname, xprec, xmode, xsites, f[0], f[1], f[2], f[3], xtiles, False),
                "gpu_launches": (2 + (1 if xmode == gpspin.IMAG else 0)) * xsteps,
                "clocks": xclocks.summary(),
            }

    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64",
            "data": "synthetic (seeded Gaussian + splitmix64 phase noise)",
            "config": dict(config_dict(c, p, name, prec, prep_steps),
                           tiling="default" if tuned_ms is None else "autotuned",
                           splitting=args.splitting, magnetization=args.magnetization, tiles=tiles),
            "roofline": roofline, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks.summary(), "wall_s_timed_loop": wall,
        }
        if extras:
            out["extra_workloads"] = extras
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out


# ----------------------------------------------------------- CPU oracle ----
def oracle_rate(p, nx, steps, seconds=None, mode=0):
    """Oracle site-steps/s on an nx x nx grid with the workload's dx, dt and physics."""
    import oracle
    from paper_2105_10517_gb300 import inputs
    dx = p["xlen"] / p["nx"]
    q = dict(p, nx=nx, ny=nx, xlen=dx * nx, ylen=dx * nx)
    psi = inputs.gaussian_state(nx, nx, q["xlen"], q["ylen"], seed=2)
    done, t0 = 0, time.perf_counter()
    while True:
        psi = oracle.step(q, psi, mode)
        done += 1
        el = time.perf_counter() - t0
        if (steps is not None and done >= steps) or (seconds is not None and el >= seconds and done >= 2):
            break
    return nx * nx * done / el, done, el


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(p, seconds, mode=0):
    """The oracle as it stands on the full workload: one leg single-threaded, one
    leg with its line loops on every host core (the paper's program is OpenMP
    over grid lines).  The all-cores leg is the reported value."""
    import oracle
    kind = "imaginary" if mode == 0 else "real"
    legs = []
    for want in (1, host_cores()):
        n = oracle.set_threads(want)
        rate, done, el = oracle_rate(p, p["nx"], None, seconds, mode)
        legs.append({"value": rate / 1e6, "unit": UNIT, "cores": n,
                     "sample": f"{done} {kind}-time steps of the full {p['nx']}x{p['ny']} workload ({el:.1f} s)"})
        if n == 1 and want > 1:
            break
    main = legs[-1]
    return {"value": main["value"], "unit": UNIT, "cores": main["cores"], "kind": "oracle",
            "sample": main["sample"] + f", C oracle with OpenMP over lines on {main['cores']} host threads",
            "legs": legs}


def run_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return None
    import oracle
    oracle.build()
    cores = oracle.set_threads(host_cores())
    c, p = workload(args.workload)
    # calibrate: size the sample grid so that warmup + steps take about two
    # minutes (on a grid large enough for the threads to have work)
    r, _, _ = oracle_rate(p, min(256, p["nx"]), 3, mode=c["mode"])
    budget = 120.0 / max(1, args.steps + args.warmup)
    n = int(max(16, min(p["nx"], math.sqrt(budget * r))))
    oracle_rate(p, n, max(1, args.warmup), mode=c["mode"])
    rate, done, el = oracle_rate(p, n, args.steps, mode=c["mode"])
    value = rate / 1e6
    sample = (f"{n}x{n} grid with the {p['nx']}x{p['ny']} workload's dx, dt and physics, "
              f"{done} timed steps after {args.warmup} warm-up steps ({el:.1f} s), "
              f"C oracle with OpenMP over lines on {cores} host threads")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / done * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Gaussian)",
        "config": config_dict(c, p, args.workload),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def run_serving(args):
    """Parameter-sweep serving: continuous batching (FP32 storage then FP64
    refinement, and FP64 throughout) against the plain one-at-a-time FP64 path
    on the same seeded trace; solves/s, p50/p99 arrival-to-converged latency and
    the energy agreement of every served result with the plain FP64 result."""
    import numpy as np
    import torch
    from paper_2105_10517_gb300 import gpspin, inputs, serve
    gpspin.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    trace = inputs.serving_trace(n=args.requests, rate=args.rate, seed=4)
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.8)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    lim = args.max_running_sites
    mixed, rm = serve.serve_batched(trace, policy=gpspin.POLICY_FP32_REFINE, max_bytes=budget, cap=args.cap,
                                    tol=args.tol, max_running_sites=lim)
    b64, rb = serve.serve_batched(trace, policy=gpspin.POLICY_FP64, max_bytes=budget, cap=args.cap, tol=args.tol,
                                  max_running_sites=lim)
    if args.no_plain:  # batched FP64 equals the plain path to rounding (tested): use it as the reference
        plain, rp = dict(b64, note="not run; batched FP64 used as the reference"), rb
    else:
        plain, rp = serve.serve_one_at_a_time(trace, cap=args.cap, tol=args.tol)
    clocks.stop()

    ref = {r["arrival"]: r for r in rp}

    def rel_de(r):
        q = ref[r["arrival"]]
        return abs(r["energy"] - q["energy"]) / abs(q["energy"])

    def agreement(ra):
        d_conv, d_cap = [], []
        for r in ra:
            q = ref[r["arrival"]]
            (d_cap if (r["steps"] >= args.cap or q["steps"] >= args.cap) else d_conv).append(rel_de(r))
        f = lambda v: {"n": len(v), "max_rel_dE": max(v) if v else None,
                       "frac_within_1e-6": (sum(x <= 1e-6 for x in v) / len(v)) if v else None}
        return {"converged": f(d_conv), "capped": f(d_cap)}

    def at_bar(summary, ra, tol=1e-6):
        """Solves/s and p50/p99 counting only results within |dE/E| <= tol of the
        plain FP64 result of the same request (the metric's accuracy bar)."""
        ok = [r for r in ra if r["state"] == gpspin.REQ_DONE and rel_de(r) <= tol]
        lat = [r["latency"] for r in ok]
        pct = lambda q: float(np.percentile(lat, q)) if lat else None
        return {"solves": len(ok), "solves_per_s": len(ok) / summary["makespan_s"], "p50_s": pct(50),
                "p99_s": pct(99), "tol_rel_dE": tol}

    paths = {"batched_mixed": (mixed, rm), "batched_fp64": (b64, rb), "plain_fp64_one_at_a_time": (plain, rp)}
    bar = {k: at_bar(v[0], v[1]) for k, v in paths.items()}
    best = max(("batched_mixed", "batched_fp64"), key=lambda k: bar[k]["solves_per_s"])
    capped = sum(1 for r in rp if r["steps"] >= args.cap)
    return {
        "metric": METRIC, "mode": "serving", "value": bar[best]["solves_per_s"], "unit": "solves/s",
        "value_path": best, "value_definition": "solves/s counting only results within |dE/E| <= 1e-6 of the "
                                                "plain one-at-a-time FP64 result of the same request",
        "higher_is_better": True, "n_gpus": 1,
        "dtype": "f32 storage + f64 refinement" if best == "batched_mixed" else "f64",
        "data": f"synthetic request trace: {args.requests} requests, Poisson arrivals at {args.rate}/s (seed 4), "
                f"N in {{128,256,384,512}}, DX=32/N, DT=0.1 DX^2, imaginary time to |dE|<{args.tol:g} per 100 "
                f"steps, cap {args.cap}",
        "plain_requests_at_cap": capped,
        "at_1e-6": bar,
        "speedup_at_1e-6_vs_plain": {k: bar[k]["solves_per_s"] / bar["plain_fp64_one_at_a_time"]["solves_per_s"]
                                     for k in ("batched_mixed", "batched_fp64")},
        "batched_mixed": mixed, "batched_fp64": b64, "plain_fp64_one_at_a_time": plain,
        "speedup_solves_per_s_vs_plain": mixed["solves_per_s"] / plain["solves_per_s"],
        "speedup_fp64_batched_vs_plain": b64["solves_per_s"] / plain["solves_per_s"],
        "energy_agreement_vs_plain_fp64": {"batched_mixed": agreement(rm), "batched_fp64": agreement(rb)},
        "device_budget_bytes": budget, "max_running_sites": lim, "clocks": clocks.summary(),
    }


def main():
    args = parse()
    if args.substeps:
        print(json.dumps(run_substeps(args)))
        return
    if args.serve:
        print(json.dumps(run_serving(args)))
        return
    if args.impl == "reference":
        out = run_reference(args)
        if out:
            print(json.dumps(out))
        return
    out = run_ours(args)
    if out is not None:
        world = out["n_gpus"]
        if world == 1 and not args.no_cpu_baseline:
            c, p = workload(args.workload)
            out["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds, c["mode"])
        print(json.dumps(out))


if __name__ == "__main__":
    main()
