"""Benchmark of the Stokes layer-operator apply and solve on SH drop surfaces (one JSON line).

Workload (default): one drop of SH degree p = 32, sphere plus a seeded SH perturbation of
amplitude 0.05 (degrees 1..6), viscosity ratio 5, shear u_inf = (z, 0, 0), self quadrature on the
grid of degree 2p+1 = 65.  One step = the right-hand side 2 u_inf + S[f] (FP64) followed by the
mixed-precision GMRES solve with FP64 iterative refinement to a relative residual of 1e-10.
value = Stokes pair interactions evaluated per second (singular self-rule pairs of every operator
apply in the step, divided by the step time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BIE matvec time & Stokes pair-interactions/s, FP64 vs mixed at 1e-8 rel err"
UNIT = "pair-interactions/s"
WORKLOAD = "one drop p=32 (sphere + 0.05 SH perturbation, n<=6), lambda=5, shear (z,0,0), self rule on the p_q=65 grid"
FP32_ALU_PEAK = 152 * 128 * 2 * 2.070e9 / 1e12  # TFLOP/s: SMs x FP32 lanes x FMA x max SM clock
FP64_ALU_PEAK = 1.25                              # TFLOP/s: nominal GB300 FP64 rate


def hbm_peak():
    """Measured copy bandwidth (GB/s) of the GB300s, else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"
# DRAM bytes (read + write) per launch from one ncu capture of the current kernels on this workload
# (profiles/self_proj_f64_c2.md, profiles/self_proj_f32_c2.md); null for any other kernel.
PROFILED_TRAFFIC = {"self_proj_f64": 120.644352e6 + 3.24864e6, "self_proj_f32": 60.3456e6 + 0.499456e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-aux", action="store_true", help="skip the many-drop apply measurements in the main line")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c4s", "c5"],
                    help="c2 (default): the solve step below; the others time one operator apply per step")
    ap.add_argument("--coupled", default=None, choices=["c4", "c5"],
                    help="print only the timing of coupled drop/surfactant steps (Alg. 1) on this workload")
    return ap.parse_args()


def max_over_ranks(t_local, device="cuda"):
    """The job's time: the largest of the ranks' times (t_local itself in a single process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_local
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, t_max):
    """Units processed by all ranks per second of the job's (slowest rank's) time."""
    return world * units_per_rank / t_max


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# algorithmic work of the singular self kernels, per target (FMA = 2 flops, rsqrt = 1)
# ------------------------------------------------------------------------------------------------
def self_work_per_target(name: str, p: int, pq: int, kind: str = "D"):
    """(flops, bytes) of one target of the self kernel `name` (self_proj_* or self_direct_*).

    Counts the arithmetic the kernel's algorithm performs: the projected form rotates the four
    targets (theta, phi_b), (theta, phi_b + pi), (pi - theta, phi_b), (pi - theta, phi_b + pi) in one
    pass over latitude theta's Wigner blocks (even/odd orders), then contracts each rotated
    coefficient (n, m >= 0; Re, Im x 3 components) with the target's 6 complex projected kernel
    factors.
    """
    esize = 8 if name.endswith("f64") or name.endswith("df") else 4  # double-float: two FP32 words
    wig = sum((n + 1) ** 2 + n * n for n in range(p + 1))          # rotation blocks of one latitude
    rot = 2.0 * 3 * wig                                              # three components
    nq = (pq + 1) * (2 * pq + 2)
    if "proj" in name:
        ng = (p + 1) * (2 * p + 2)
        rot *= ((p + 2) // 2) * (p + 1) / ng  # one pass over the blocks per target quadruple
        ntri = (p + 1) * (p + 2) // 2
        contr = 36.0 * ntri                                          # 3x3 complex symmetric times rho'_n^m
        return rot + contr, 12.0 * ntri * esize                      # Q read once per apply
    leg = 3.0 * (pq + 1) * (2 * (p + 1) + 4 * sum(p + 1 - m for m in range(1, p + 1)))
    phi = 3.0 * (pq + 1) * (pq + 1) * (4 * p + 2)                    # longitude pairs, even/odd orders
    pair = (32.0 if kind == "D" else 29.0) * nq
    return rot + leg + phi + pair, nq * (7 if kind == "D" else 4) * esize


class Scrub:
    """Writes a buffer larger than L2 (129 MB) between timed intervals, so that no timed step starts
    with a warm L2; the write itself sits outside every timed event pair."""

    def __init__(self, nbytes=512 << 20):
        import torch
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.k = 0

    def __call__(self):
        self.k = (self.k + 1) & 255
        self.buf.fill_(self.k)


def timed_steps(fn, n, stream, scrub):
    """Total milliseconds of n calls of fn, each timed with its own CUDA events on `stream`, with an
    L2 scrub before each (outside the events)."""
    import torch
    evs = []
    for _ in range(n):
        scrub()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs)


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1707_02156_gb300 import api, build, inputs
    build.build()
    ctx = api.Context(local)
    w = inputs.perturbed_drop()
    p, pq = w.p[0], w.pq[0]
    x = torch.tensor(w.xcoef, device="cuda")
    torch.cuda.synchronize()
    ctx.profile(True)  # set-up stages as phases
    t_geo = time.perf_counter()
    geo = ctx.geometry(w.p, w.pq, x, w.lam)
    torch.cuda.synchronize()
    geometry_ms = 1e3 * (time.perf_counter() - t_geo)
    geometry_stages = {k: v[0] for k, v in ctx.profile_read().items()}
    ctx.profile(False)
    nco = geo.info["ncoef"]
    pairs_per_apply = geo.info["self_pairs"]
    f = torch.tensor(w.density, device="cuda")
    uinf = torch.zeros(nco, dtype=torch.float64, device="cuda")
    uinf.view(3, -1)[0] = x.view(3, -1)[2] * w.shear   # u_inf = (z, 0, 0): linear, exactly band-limited
    rhs = torch.zeros_like(uinf)
    u = torch.zeros_like(uinf)
    stream = torch.cuda.current_stream()

    def step(precision, uvec, rhs_out):
        # b = 2 u_inf + S[f], FP64-grade: double-float for the mixed step, FP64 for the FP64 step
        geo.rhs(uinf, f, rhs_out, precision=2 if precision == 1 else 0)
        uvec.zero_()
        info = geo.solve(rhs_out, uvec, precision=precision, tol=1e-10, inner_tol=1e-5)
        return info

    scrub = Scrub()
    # warm-up
    step(1, u, rhs)
    step(0, u, rhs)
    for _ in range(args.warmup):
        info = step(1, u, rhs)
    torch.cuda.synchronize()

    # timed region: K mixed solves, default library behaviour (applies replayed as CUDA graphs)
    launches0 = api.launch_count()
    applies = 0
    last = {}

    def mixed_step():
        last["info"] = step(1, u, rhs)

    with ClockSampler(local) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ms_total = 0.0
        for _ in range(args.steps):
            ms_total += timed_steps(mixed_step, 1, stream, scrub)
            info = last["info"]
            applies += 1 + info["applies_fp64"] + info["applies_mixed"]
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    launches = api.launch_count() - launches0
    t_max = max_over_ranks(ms_total / 1e3)
    ms_step = 1e3 * t_max / args.steps
    value = whole_job_rate(applies * pairs_per_apply, world, t_max)
    # the same K steps again with the library's per-phase CUDA events on (kernels launched one by one)
    ctx.profile(True)
    ms_step_profiled = timed_steps(lambda: step(1, u, rhs), args.steps, stream, scrub) / args.steps
    phases = ctx.profile_read()
    ctx.profile(False)
    u_mixed = u.clone()
    mixed_info = info

    # FP64 reference solve on the GPU (same step, plain FP64 path), and the accuracy of mixed vs FP64
    u64 = torch.zeros_like(u)
    step(0, u64, rhs)
    torch.cuda.synchronize()

    def fp64_step():
        last["info64"] = step(0, u64, rhs)

    fp64_ms = timed_steps(fp64_step, 1, stream, scrub)
    info64 = last["info64"]
    rel = float(torch.linalg.norm(u_mixed - u64) / torch.linalg.norm(u64))
    rel_inf = float((u_mixed - u64).abs().max() / u64.abs().max())

    # matvec times (double layer) at each precision
    out = torch.zeros_like(u)
    mv = {}
    for prec in (0, 1):
        for _ in range(3):
            geo.apply_double(u64, out, precision=prec)
        mv[prec] = timed_steps(lambda: geo.apply_double(u64, out, precision=prec), 10, stream, scrub) / 10

    # end to end through the public API with host buffers: H2D of (f, u_inf), step, D2H of u
    f_h = torch.tensor(w.density).pin_memory()
    uinf_h = uinf.cpu().pin_memory()
    u_h = torch.zeros(nco, dtype=torch.float64).pin_memory()
    n_e2e = max(3, args.steps // 2)

    def e2e_step():
        f.copy_(f_h, non_blocking=True)
        uinf.copy_(uinf_h, non_blocking=True)
        step(1, u, rhs)
        u_h.copy_(u, non_blocking=True)

    e2e_s = timed_steps(e2e_step, n_e2e, stream, scrub) / 1e3 / n_e2e
    e2e_value = world * (applies / args.steps) * pairs_per_apply / e2e_s

    # roofline of the dominant kernel (the self kernel with the largest total time in the profiled steps)
    selfk = {k: v for k, v in phases.items() if k.startswith("self_")}
    dom_name, (dom_ms, dom_calls) = max(selfk.items(), key=lambda kv: kv[1][0])
    ntarget = geo.info["ntarget"]
    fl, by = self_work_per_target(dom_name, p, pq)
    flops, nbytes = fl * ntarget, by * ntarget
    avg_s = dom_ms / 1e3 / max(1, dom_calls)
    f64 = dom_name.endswith("f64")
    alu_peak = FP64_ALU_PEAK if f64 else FP32_ALU_PEAK
    bw_peak, bw_src = hbm_peak()
    # the roofline that bounds the kernel: the larger of its algorithmic times at the two peaks
    t_alu, t_hbm = flops / (alu_peak * 1e12), nbytes / (bw_peak * 1e9)
    if t_hbm > t_alu:
        achieved = nbytes / avg_s / 1e9
        roof = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": bw_peak, "unit": "GB/s",
                "frac": achieved / bw_peak, "peak_source": bw_src}
    else:
        achieved = flops / avg_s / 1e12
        roof = {"bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak,
                "peak_source": ("nominal GB300 FP64 rate 1.25 TFLOP/s (no measured FP64 peak available)" if f64 else
                                "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz")}
    roof.update({"traffic": PROFILED_TRAFFIC.get(dom_name), "algorithmic_flops_per_launch": flops,
                 "algorithmic_bytes_per_launch": nbytes, "tflops_achieved": flops / avg_s / 1e12,
                 "hbm_gbs_achieved": nbytes / avg_s / 1e9, "avg_launch_ms": avg_s * 1e3})

    # the inter-drop rows (regions, regular and upsampled pair sums) on the many-drop workloads
    also = {}
    if not args.no_aux:
        geo.close()
        for name in ("c4", "c5"):
            runs = ((1, 3, 2), (2, 2, 1), (0, 1, 0))
            info_a, pairs_a, res_a, sol = time_apply(name, local, runs, solve="both" if name == "c4" else "mixed")
            ma = res_a[1]
            also[name] = {"workload": APPLY_WORKLOADS[name], "step": "one mixed double-layer apply",
                          "ms_per_apply": ma["ms"], "pairs": pairs_a, "value": pairs_a / (ma["ms"] / 1e3),
                          "unit": UNIT, "far_pairs": info_a["far_pairs"], "up_pairs": info_a["up_pairs"],
                          "roofline": interdrop_roofline(info_a, ma["phases"], 3),
                          "setup_ms": info_a["setup_ms"], "precisions": apply_summary(res_a)}
            if sol and "fp64" in sol:
                rel_a = float(torch.linalg.norm(sol["mixed"]["u"] - sol["fp64"]["u"]) / torch.linalg.norm(sol["fp64"]["u"]))
                also[name]["solve"] = {
                    "step": "rhs + solve to 1e-10: mixed GMRES with double-float refinement residuals vs FP64 GMRES",
                    "mixed": {k: v for k, v in sol["mixed"].items() if k != "u"},
                    "fp64": {k: v for k, v in sol["fp64"].items() if k != "u"},
                    "speedup_vs_fp64": sol["fp64"]["ms"] / sol["mixed"]["ms"], "rel_err_mixed_vs_fp64": rel_a}
            elif sol:
                # an FP64 GMRES solve here takes minutes: its time is estimated, not measured, as
                # (iterations of the mixed solve + 1 right-hand side) FP64 applies
                est = (sol["mixed"]["iterations"] + 1) * res_a[0]["ms"]
                also[name]["solve"] = {
                    "step": "rhs + solve to 1e-10: mixed GMRES with double-float refinement residuals",
                    "mixed": {k: v for k, v in sol["mixed"].items() if k != "u"},
                    "fp64_estimate_ms": est, "fp64_estimate": "(mixed iterations + 1) x measured FP64 apply; not run",
                    "speedup_vs_fp64_estimate": est / sol["mixed"]["ms"]}

    if not args.no_aux:
        also["c4"]["time_step"] = time_midpoint("c4", local)
        also["c4"]["coupled_step"] = guarded(time_coupled, "c4", local)
    cpu = cpu_baseline_sample(w, budget_s=15.0) if rank == 0 else None
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "p": p, "p_q": pq, "targets": ntarget,
                   "pairs_per_apply": pairs_per_apply, "step": "rhs (double-float S apply) + mixed GMRES solve with double-float refinement residuals, tol 1e-10",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "L2 flushed (512 MB write) before every timed step; within a step the applies re-read "
                         "the projected kernel factors (FP32 59 MB, FP64 117 MB)"},
        "setup_ms": {"geometry": geometry_ms, "stages": geometry_stages,
                     "note": "geometry set-up includes the projected kernel factors of both layers"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * nco * 8, "d2h_bytes_per_step": nco * 8},
        "gpu_launches": launches,
        "roofline": roof,
        "phases_ms": {k: {"ms": v[0], "calls": v[1]} for k, v in phases.items()},
        "ms_per_step_profiled": ms_step_profiled,
        "solve": {"mixed_ms": ms_step, "fp64_ms": fp64_ms, "speedup_vs_fp64": fp64_ms / ms_step,
                  "mixed_iterations": mixed_info["iterations"], "mixed_refinements": mixed_info["refinements"],
                  "mixed_applies_fp64": mixed_info["applies_fp64"], "mixed_applies_f32": mixed_info["applies_mixed"],
                  "fp64_iterations": info64["iterations"], "rel_err_mixed_vs_fp64": rel, "rel_err_inf_mixed_vs_fp64": rel_inf,
                  "residual_mixed": mixed_info["residual"], "residual_fp64": info64["residual"]},
        "matvec": {"fp64_ms": mv[0], "mixed_ms": mv[1], "pairs_per_s_fp64": pairs_per_apply / (mv[0] / 1e3),
                   "pairs_per_s_mixed": pairs_per_apply / (mv[1] / 1e3)},
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "also": also,
    }
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline_sample(w, budget_s=15.0, lats=None):
    """The FP64 oracle's singular self rule (one double-layer apply) on a sample of latitudes."""
    from oracle import layer
    p, pq = w.p[0], w.pq[0]
    q = layer.SelfQuadrature(w.xcoef.reshape(3, -1), p, pq, cache=False)
    nb = 2 * p + 2
    done, t0 = 0, time.perf_counter()
    lat_list = lats if lats is not None else [0, p // 2, p, 1, p - 1, p // 3, 2 * p // 3]
    for a in lat_list:
        q.apply(w.density, "D", lats=[a])
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    pairs = done * nb * (pq + 1) * (2 * pq + 2)
    return {"value": pairs / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle FP64 singular self rule (rotated geometry + density, double layer), "
                      f"{done} of {p + 1} latitudes = {done * nb} of {(p + 1) * nb} targets of the p=32, p_q=65 drop"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_1707_02156_gb300 import inputs
    w = inputs.perturbed_drop()
    p, pq = w.p[0], w.pq[0]
    for _ in range(args.warmup):
        cpu_baseline_sample(w, budget_s=0.0, lats=[0])
    t0 = time.perf_counter()
    pairs = 0
    for i in range(args.steps):
        r = cpu_baseline_sample(w, budget_s=0.0, lats=[i % (p + 1)])
        pairs += (2 * p + 2) * (pq + 1) * (2 * pq + 2)
    dt = time.perf_counter() - t0
    v = pairs / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": "oracle double-layer self rule at one latitude (66 targets)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "one latitude (66 of 2178 targets) of one FP64 double-layer apply per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


APPLY_WORKLOADS = {
    "c3": "two unit spheres at gap 0.05, p=32, U=4, lambda=0.5 (all three regions)",
    "c4": "64 spheres, p in {16,24,32,48}, radii U[0.8,1.2], 10% volume fraction, lambda U[0.2,5], U=2",
    "c4s": "16 spheres, p in {16,24}, radii U[0.8,1.2], 10% volume fraction, lambda U[0.2,5], U=2",
    "c5": "512 ellipsoids + SH noise, p=24, 10% volume fraction, U=2",
}


def time_apply(name, local, runs=((1, 3, 2),), solve=False):
    """Double-layer applies of a multi-drop workload at the precisions of `runs` = ((prec, steps,
    warm-up), ...); returns the geometry info, the pairs per apply, per-precision timings, phases and
    outputs, and (with solve) a mixed solve with double-float residuals next to the plain FP64 solve."""
    import torch
    from paper_1707_02156_gb300 import api, build, inputs
    build.build()
    w = inputs.config(name)
    ctx = api.Context(local, upsample=w.up)
    x = torch.tensor(w.xcoef, device="cuda")
    torch.cuda.synchronize()
    ctx.profile(True)  # set-up stages as phases
    t0 = time.perf_counter()
    geo = ctx.geometry(w.p, w.pq, x, w.lam)
    torch.cuda.synchronize()
    setup = {"geometry": 1e3 * (time.perf_counter() - t0),
             "stages": {k: v[0] for k, v in ctx.profile_read().items()}}
    ctx.profile(False)
    info = dict(geo.info)
    pairs = info["self_pairs"] + info["far_pairs"] + info["up_pairs"] + info["near_pairs"]
    f = torch.tensor(w.density, device="cuda")
    out = torch.zeros_like(f)
    stream = torch.cuda.current_stream()
    scrub = Scrub()
    res = {}
    for prec, steps, warmup in runs:
        for _ in range(warmup):
            geo.apply_double(f, out, precision=prec)
        torch.cuda.synchronize()
        ctx.profile(True)
        launches0 = api.launch_count()
        with ClockSampler(local) as clk:
            ms = timed_steps(lambda: geo.apply_double(f, out, precision=prec), steps, stream, scrub)
        res[prec] = {"ms": ms / steps, "phases": ctx.profile_read(),
                     "launches": api.launch_count() - launches0, "clocks": clk.summary(), "out": out.clone()}
        ctx.profile(False)
    sol = None
    if solve:
        # b = 2 u_inf + S[f] with u_inf = (z, 0, 0), then the solve: mixed GMRES inside refinement with
        # double-float residuals, against FP64 GMRES (both to 1e-10)
        uinf = torch.zeros_like(f)
        o = 0
        for p in w.p:
            k = (p + 1) ** 2
            uinf[o:o + k] = torch.tensor(w.xcoef[o + 2 * k:o + 3 * k], device="cuda")
            o += 3 * k
        sol = {}
        cases = (("mixed", 1, 2), ("fp64", 0, 0)) if solve == "both" else (("mixed", 1, 2),)
        for label, prec, rprec in cases:
            b = torch.zeros_like(f)
            u = torch.zeros_like(f)
            last = {}

            def run():
                geo.rhs(uinf, f, b, precision=rprec)
                u.zero_()
                last["info"] = geo.solve(b, u, precision=prec, tol=1e-10, residual_precision=2)

            ms = timed_steps(run, 1, stream, scrub)
            sol[label] = {"ms": ms, **{k: last["info"][k] for k in ("iterations", "refinements", "applies_fp64",
                                                                     "applies_mixed", "residual")}, "u": u.clone()}
    geo.close()
    # a second geometry in the same context, as a time step builds it: the per-degree tables are cached
    torch.cuda.synchronize()
    ctx.profile(True)
    t0 = time.perf_counter()
    geo = ctx.geometry(w.p, w.pq, x, w.lam)
    torch.cuda.synchronize()
    setup["geometry_repeat"] = 1e3 * (time.perf_counter() - t0)
    setup["stages_repeat"] = {k: v[0] for k, v in ctx.profile_read().items()}
    ctx.profile(False)
    geo.close()
    ctx.close()
    del f, out
    torch.cuda.empty_cache()
    info["setup_ms"] = setup
    return info, pairs, res, sol


def time_midpoint(name, local, nsteps=2, dt=0.01):
    """Wall time of midpoint steps of the drop shapes (two geometries, two right-hand sides and two
    mixed solves with double-float residuals per step) on a many-drop workload in shear."""
    import torch
    from paper_1707_02156_gb300 import api, build, inputs
    build.build()
    w = inputs.config(name)
    shear = w.shear if w.shear else 1.0
    ctx = api.Context(local, upsample=w.up)
    x = torch.tensor(w.xcoef, device="cuda")
    g = torch.tensor(w.gamma, device="cuda")
    out = []
    for _ in range(nsteps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = api.midpoint_step(ctx, w.p, w.pq, x, g, w.elasticity, 0.0, w.lam, shear, dt)
        torch.cuda.synchronize()
        out.append({"ms": 1e3 * (time.perf_counter() - t0),
                    "iterations": [i["iterations"] for i in infos], "residual": [i["residual"] for i in infos]})
    ctx.close()
    torch.cuda.empty_cache()
    return {"step": f"midpoint step dt={dt} in shear {shear}: geometry, force, rhs and mixed solve at x and x+dt/2 u",
            "first_includes": "the context's per-degree tables", "steps": out}


def guarded(fn, *a):
    """fn(*a), or its error as a string: an auxiliary measurement never ends the bench."""
    try:
        return fn(*a)
    except Exception as e:  # recorded in the JSON line instead
        return {"error": f"{type(e).__name__}: {e}"}


def time_coupled(name, local, nsteps=2, dt=0.01, inv_pe=0.1):
    """Wall time of steps of Alg. 1 on a many-drop workload in shear: per step two geometries, two
    interfacial forces, right-hand sides and mixed solves (double-float residuals), the explicit
    surfactant rates at t and t + dt/2, the preconditioned implicit stage and the error estimates.
    The surfactant work alone (two rate evaluations and one implicit solve) is timed after the
    steps.  Pe = 10 (1/Pe = 0.1)."""
    import torch
    from paper_1707_02156_gb300 import api, build, inputs
    build.build()
    w = inputs.config(name)
    shear = w.shear if w.shear else 1.0
    ctx = api.Context(local, upsample=w.up)
    x = torch.tensor(w.xcoef, device="cuda")
    g = torch.tensor(w.gamma, device="cuda")
    u0, x1, g1 = torch.zeros_like(x), torch.zeros_like(x), torch.zeros_like(g)
    m0 = api.surfactant_mass(ctx, w.p, x, g)
    steps = []
    for _ in range(nsteps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = api.coupled_step(ctx, w.p, w.pq, x, g, u0, False, w.elasticity, 0.0, w.lam, shear, inv_pe, dt, x1, g1)
        torch.cuda.synchronize()
        steps.append({"ms": 1e3 * (time.perf_counter() - t0), "err_drop": info["err_drop"],
                      "err_conservation": info["err_conservation"], "implicit_iterations": info["implicit_iterations"],
                      "solve_iterations": [s["iterations"] for s in info["solve"]]})
        x, x1 = x1, x
        g, g1 = g1, g
    m1 = api.surfactant_mass(ctx, w.p, x, g)
    fe, fi, y = torch.zeros_like(g), torch.zeros_like(g), torch.zeros_like(g)
    api.surfactant_implicit(ctx, w.p, x, g, 0.5 * dt * inv_pe, y)  # warm-up of the plans
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.surfactant_rates(ctx, w.p, x, u0, g, 0.0, fe, None)
    api.surfactant_rates(ctx, w.p, x, u0, g, inv_pe, fe, fi)
    it = api.surfactant_implicit(ctx, w.p, x, g, 0.5 * dt * inv_pe, y)
    torch.cuda.synchronize()
    surf_ms = 1e3 * (time.perf_counter() - t0)
    ctx.close()
    torch.cuda.empty_cache()
    return {"step": f"coupled step of Alg. 1, dt={dt}, shear {shear}, Pe={1.0 / inv_pe:g}: midpoint shapes, "
                    "IMEX-2 surfactant, mixed velocity solves",
            "first_includes": "the context's per-degree tables", "steps": steps,
            "surfactant_only_ms": surf_ms, "surfactant_only": "two rate evaluations + the implicit stage",
            "implicit_iterations": it,
            "mass_change_max": max(abs(b - a) / abs(a) for a, b in zip(m0, m1))}


def interdrop_roofline(info, phases, steps):
    """Roofline entry of the inter-drop pair kernel: 32 flops per stresslet pair (FP32 FMA pipe)."""
    ms, calls = phases.get("interdrop_f32", (0.0, 0))
    if not calls:
        return None
    flops = 32.0 * (info["far_pairs"] + info["up_pairs"])
    avg = ms / 1e3 / calls
    ach = flops / avg / 1e12
    return {"bound": "alu", "kernel": "interdrop_f32", "achieved": ach, "peak": FP32_ALU_PEAK, "unit": "TFLOP/s",
            "frac": ach / FP32_ALU_PEAK, "traffic": None, "algorithmic_flops_per_launch": flops,
            "avg_launch_ms": avg * 1e3, "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz"}


def run_apply(args):
    """Auxiliary mode: time one double-layer apply per step (mixed, then double-float and FP64) on a
    multi-drop workload."""
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    runs = ((1, args.steps, args.warmup), (2, 1, 1), (0, 1, 0))
    info, pairs, res, _ = time_apply(args.workload, local, runs)
    m = res[1]
    print(json.dumps({
        "metric": METRIC, "value": pairs / (m["ms"] / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": APPLY_WORKLOADS[args.workload], "step": "one mixed double-layer apply",
                   "pairs": pairs, **{k: info[k] for k in ("ntarget", "self_pairs", "far_pairs", "up_pairs",
                                                               "near_targets", "near_pairs")}},
        "gpu_launches": m["launches"], "clocks": m["clocks"],
        "roofline": interdrop_roofline(info, m["phases"], args.steps),
        "phases_ms": {k: {"ms": v[0], "calls": v[1]} for k, v in m["phases"].items()},
        "precisions": apply_summary(res), "setup_ms": info["setup_ms"],
    }))


def apply_summary(res):
    """Per-precision apply times and relative errors against the FP64 apply."""
    import torch
    ref = res[0]["out"] if 0 in res else None
    out = {}
    for prec, name in ((1, "mixed"), (2, "df"), (0, "fp64")):
        if prec not in res:
            continue
        r = res[prec]
        e = {"ms_per_apply": r["ms"], "phases_ms": {k: {"ms": v[0], "calls": v[1]} for k, v in r["phases"].items()}}
        if ref is not None and prec != 0:
            e["rel_err_vs_fp64"] = float(torch.linalg.norm(r["out"] - ref) / torch.linalg.norm(ref))
            e["rel_err_inf_vs_fp64"] = float((r["out"] - ref).abs().max() / ref.abs().max())
            e["speedup_vs_fp64"] = res[0]["ms"] / r["ms"]
        out[name] = e
    return out


if __name__ == "__main__":
    a = parse()
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    if a.impl == "reference":
        run_reference(a)
    elif a.coupled:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"workload": a.coupled, "coupled": time_coupled(a.coupled, 0)}))
    elif a.workload != "c2":
        run_apply(a)
    else:
        run_ours(a)
