"""Benchmark of the Stokes layer-operator applies and the solve on SH drop surfaces (one JSON line).

Workload (default, c5): 512 randomly oriented ellipsoidal drops (axes U[0.7, 1.3]) plus SH noise of
amplitude 0.1 (degrees 2..8), SH degree p = 24, upsampling factor 2 for the intermediate region,
10% volume fraction in a cube of side 27.8, viscosity ratios U[0.2, 5], shear u_inf = (z, 0, 0),
interfacial force of a random decaying surfactant with sigma = 1 - 0.2 Gamma.

One step = the right-hand side 2 u_inf + S[f] (double-float: FP64-grade) and the mixed-precision
solve of (lambda + 1) u - D[u] = b: FP32 inner GMRES (FP32 rotation, contraction and pair sums)
inside iterative refinement with double-float residuals, to a relative residual of 1e-10.  Every
row of the hot path runs in each step: Wigner rotation and contraction of the singular self term,
source synthesis, inter-drop pair sums by region, Galerkin projection, Krylov kernels.
value = Stokes pair interactions evaluated per second: (self-rule + regular + upsampled +
near-singular pairs of one operator apply) x (operator applies in the step) / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload c1..c5]
                  [--no-aux] [--timesteps N] [--fp64-solve] [--tensor-rotation] [--coupled c4|c5]

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload, on the host's
cores.  The other configurations (c1 .. c4) are reported under "also" unless --no-aux.
"""
from __future__ import annotations

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

METRIC = "BIE matvec time & Stokes pair-interactions/s, FP64 vs mixed at 1e-8 rel err"
UNIT = "pair-interactions/s"
WORKLOADS = {
    "c1": "one unit sphere, p=16, lambda=1, random band-limited density: one singular single-layer apply",
    "c2": "one drop p=32 (sphere + 0.05 SH perturbation, n<=6), lambda=5, shear (z,0,0), self rule on the "
          "p_q=65 grid",
    "c3": "two unit spheres at gap 0.05, p=32, U=4, lambda=0.5, Gamma=1+0.3Y_2^0, sigma=1-0.2Gamma, shear (z,0,0)",
    "c4": "64 spheres, p in {16,24,32,48}, radii U[0.8,1.2], 10% volume fraction, lambda U[0.2,5], U=2, "
          "shear (z,0,0)",
    "c4s": "16 spheres, p in {16,24}, radii U[0.8,1.2], 10% volume fraction, lambda U[0.2,5], U=2",
    "c5": "512 ellipsoids (axes U[0.7,1.3], random orientation) + SH noise 0.1 (n<=8), p=24, U=2, 10% volume "
          "fraction, lambda U[0.2,5], shear (z,0,0), interfacial force of a random decaying Gamma, "
          "sigma=1-0.2Gamma",
}
STEP = ("rhs 2 u_inf + S[f] (double-float S apply) + mixed solve: FP32 inner GMRES inside refinement with "
        "double-float residuals, tol 1e-10")

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a kernel on a workload,
# from one ncu capture, with the SHA-256 prefix of the kernel's source file at the time of the
# capture: a capture of an older version of the kernel is not reported (traffic null).
# bie_config.tensor_rotation of every context the bench makes (--tensor-rotation)
TENSOR_ROTATION = False

PROFILED_TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum -k regex:k_interdrop_x2
    #     -s 16 -c 1 python bench.py --no-aux --steps 1 --warmup 3   (one pass; 183.82 MB read, 132.60 MB written)
    ("interdrop_f32", "c5"): {"bytes": 316.42e6, "source": "interdrop.cu", "sha": "3d31e48d7720c587"},
    # ncu --set full --kernel-name-base demangled -k regex:"k_self_proj<float" -s 4 -c 1
    #     python bench.py --workload c2 --no-aux --steps 1 --warmup 3   (60.35 MB read, 0.70 MB written)
    ("self_proj_f32", "c2"): {"bytes": 61.05e6, "source": "self.cu", "sha": "ea9853933df42712"},
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5", choices=["c1", "c2", "c3", "c4", "c4s", "c5"])
    ap.add_argument("--no-aux", action="store_true", help="leave out the other configurations and the CPU baseline")
    ap.add_argument("--timesteps", type=int, default=0,
                    help="also time this many midpoint time steps of the workload (two solves each)")
    ap.add_argument("--fp64-solve", action="store_true",
                    help="also time the plain FP64 GMRES solve of the headline workload (minutes on c5)")
    ap.add_argument("--tensor-rotation", action="store_true",
                    help="rotate the projected self form on the tensor cores (bie_config.tensor_rotation)")
    ap.add_argument("--coupled", default=None, choices=["c4", "c5"],
                    help="print only the timing of coupled drop/surfactant steps (Alg. 1) on this workload")
    return ap.parse_args(argv)


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
        sm, smax, power, reasons = [], [], [], set()
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
            try:
                power.append(float(f[2]))
            except ValueError:
                pass
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
               "samples": len(sm)}
        if power:
            out["power_w_median"] = statistics.median(power)
        return out


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


def timed_each(fn, n, stream, scrub):
    """Milliseconds of each of n calls of fn, each timed with its own CUDA events on `stream`, with an
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
    return [a.elapsed_time(b) for a, b in evs]


def timed_steps(fn, n, stream, scrub):
    """Total milliseconds of n calls of fn (see timed_each)."""
    return sum(timed_each(fn, n, stream, scrub))


# ------------------------------------------------------------------------------------------------
# peaks and rooflines
# ------------------------------------------------------------------------------------------------
def hbm_peak():
    """Measured copy bandwidth (GB/s) of the GB300s, else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def alu_peaks(ctx):
    """FP32, packed FP32 and FP64 FMA rates (TFLOP/s) measured on this GPU in this run (best of two
    calls of bie_alu_peak each)."""
    return {name: max(ctx.alu_peak(w) for _ in range(2)) for w, name in ((0, "fp32"), (1, "fp32x2"), (2, "fp64"))}


def source_sha(fname):
    with open(os.path.join(ROOT, "paper_1707_02156_gb300", "csrc", fname), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def profiled_traffic(kernel, workload):
    e = PROFILED_TRAFFIC.get((kernel, workload))
    if not e or e["bytes"] is None or e["sha"] != source_sha(e["source"]):
        return None
    return e["bytes"]


def self_work_per_target(name: str, p: int, pq: int):
    """(flops, bytes) per target of the projected-form self kernel `name` (self_proj_*): the rotation
    of four targets (theta, phi_b), (theta, phi_b + pi), (pi - theta, phi_b), (pi - theta, phi_b + pi)
    in one pass over latitude theta's Wigner blocks (even/odd orders), then the contraction of each
    rotated coefficient (n, m >= 0; Re, Im x 3 components) with the target's projected factors,
    which are read once per apply (FMA = 2 flops)."""
    esize = 8 if name.endswith("f64") or name.endswith("df") else 4
    wig = sum((n + 1) ** 2 + n * n for n in range(p + 1))
    ng = (p + 1) * (2 * p + 2)
    rot = 2.0 * 3 * wig * ((p + 2) // 2) * (p + 1) / ng
    ntri = (p + 1) * (p + 2) // 2
    return rot + 36.0 * ntri, 12.0 * ntri * esize


def roofline(phases, info, peaks, workload, p_of=None):
    """Roofline entry of the kernel with the largest time in `phases` (the library's per-phase CUDA
    events on the launching stream).  Pair kernels: 32 flops per stresslet pair against the
    measured FP32 (or FP64) FMA rate.  Self kernels: the larger of the HBM and ALU algorithmic
    times decides the bound."""
    cand = {k: v for k, v in phases.items() if k.startswith(("interdrop_f32", "interdrop_f64", "self_proj_"))}
    if not cand:
        return None
    name, (ms, calls) = max(cand.items(), key=lambda kv: kv[1][0])
    avg_s = ms / 1e3 / max(1, calls)
    fp32_peak = max(peaks["fp32"], peaks["fp32x2"])
    if name.startswith("interdrop"):
        flops = 32.0 * (info["far_pairs"] + info["up_pairs"])
        f64 = name.endswith("f64")
        peak = peaks["fp64"] if f64 else fp32_peak
        ach = flops / avg_s / 1e12
        return {"bound": "alu", "kernel": name, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": profiled_traffic(name, workload), "algorithmic_flops_per_launch": flops,
                "algorithmic_unit": "32 flops per stresslet pair x (regular + upsampled pairs of one apply)",
                "avg_launch_ms": avg_s * 1e3, "launches": calls,
                "peak_source": ("measured in this run: FP64 FMA rate (bie_alu_peak)" if f64 else
                                "measured in this run: FP32 FMA rate, max of fma.rn.f32 and fma.rn.f32x2 "
                                "(bie_alu_peak)")}
    p, pq, ntarget = p_of
    fl, by = self_work_per_target(name, p, pq)
    flops, nbytes = fl * ntarget, by * ntarget
    bw, bw_src = hbm_peak()
    alu = peaks["fp64"] if name.endswith("f64") else fp32_peak
    t_alu, t_hbm = flops / (alu * 1e12), nbytes / (bw * 1e9)
    if t_hbm > t_alu:
        ach = nbytes / avg_s / 1e9
        r = {"bound": "hbm", "achieved": ach, "peak": bw, "unit": "GB/s", "frac": ach / bw, "peak_source": bw_src}
    else:
        ach = flops / avg_s / 1e12
        r = {"bound": "alu", "achieved": ach, "peak": alu, "unit": "TFLOP/s", "frac": ach / alu,
             "peak_source": "measured in this run (bie_alu_peak)"}
    r.update({"kernel": name, "traffic": profiled_traffic(name, workload), "algorithmic_flops_per_launch": flops,
              "algorithmic_bytes_per_launch": nbytes, "avg_launch_ms": avg_s * 1e3, "launches": calls})
    return r


# ------------------------------------------------------------------------------------------------
# one workload on the GPU
# ------------------------------------------------------------------------------------------------
class Case:
    """A workload's context, geometry, force and far field on the device."""

    def __init__(self, name, local):
        import torch
        from paper_1707_02156_gb300 import api, build, inputs
        build.build()
        self.name = name
        self.w = w = inputs.config(name)
        self.ctx = api.Context(local, upsample=w.up, tensor_rotation=TENSOR_ROTATION)
        self.x = torch.tensor(w.xcoef, device="cuda")
        torch.cuda.synchronize()
        self.ctx.profile(True)
        t0 = time.perf_counter()
        self.geo = self.ctx.geometry(w.p, w.pq, self.x, w.lam)
        torch.cuda.synchronize()
        self.setup = {"geometry": 1e3 * (time.perf_counter() - t0),
                      "stages": {k: v[0] for k, v in self.ctx.profile_read().items()},
                      "note": "geometry set-up includes the projected kernel factors of both layers"}
        self.ctx.profile(False)
        self.info = dict(self.geo.info)
        self.pairs = sum(self.info[k] for k in ("self_pairs", "far_pairs", "up_pairs", "near_pairs"))
        nco = self.info["ncoef"]
        self.f = torch.tensor(w.density, device="cuda")
        self.force = "seeded band-limited density"
        if w.gamma is not None and w.elasticity > 0:  # the interfacial force of the surfactant
            g = torch.tensor(w.gamma, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            self.geo.interfacial_force(g, w.elasticity, 0.0, self.f)
            torch.cuda.synchronize()
            self.setup["interfacial_force"] = 1e3 * (time.perf_counter() - t0)
            self.force = f"interfacial force of Gamma, sigma = 1 - {w.elasticity} Gamma"
        self.shear = w.shear if w.shear else 1.0
        self.uinf = torch.zeros(nco, dtype=torch.float64, device="cuda")
        o = 0
        for p in w.p:  # u_inf = (shear z, 0, 0): z's coefficients in the first component
            k = (p + 1) ** 2
            self.uinf[o:o + k] = self.shear * self.x[o + 2 * k:o + 3 * k]
            o += 3 * k
        self.b = torch.zeros_like(self.uinf)
        self.u = torch.zeros_like(self.uinf)

    def step(self, precision=1, u=None, b=None):
        """Right-hand side (double-float for the mixed step, FP64 for the FP64 step) and solve."""
        u = self.u if u is None else u
        b = self.b if b is None else b
        self.geo.rhs(self.uinf, self.f, b, precision=2 if precision == 1 else 0)
        u.zero_()
        return self.geo.solve(b, u, precision=precision, tol=1e-10, residual_precision=2, max_iter=600)

    def setup_repeat(self):
        """A second geometry in the same context, as a time step builds it (per-degree tables cached)."""
        import torch
        torch.cuda.synchronize()
        self.ctx.profile(True)
        t0 = time.perf_counter()
        g2 = self.ctx.geometry(self.w.p, self.w.pq, self.x, self.w.lam)
        torch.cuda.synchronize()
        self.setup["geometry_repeat"] = 1e3 * (time.perf_counter() - t0)
        self.setup["stages_repeat"] = {k: v[0] for k, v in self.ctx.profile_read().items()}
        self.ctx.profile(False)
        g2.close()

    def close(self):
        import torch
        self.geo.close()
        self.ctx.close()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()


def apply_stats(case, vec, stream, scrub, runs):
    """Double-layer applies D[vec] at the precisions of `runs` = ((prec, n, warm-up), ...): per-precision
    ms per apply, phases, and errors against the FP64 apply."""
    import torch
    geo, api_ctx = case.geo, case.ctx
    out = torch.zeros_like(case.uinf)
    res = {}
    for prec, n, warm in runs:
        for _ in range(warm):
            geo.apply_double(vec, out, precision=prec)
        torch.cuda.synchronize()
        api_ctx.profile(True)
        ms = timed_steps(lambda: geo.apply_double(vec, out, precision=prec), n, stream, scrub)
        res[prec] = {"ms": ms / n, "phases": api_ctx.profile_read(), "out": out.clone()}
        api_ctx.profile(False)
    return apply_summary(res), res


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


def fp64_residual(case, u, d64, stream, scrub):
    """||b - A u|| / ||b|| with the right-hand side b = 2 u_inf + S[f] and the operator part D[u] (given:
    d64) both evaluated by the plain FP64 operators; also the FP64 right-hand side's time."""
    import torch
    b64 = torch.zeros_like(case.uinf)
    ms = timed_steps(lambda: case.geo.rhs(case.uinf, case.f, b64, precision=0), 1, stream, scrub)
    lam = torch.zeros_like(case.uinf)
    o = 0
    for p, l in zip(case.w.p, case.w.lam):
        k = 3 * (p + 1) ** 2
        lam[o:o + k] = l + 1.0
        o += k
    r = b64 - (lam * u - d64)
    torch.cuda.synchronize()
    return float(torch.linalg.norm(r) / torch.linalg.norm(b64)), ms


def solve_line(name, local, steps, warmup, world, peaks, headline=False, fp64_solve=False, fp64_apply=True):
    """Time K steps (rhs + mixed solve) of a workload, with its profile, applies per precision,
    accuracy against the FP64 operators and (headline) the end-to-end variant through host buffers."""
    import torch
    from paper_1707_02156_gb300 import api
    case = Case(name, local)
    stream = torch.cuda.current_stream()
    scrub = Scrub()
    for _ in range(warmup):
        info = case.step(1)
    torch.cuda.synchronize()
    launches0 = api.launch_count()
    applies = 0
    last = {}

    def mixed_step():
        last["info"] = case.step(1)

    with ClockSampler(local) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        # the timed steps are the range a profiler started with --profile-from-start off records
        torch.cuda.profiler.start()
        times = []
        for _ in range(steps):
            times += timed_each(mixed_step, 1, stream, scrub)
            info = last["info"]
            applies += 1 + info["applies_fp64"] + info["applies_mixed"]
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        if world > 1:
            torch.distributed.barrier()
    launches = api.launch_count() - launches0
    t_max = max_over_ranks(sum(times) / 1e3)
    line = {"workload": WORKLOADS[name], "step": STEP, "steps": steps, "warmup": warmup,
            "ms_per_step": 1e3 * t_max / steps, "ms_per_step_each": times,
            "value": whole_job_rate(applies * case.pairs, world, t_max), "unit": UNIT,
            "pairs_per_apply": case.pairs, "applies_per_step": applies / steps, "gpu_launches": launches,
            "clocks": clk.summary(), "force": case.force,
            "geometry": {k: case.info[k] for k in ("ndrop", "ntarget", "self_pairs", "far_pairs", "up_pairs",
                                                      "near_targets", "near_pairs", "interdrop_tpt", "pair_slots")},
            "solve": {k: info[k] for k in ("iterations", "refinements", "applies_fp64", "applies_mixed",
                                           "residual")}}
    u_mixed = case.u.clone()
    # one more step with the library's per-phase CUDA events on (kernels launched one by one)
    case.ctx.profile(True)
    line["ms_per_step_profiled"] = timed_steps(lambda: case.step(1), 1, stream, scrub)
    phases = case.ctx.profile_read()
    case.ctx.profile(False)
    line["phases_ms"] = {k: {"ms": v[0], "calls": v[1]} for k, v in phases.items()}
    p0 = case.w.p[0]
    line["roofline"] = roofline(phases, case.info, peaks, name, (p0, case.w.pq[0], case.info["ntarget"]))
    # double-layer applies to the mixed solution per precision; the FP64 apply is the reference of the
    # mixed and double-float errors and, with the FP64 right-hand side, gives the FP64 residual
    runs = [(1, 5, 1), (2, 2, 1)] + ([(0, 1, 0)] if fp64_apply else [])
    line["precisions"], res = apply_stats(case, u_mixed, stream, scrub, runs)
    if fp64_apply:
        rr, ms_rhs = fp64_residual(case, u_mixed, res[0]["out"], stream, scrub)
        line["fp64_residual_of_mixed_solution"] = rr
        line["fp64_rhs_ms"] = ms_rhs
    if fp64_solve:
        u64 = torch.zeros_like(case.u)
        b64 = torch.zeros_like(case.u)
        info64 = {}

        def s64():
            info64["i"] = case.step(0, u=u64, b=b64)

        ms64 = timed_steps(s64, 1, stream, scrub)
        line["fp64_solve"] = {"ms": ms64, **{k: info64["i"][k] for k in ("iterations", "residual")},
                              "speedup_mixed_vs_fp64": ms64 / line["ms_per_step"],
                              "rel_err_mixed_vs_fp64": float(torch.linalg.norm(u_mixed - u64) /
                                                             torch.linalg.norm(u64))}
    if headline:
        # end to end through the public API with host buffers: H2D of (f, u_inf), the step, D2H of u
        f_h = case.f.cpu().pin_memory()
        uinf_h = case.uinf.cpu().pin_memory()
        u_h = torch.zeros_like(case.u, device="cpu").pin_memory()
        n_e2e = min(steps, 3)

        def e2e_step():
            case.f.copy_(f_h, non_blocking=True)
            case.uinf.copy_(uinf_h, non_blocking=True)
            case.step(1)
            u_h.copy_(case.u, non_blocking=True)

        e2e_s = max_over_ranks(timed_steps(e2e_step, n_e2e, stream, scrub) / 1e3) / n_e2e
        line["e2e"] = {"value": world * (applies / steps) * case.pairs / e2e_s, "unit": UNIT,
                       "h2d_bytes_per_step": 2 * case.info["ncoef"] * 8, "d2h_bytes_per_step": case.info["ncoef"] * 8,
                       "steps": n_e2e}
    case.setup_repeat()
    line["setup_ms"] = case.setup
    case.close()
    return line


def apply_line(name, local, steps, warmup, peaks):
    """Latency of one operator apply (c1: the singular single-layer apply of one sphere)."""
    import torch
    case = Case(name, local)
    stream = torch.cuda.current_stream()
    scrub = Scrub()
    out = torch.zeros_like(case.uinf)
    res = {}
    for prec in (0, 1):
        for _ in range(warmup):
            case.geo.apply_single(case.f, out, precision=prec)
        torch.cuda.synchronize()
        t = timed_each(lambda: case.geo.apply_single(case.f, out, precision=prec), steps, stream, scrub)
        res[prec] = {"us_median": 1e3 * statistics.median(t), "out": out.clone()}
    rel = float(torch.linalg.norm(res[1]["out"] - res[0]["out"]) / torch.linalg.norm(res[0]["out"]))
    line = {"workload": WORKLOADS[name], "step": "one singular single-layer apply (graph replay)",
            "fp64_us": res[0]["us_median"], "mixed_us": res[1]["us_median"], "rel_err_mixed_vs_fp64": rel,
            "pairs_per_apply": case.pairs, "value": case.pairs / (res[0]["us_median"] * 1e-6), "unit": UNIT,
            "value_precision": "fp64", "setup_ms": case.setup}
    case.close()
    return line


def fluid_points(w, n, clearance, seed=11):
    """n seeded points of the workload's box that lie farther than `clearance` from every drop centre
    (outside every drop when clearance exceeds the largest drop radius), as a [3][n] array."""
    import numpy as np
    rng = np.random.default_rng(seed)
    cen, o = [], 0
    for p in w.p:
        k = (p + 1) ** 2
        cen.append(w.xcoef[o:o + 3 * k].reshape(3, k)[:, 0] / math.sqrt(4 * math.pi))
        o += 3 * k
    cen = np.array(cen)
    lo, hi = cen.min(axis=0), cen.max(axis=0)
    keep = []
    while sum(k.shape[1] for k in keep) < n:
        cand = lo[:, None] + (hi - lo)[:, None] * rng.random((3, 4 * n))
        d2 = np.full(cand.shape[1], np.inf)
        for c in cen:
            d2 = np.minimum(d2, np.sum((cand - c[:, None]) ** 2, axis=0))
        keep.append(cand[:, d2 > clearance ** 2])
    return np.ascontiguousarray(np.concatenate(keep, axis=1)[:, :n])


def near_surface_points(ctx, w, n, offset, seed=12):
    """n seeded points `offset` outside the drops: random standard-grid points of random drops moved
    out along the ray from the drop's centre (outward for these convex, near-spherical shapes), as a
    [3][n] device array; with offset below h = R pi/(p+1) they lie in that drop's Omega_2."""
    import numpy as np
    import torch
    rng = np.random.default_rng(seed)
    grid = torch.zeros(sum(3 * (p + 1) * (2 * p + 2) for p in w.p), dtype=torch.float64, device="cuda")
    ctx.sh_synthesize(w.p, w.p, 3, torch.tensor(w.xcoef, device="cuda"), grid)
    g = grid.cpu().numpy()
    blocks, o, oc = [], 0, 0
    for p in w.p:
        ng, k = (p + 1) * (2 * p + 2), (p + 1) ** 2
        c = w.xcoef[oc:oc + 3 * k].reshape(3, k)[:, 0] / math.sqrt(4 * math.pi)
        blocks.append((g[o:o + 3 * ng].reshape(3, ng), c))
        o += 3 * ng
        oc += 3 * k
    out = np.empty((3, n))
    for i in range(n):
        x, c = blocks[rng.integers(len(blocks))]
        y = x[:, rng.integers(x.shape[1])]
        out[:, i] = y + offset * (y - c) / np.linalg.norm(y - c)
    return torch.tensor(out, device="cuda")


def offsurface_line(name, local, steps, warmup, npoint=131072):
    """The velocity u_inf + (S[f] + D[u]) / 2 at npoint fluid points among the drops (bie_eval_velocity:
    region classification, pair sums on the standard / upsampled grids, near-singular interpolation
    for points within h of a surface), mixed against FP64, with a seeded density for u."""
    import torch
    case = Case(name, local)
    pts = torch.tensor(fluid_points(case.w, npoint, 1.6), device="cuda")
    u = torch.tensor(case.w.density, device="cuda")
    uinf = torch.zeros_like(pts)
    uinf[0] = (case.w.shear if case.w.shear else 1.0) * pts[2]
    stream = torch.cuda.current_stream()
    scrub = Scrub()
    res = {}
    for prec in (1, 0):
        out = torch.zeros_like(pts)
        for _ in range(warmup if prec == 1 else 1):
            case.geo.velocity_at(pts, case.f, u, out, uinf=uinf, precision=prec)
        torch.cuda.synchronize()
        t = timed_each(lambda: case.geo.velocity_at(pts, case.f, u, out, uinf=uinf, precision=prec),
                       steps if prec == 1 else 1, stream, scrub)
        res[prec] = {"ms": statistics.median(t), "out": out.clone()}
    rel = float(torch.linalg.norm(res[1]["out"] - res[0]["out"]) / torch.linalg.norm(res[0]["out"]))
    # one more mixed call with the library's per-phase events on
    case.ctx.profile(True)
    case.geo.velocity_at(pts, case.f, u, res[1]["out"], uinf=uinf, precision=1)
    torch.cuda.synchronize()
    phases = {k: {"ms": v[0], "calls": v[1]} for k, v in case.ctx.profile_read().items()}
    case.ctx.profile(False)
    # points 0.06 off the surfaces (in Omega_2 of the nearest drop): the near-singular step's cost
    nn = 8192
    near_pts = near_surface_points(case.ctx, case.w, nn, 0.06)
    uinf_n = torch.zeros_like(near_pts)
    uinf_n[0] = (case.w.shear if case.w.shear else 1.0) * near_pts[2]
    near_res = {}
    for prec in (1, 0):
        out = torch.zeros_like(near_pts)
        case.ctx.profile(prec == 1)
        t = timed_each(lambda: case.geo.velocity_at(near_pts, case.f, u, out, uinf=uinf_n, precision=prec), 1, stream,
                       scrub)
        near_res[prec] = {"ms": t[0], "out": out.clone()}
        if prec == 1:
            near_res["phases"] = {k: {"ms": v[0], "calls": v[1]} for k, v in case.ctx.profile_read().items()}
            case.ctx.profile(False)
    near_rel = float(torch.linalg.norm(near_res[1]["out"] - near_res[0]["out"]) / torch.linalg.norm(near_res[0]["out"]))
    line = {"workload": WORKLOADS[name], "points": npoint, "phases_ms_mixed": phases,
            "near_surface": {"points": nn, "offset": 0.06, "ms_mixed": near_res[1]["ms"], "ms_fp64": near_res[0]["ms"],
                             "rel_err_mixed_vs_fp64": near_rel, "phases_ms_mixed": near_res["phases"]},
            "step": "velocity at seeded fluid points farther than 1.6 from every drop centre (bie_eval_velocity)",
            "ms_mixed": res[1]["ms"], "ms_fp64": res[0]["ms"], "points_per_s_mixed": npoint / (res[1]["ms"] * 1e-3),
            "speedup_mixed_vs_fp64": res[0]["ms"] / res[1]["ms"], "rel_err_mixed_vs_fp64": rel}
    case.close()
    return line


def time_midpoint(name, local, nsteps=2, dt=0.01):
    """Wall time of midpoint steps of the drop shapes (two geometries, two right-hand sides and two
    mixed solves with double-float residuals per step) on a workload in shear."""
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
            "first_includes": "the context's per-degree tables", "steps": out,
            "total_ms": sum(s["ms"] for s in out)}


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
    Pe = 10 (1/Pe = 0.1)."""
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
    ctx.close()
    torch.cuda.empty_cache()
    return {"step": f"coupled step of Alg. 1, dt={dt}, shear {shear}, Pe={1.0 / inv_pe:g}: midpoint shapes, "
                    "IMEX-2 surfactant, mixed velocity solves",
            "first_includes": "the context's per-degree tables", "steps": steps,
            "mass_change_max": max(abs(b - a) / abs(a) for a, b in zip(m0, m1))}


# ------------------------------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# ------------------------------------------------------------------------------------------------
def _oracle_inputs(name):
    from paper_1707_02156_gb300 import inputs
    w = inputs.config(name)
    xs, ds, o = [], [], 0
    for p in w.p:
        k = 3 * (p + 1) ** 2
        xs.append(w.xcoef[o:o + k].reshape(3, -1))
        ds.append(w.density[o:o + k].reshape(3, -1))
        o += k
    return w, xs, ds


def _oracle_loop(conn, name, js, self_drop):
    """One host process of the oracle sample: it owns the source drops `js` (their oracle grids,
    densities and bounding spheres are built once, untimed, as the GPU's geometry set-up is) and the
    singular rule of drop `self_drop`; per request (targets, their drops, a self latitude) it returns
    (far pairs, seconds, self pairs, seconds) of the timed sums."""
    import numpy as np
    sys.path.insert(0, ROOT)
    from oracle import geometry, layer
    w, xs, ds = _oracle_inputs(name)
    prep = []
    for j in js:
        pj = w.p[j]
        std = layer.DropGrid(xs[j], pj, pj)
        ups = layer.DropGrid(xs[j], pj, w.up * (pj + 1) - 1)
        h = geometry.mean_radius(xs[j], pj) * math.pi / (pj + 1)
        c = xs[j][:, 0] / math.sqrt(4 * math.pi)
        bound = float(np.max(np.linalg.norm(ups.x - c[:, None], axis=0)))
        prep.append((j, (w.lam[j] - 1.0) / (4 * math.pi), std, std.density(ds[j]), ups, ups.density(ds[j]), h, c,
                     bound))
    sq = layer.SelfQuadrature(xs[self_drop], w.p[self_drop], w.pq[self_drop], cache=False) if self_drop >= 0 else None
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg is None:
            break
        pts, tdrops, lat = msg
        sels = []
        for j, wgt, std, rho, ups, rho_u, h, c, bound in prep:  # regions (set-up work, not timed)
            mask = tdrops != j
            near = mask & (np.linalg.norm(pts - c[:, None], axis=0) - bound <= 5.0 * h)
            reg = np.zeros(pts.shape[1], dtype=int)
            for k in np.nonzero(near)[0]:
                if np.sqrt(np.min(np.sum((ups.x - pts[:, k:k + 1]) ** 2, axis=0))) <= 5.0 * h:
                    reg[k] = 1
            sels.append([np.nonzero((reg == r) & mask)[0] for r in (0, 1)])
        val = np.zeros_like(pts)
        pairs = 0
        t0 = time.perf_counter()
        for (j, wgt, std, rho, ups, rho_u, h, c, bound), sel2 in zip(prep, sels):
            for src, rr, sel in ((std, rho, sel2[0]), (ups, rho_u, sel2[1])):
                if len(sel):
                    val[:, sel] += wgt * layer.regular_sum(pts[:, sel], src, rr, "D")
                    pairs += len(sel) * src.x.shape[1]
        far_s = time.perf_counter() - t0
        self_pairs, self_s = 0, 0.0
        if sq is not None and lat >= 0:
            t0 = time.perf_counter()
            sq.apply(ds[self_drop], "D", lats=[lat])
            self_s = time.perf_counter() - t0
            p, pq = w.p[self_drop], w.pq[self_drop]
            self_pairs = (2 * p + 2) * (pq + 1) * (2 * pq + 2)
        conn.send((pairs, far_s, self_pairs, self_s))
    conn.close()


class OraclePool:
    """`cores` spawned host processes running the FP64 oracle on a sample of a workload: process c
    owns the source drops c, c + stride, c + 2 stride, ... (below ndrop) and the singular rule of drop
    37 c mod ndrop.  Spawned, so it is safe to start after CUDA is initialised."""

    def __init__(self, name, cores, stride=None):
        import multiprocessing as mpc
        from paper_1707_02156_gb300 import inputs
        self.name, self.cores = name, cores
        self.w = inputs.config(name)
        nd = len(self.w.p)
        stride = stride or cores
        ctx = mpc.get_context("spawn")
        self.conns, self.procs = [], []
        for c in range(cores):
            js = list(range(c, nd, stride)) if nd > 1 else []
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_loop, args=(b, name, js, (37 * c) % nd), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        for cn in self.conns:
            assert cn.recv() == "ready"
        self.targets = {}

    def sample(self, ntarget, seed, self_rule=True):
        """Pair sums of `ntarget` random grid targets (and one random latitude of each process's self
        rule): pairs per second of the parallel timed sums (the slowest process's time)."""
        import numpy as np
        from oracle import sh
        w = self.w
        _, xs, _ = _oracle_inputs(self.name) if not hasattr(self, "_xs") else (None, self._xs, None)
        self._xs = xs
        rng = np.random.default_rng(seed)
        nd = len(w.p)
        tdrops = rng.integers(0, nd, size=ntarget)
        pts = np.zeros((3, ntarget))
        for t, i in enumerate(tdrops):
            if i not in self.targets:
                self.targets[i] = np.stack([sh.synthesize(xs[i][c], w.p[i], w.p[i]).reshape(-1) for c in range(3)])
            g = self.targets[i]
            pts[:, t] = g[:, rng.integers(0, g.shape[1])]
        for c, cn in enumerate(self.conns):
            sd = (37 * c) % nd
            cn.send((pts, tdrops, int(rng.integers(0, w.p[sd] + 1)) if self_rule else -1))
        res = [cn.recv() for cn in self.conns]
        pairs = sum(r[0] + r[2] for r in res)
        secs = max(r[1] + r[3] for r in res)
        return {"pairs": pairs, "seconds": secs, "value": pairs / max(secs, 1e-9)}

    def close(self):
        for cn in self.conns:
            try:
                cn.send(None)
            except (BrokenPipeError, OSError):
                pass
        for pr in self.procs:
            pr.join(timeout=10)


def cpu_baseline(name, pairs_per_apply, samples=3):
    """The oracle timed on one core and on every core of the host, on samples of the same workload
    (random grid targets against every drop's sources by region, plus one latitude of the singular
    rule per process); the full apply's time is extrapolated linearly from each rate."""
    cores = os.cpu_count() or 1
    nd = len(_oracle_inputs(name)[0].p)
    one = OraclePool(name, 1, stride=max(1, nd // 64))  # one process, a 1/8-ish subset of the source drops
    r1 = [one.sample(64, 10 + k) for k in range(samples)]
    one.close()
    allc = OraclePool(name, cores)
    rn = [allc.sample(32 * cores, 20 + k) for k in range(samples)]
    allc.close()
    v1 = sum(r["pairs"] for r in r1) / sum(r["seconds"] for r in r1)
    vn = sum(r["pairs"] for r in rn) / sum(r["seconds"] for r in rn)
    return {"value": vn, "unit": UNIT, "cores": cores, "kind": "oracle", "single_core_value": v1, "nproc": cores,
            "sample": f"oracle FP64 (NumPy) on {name}: per sample {32 * cores} random grid targets against every "
                      f"other drop's sources (regular / upsampled rule by region) plus one latitude of the singular "
                      f"self rule per process, {samples} samples, {cores} processes; single core: 64 targets against "
                      f"every {max(1, nd // 64)}th drop; the oracle's per-geometry preparation is not timed",
            "extrapolated_apply_s": {"all_cores": pairs_per_apply / vn, "single_core": pairs_per_apply / v1,
                                     "label": "extrapolated"}}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    name = getattr(args, "workload", "c5")
    nt = 16 * cores
    pool = OraclePool(name, cores)
    for i in range(args.warmup):
        pool.sample(cores, 50 + i)
    pairs, secs = 0, 0.0
    t0 = time.perf_counter()
    for i in range(args.steps):
        r = pool.sample(nt, 100 + i)
        pairs += r["pairs"]
        secs += r["seconds"]
    wall = time.perf_counter() - t0
    pool.close()
    v = pairs / secs
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[name], "name": name,
                   "step": f"oracle (FP64, NumPy) pair sums of {nt} random grid targets against every other drop plus "
                           f"one latitude of the singular self rule per process, on {cores} host processes"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "per step: the sample above; the oracle's per-geometry preparation not timed"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }))


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1707_02156_gb300 import api, build
    build.build()
    pctx = api.Context(local)
    peaks = alu_peaks(pctx)
    pctx.close()
    bw, bw_src = hbm_peak()
    name = args.workload
    if name == "c1":
        head = apply_line(name, local, max(args.steps, 20), args.warmup, peaks)
        head.update({"ms_per_step": head["fp64_us"] / 1e3, "gpu_launches": None})
    else:
        head = solve_line(name, local, args.steps, args.warmup, world, peaks, headline=True,
                          fp64_solve=args.fp64_solve)
    also = {}
    if not args.no_aux:
        for other in ("c1", "c2", "c3", "c4"):
            if other == name:
                continue
            if other == "c1":
                also[other] = guarded(apply_line, other, local, 20, 5, peaks)
            else:
                also[other] = guarded(solve_line, other, local, 3, 2, world, peaks, False, other in ("c2", "c3", "c4"))
    if not args.no_aux and name != "c1":
        also["offsurface_" + name] = guarded(offsurface_line, name, local, 3, 2)
    if args.timesteps:
        head["time_steps"] = guarded(time_midpoint, name, local, args.timesteps)
    cpu = guarded(cpu_baseline, name, head.get("pairs_per_apply", 1)) if (rank == 0 and not args.no_aux) else None
    res = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[name], "name": name, "step": head.get("step"),
                   "pairs_per_apply": head.get("pairs_per_apply"),
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "L2 flushed (512 MB write) before every timed step; within a step the applies re-read the "
                         "projected kernel factors and sources"},
        "e2e": head.get("e2e"),
        "gpu_launches": head.get("gpu_launches"),
        "roofline": head.get("roofline"),
        "clocks": head.get("clocks"),
        "cpu_baseline": cpu,
        "peaks": {"alu_tflops_measured": peaks, "hbm_gbs": bw, "hbm_source": bw_src},
        "detail": {k: v for k, v in head.items() if k not in ("e2e", "roofline", "clocks", "value", "gpu_launches")},
        "also": also,
    }
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    TENSOR_ROTATION = a.tensor_rotation
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    if a.impl == "reference":
        run_reference(a)
    elif a.coupled:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"workload": a.coupled, "coupled": time_coupled(a.coupled, 0)}))
    else:
        run_ours(a)
