"""Thin Python binding of libbie.so (argument marshalling only).

Every step of the operator apply and the solve runs in the library's CUDA kernels; this module
only converts torch tensors to raw device pointers and checks status codes.  There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

c_int, c_double, c_ll, c_void = ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_void_p
P_int = ctypes.POINTER(ctypes.c_int)
P_double = ctypes.POINTER(ctypes.c_double)

BIE_FP64, BIE_MIXED, BIE_DF, BIE_RAW, BIE_GRID_OUT = 0, 1, 2, 0x100, 0x200
STATUS = {0: "ok", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ETIMEOUT", 6: "EOVERLAP", 7: "ENOTSUP"}


class bie_config(ctypes.Structure):
    """bie_config of bie.h: device, upsampling factor, A~, L, self-rule form, graph replay, tensor-core
    rotation."""

    _fields_ = [("device", c_int), ("upsample", c_int), ("a_tilde", c_double), ("n_interp", c_int),
                ("self_direct", c_int), ("use_graphs", c_int), ("tensor_rotation", c_int)]


class bie_geom_info(ctypes.Structure):
    """bie_geom_info of bie.h: sizes and pair counts of a geometry."""

    _fields_ = [("ndrop", c_int), ("ncoef", c_ll), ("ntarget", c_ll), ("self_pairs", c_ll), ("far_pairs", c_ll),
                ("up_pairs", c_ll), ("near_targets", c_ll), ("near_pairs", c_ll), ("cache_bytes", c_double),
                ("interdrop_tpt", c_int), ("pair_slots", c_ll)]


class bie_solve_opts(ctypes.Structure):
    """bie_solve_opts of bie.h: solve precision, tolerances, restart and refinement limits."""

    _fields_ = [("precision", c_int), ("tol", c_double), ("restart", c_int), ("max_iter", c_int),
                ("inner_tol", c_double), ("max_refine", c_int), ("residual_precision", c_int)]


class bie_solve_info(ctypes.Structure):
    """bie_solve_info of bie.h: iterations, refinements, applies per precision, residual."""

    _fields_ = [("iterations", c_int), ("refinements", c_int), ("applies_fp64", c_int), ("applies_mixed", c_int),
                ("residual", c_double), ("converged", c_int)]


class bie_phase_stat(ctypes.Structure):
    """bie_phase_stat of bie.h: one profiled phase."""

    _fields_ = [("name", ctypes.c_char * 24), ("ms", c_double), ("calls", c_ll)]


class bie_coupled_info(ctypes.Structure):
    """bie_coupled_info of bie.h: error estimates and solves of one coupled step."""

    _fields_ = [("err_drop", c_double), ("err_conservation", c_double), ("err_imex1", c_double),
                ("velocity_solves", c_int), ("implicit_iterations", c_int), ("solve", bie_solve_info * 2)]


class bie_run_info(ctypes.Structure):
    """bie_run_info of bie.h: outcome of an adaptive coupled run."""

    _fields_ = [("t", c_double), ("dt_next", c_double), ("err_max_accepted", c_double), ("steps_accepted", c_int),
                ("steps_rejected", c_int), ("velocity_solves", c_int), ("reparam_iterations", c_int)]


class bie_reparam_opts(ctypes.Structure):
    """bie_reparam_opts of bie.h: options of the angle reparametrisation (Alg. 2)."""

    _fields_ = [("u_rep", c_int), ("p_cutoff", c_double), ("smooth", c_int), ("dtau", c_double), ("eps", c_double),
                ("max_iter", c_int)]


class bie_reparam_info(ctypes.Structure):
    """bie_reparam_info of bie.h: outcome of an angle reparametrisation."""

    _fields_ = [("iterations", c_int), ("converged", c_int), ("g_max", c_double), ("energy_first_max", c_double),
                ("energy_last_max", c_double)]


BIE_ERR_CONSERVATION, BIE_ERR_IMEX1 = 0, 1
BIE_PEAK_FP32, BIE_PEAK_FP32X2, BIE_PEAK_FP64 = 0, 1, 2


EXPORTS = {
    "bie_config_default": (None, [ctypes.POINTER(bie_config)]),
    "bie_create": (c_int, [ctypes.POINTER(c_void), ctypes.POINTER(bie_config)]),
    "bie_destroy": (None, [c_void]),
    "bie_strerror": (ctypes.c_char_p, [c_int]),
    "bie_last_error": (ctypes.c_char_p, []),
    "bie_sh_analyze": (c_int, [c_void, c_int, P_int, c_int, c_void, c_void, c_void]),
    "bie_sh_synthesize": (c_int, [c_void, c_int, P_int, P_int, c_int, c_void, c_void, c_void]),
    "bie_rotate": (c_int, [c_void, c_int, P_int, c_int, c_void, P_double, c_void, c_void]),
    "bie_rotate_noalloc": (c_int, [c_void, c_int, P_int, c_int, c_void, P_double, c_void, c_void]),
    "bie_geometry_setup": (c_int, [c_void, c_int, P_int, P_int, c_void, P_double, ctypes.POINTER(c_void), c_void]),
    "bie_geometry_destroy": (None, [c_void]),
    "bie_geometry_info": (c_int, [c_void, ctypes.POINTER(bie_geom_info)]),
    "bie_interfacial_force": (c_int, [c_void, c_void, c_void, c_double, c_double, c_void, c_void]),
    "bie_apply_single": (c_int, [c_void, c_void, c_void, c_void, c_int, c_void]),
    "bie_apply_double": (c_int, [c_void, c_void, c_void, c_void, c_int, c_void]),
    "bie_rhs": (c_int, [c_void, c_void, c_void, c_void, c_void, c_int, c_void]),
    "bie_eval_single": (c_int, [c_void, c_void, c_ll, c_void, c_void, c_void, c_int, c_void]),
    "bie_eval_double": (c_int, [c_void, c_void, c_ll, c_void, c_void, c_void, c_int, c_void]),
    "bie_eval_velocity": (c_int, [c_void, c_void, c_ll, c_void, c_void, c_void, c_void, c_void, c_int, c_void]),
    "bie_solve_opts_default": (None, [ctypes.POINTER(bie_solve_opts)]),
    "bie_solve": (c_int, [c_void, c_void, c_void, c_void, ctypes.POINTER(bie_solve_opts),
                          ctypes.POINTER(bie_solve_info), c_void]),
    "bie_profile": (c_int, [c_void, c_int]),
    "bie_profile_read": (c_int, [c_void, ctypes.POINTER(bie_phase_stat), c_int, P_int]),
    "bie_launch_count": (c_ll, []),
    "bie_alu_peak": (c_int, [c_void, c_int, P_double]),
    "bie_step_midpoint": (c_int, [c_void, c_int, P_int, P_int, c_void, c_void, c_double, c_double, P_double,
                                  c_double, c_double, c_void, c_void, c_void]),
    "bie_surfactant_rates": (c_int, [c_void, c_int, P_int, c_void, c_void, c_void, c_double, c_void, c_void, c_void]),
    "bie_surfactant_implicit": (c_int, [c_void, c_int, P_int, c_void, c_void, c_double, c_void, c_double, P_int,
                                        c_void]),
    "bie_surfactant_mass": (c_int, [c_void, c_int, P_int, c_void, c_void, P_double, c_void]),
    "bie_step_coupled": (c_int, [c_void, c_int, P_int, P_int, c_void, c_void, c_void, c_int, c_double, c_double,
                                 P_double, c_double, c_double, c_double, c_int, ctypes.POINTER(bie_solve_opts),
                                 c_void, c_void, ctypes.POINTER(bie_coupled_info), c_void]),
    "bie_next_dt": (c_double, [c_double, c_double, c_double, c_double]),
    "bie_run_coupled": (c_int, [c_void, c_int, P_int, P_int, c_void, c_void, c_double, c_double, P_double, c_double,
                                c_double, c_double, c_double, c_double, c_double, c_int, c_int,
                                ctypes.POINTER(bie_solve_opts), ctypes.POINTER(bie_reparam_opts),
                                ctypes.POINTER(bie_run_info), c_void]),
    "bie_reparam_opts_default": (None, [ctypes.POINTER(bie_reparam_opts)]),
    "bie_reparametrize": (c_int, [c_void, c_int, P_int, c_void, c_void, ctypes.POINTER(bie_reparam_opts),
                                  ctypes.POINTER(bie_reparam_info), c_void]),
    "bie_debug_table": (c_ll, [c_int, c_int, c_int, c_int, c_double, P_double, c_ll]),
}

_LIB = None


def lib(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libbie.so (raises if it is missing and build_if_missing is False)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libbie.so not built ({path}); run paper_1707_02156_gb300.build")
            _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


class BIEError(RuntimeError):
    """A status other than BIE_OK from the library, with its message."""

    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}: {lib().bie_last_error().decode()}")


def _check(st: int, what: str):
    if st != 0:
        raise BIEError(st, what)


def _ptr(t: torch.Tensor) -> int:
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ints(v):
    v = [int(x) for x in v]
    return (ctypes.c_int * len(v))(*v)


def _doubles(v):
    v = [float(x) for x in v]
    return (ctypes.c_double * len(v))(*v)


def ncoef(p: int) -> int:
    """Real-packed coefficients of one scalar of degree p."""
    return (p + 1) * (p + 1)


def ngrid(p: int) -> int:
    """Points of the degree-p grid: (p+1) latitudes times 2p+2 longitudes."""
    return (p + 1) * (2 * p + 2)


class Context:
    """A library context on one CUDA device (plan tables cached per degree)."""

    def __init__(self, device: int = 0, upsample: int = 4, a_tilde: float = 5.0, n_interp: int = 8,
                 self_direct: bool = False, use_graphs: bool = True, tensor_rotation: bool = False):
        L = lib()
        cfg = bie_config()
        L.bie_config_default(ctypes.byref(cfg))
        cfg.device, cfg.upsample, cfg.a_tilde, cfg.n_interp = device, upsample, a_tilde, n_interp
        cfg.self_direct = 1 if self_direct else 0
        cfg.use_graphs = 1 if use_graphs else 0
        cfg.tensor_rotation = 1 if tensor_rotation else 0
        h = c_void()
        _check(L.bie_create(ctypes.byref(h), ctypes.byref(cfg)), "bie_create")
        self.h = h
        self.device = device

    def close(self):
        """Release the context (idempotent)."""
        if getattr(self, "h", None):
            lib().bie_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sh_analyze(self, p, ncomp: int, grid: torch.Tensor, coef: torch.Tensor):
        """Grid values [drop][comp][j][k] -> real-packed coefficients [drop][comp][(p+1)^2]."""
        _check(lib().bie_sh_analyze(self.h, len(p), _ints(p), ncomp, _ptr(grid), _ptr(coef), _stream()),
               "bie_sh_analyze")
        return coef

    def sh_synthesize(self, p, p_out, ncomp: int, coef: torch.Tensor, grid: torch.Tensor):
        """Coefficients of degree p -> values on the grid of degree p_out >= p (zero padding)."""
        _check(lib().bie_sh_synthesize(self.h, len(p), _ints(p), _ints(p_out), ncomp, _ptr(coef), _ptr(grid),
                                       _stream()), "bie_sh_synthesize")
        return grid

    def rotate(self, p, ncomp: int, coef: torch.Tensor, euler, out: torch.Tensor):
        """Coefficients of f(R s), R = R_z(alpha) R_y(beta) R_z(gamma), per drop (euler [drop][3])."""
        flat = [float(a) for e in euler for a in e]
        _check(lib().bie_rotate(self.h, len(p), _ints(p), ncomp, _ptr(coef), _doubles(flat), _ptr(out), _stream()),
               "bie_rotate")
        return out

    def profile(self, enable: bool):
        """Start (True) or stop (False) per-phase CUDA-event timing inside the library."""
        _check(lib().bie_profile(self.h, 1 if enable else 0), "bie_profile")

    def profile_read(self) -> dict:
        """Per-phase {name: (total_ms, calls)} since profiling started; clears the record."""
        buf = (bie_phase_stat * 32)()
        n = ctypes.c_int()
        _check(lib().bie_profile_read(self.h, buf, 32, ctypes.byref(n)), "bie_profile_read")
        return {buf[i].name.decode(): (buf[i].ms, buf[i].calls) for i in range(min(n.value, 32))}

    def rotate_noalloc(self, p, ncomp: int, coef: torch.Tensor, euler, out: torch.Tensor):
        """bie_rotate without device allocation (tables staged in the library's fixed device array)."""
        flat = [float(a) for e in euler for a in e]
        _check(lib().bie_rotate_noalloc(self.h, len(p), _ints(p), ncomp, _ptr(coef), _doubles(flat), _ptr(out),
                                        _stream()), "bie_rotate_noalloc")
        return out

    def alu_peak(self, which: int) -> float:
        """Measured rate in TFLOP/s of FP32 FMA (0), packed FP32 FMA f32x2 (1) or FP64 FMA (2) on this
        context's GPU (bie_alu_peak)."""
        v = ctypes.c_double()
        _check(lib().bie_alu_peak(self.h, int(which), ctypes.byref(v)), "bie_alu_peak")
        return v.value

    def geometry(self, p, pq, xcoef: torch.Tensor, lam) -> "Geometry":
        """Set up the shape-dependent data of the drops (see Geometry)."""
        return Geometry(self, p, pq, xcoef, lam)


class Geometry:
    """Shape-dependent data of ndrop drops, reused by every apply and solve on that shape."""

    def __init__(self, ctx: Context, p, pq, xcoef: torch.Tensor, lam):
        self.ctx = ctx
        self.p, self.pq = list(p), list(pq)
        h = c_void()
        _check(lib().bie_geometry_setup(ctx.h, len(p), _ints(p), _ints(pq), _ptr(xcoef), _doubles(lam),
                                        ctypes.byref(h), _stream()), "bie_geometry_setup")
        self.h = h
        info = bie_geom_info()
        _check(lib().bie_geometry_info(self.h, ctypes.byref(info)), "bie_geometry_info")
        self.info = {k: getattr(info, k) for k, _ in bie_geom_info._fields_}

    def close(self):
        """Release the geometry (idempotent)."""
        if getattr(self, "h", None):
            lib().bie_geometry_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_single(self, f: torch.Tensor, out: torch.Tensor, precision: int = BIE_FP64, raw: bool = False,
                     grid_out: bool = False):
        """out = -(1/4pi) sum_j int f.G (raw: (1/8pi) int G.f) projected on the SH basis, or at the grid
        targets with grid_out."""
        flag = precision | (BIE_RAW if raw else 0) | (BIE_GRID_OUT if grid_out else 0)
        _check(lib().bie_apply_single(self.ctx.h, self.h, _ptr(f), _ptr(out), flag, _stream()), "bie_apply_single")
        return out

    def apply_double(self, u: torch.Tensor, out: torch.Tensor, precision: int = BIE_FP64, raw: bool = False,
                     grid_out: bool = False):
        """out = (1/4pi) sum_j (lambda_j - 1) PV int u.T.n (raw: (1/4pi) PV int u.T.n) projected on the
        SH basis, or at the grid targets with grid_out."""
        flag = precision | (BIE_RAW if raw else 0) | (BIE_GRID_OUT if grid_out else 0)
        _check(lib().bie_apply_double(self.ctx.h, self.h, _ptr(u), _ptr(out), flag, _stream()), "bie_apply_double")
        return out

    def eval_single(self, points: torch.Tensor, f: torch.Tensor, out: torch.Tensor, precision: int = BIE_FP64,
                    raw: bool = False):
        """S[f] at fluid points off the surfaces: points and out [3][n] (FP64, device, contiguous)."""
        n = points.numel() // 3
        _check(lib().bie_eval_single(self.ctx.h, self.h, n, _ptr(points), _ptr(f), _ptr(out),
                                     precision | (BIE_RAW if raw else 0), _stream()), "bie_eval_single")
        return out

    def eval_double(self, points: torch.Tensor, u: torch.Tensor, out: torch.Tensor, precision: int = BIE_FP64,
                    raw: bool = False):
        """D[u] at fluid points off the surfaces: points and out [3][n] (FP64, device, contiguous)."""
        n = points.numel() // 3
        _check(lib().bie_eval_double(self.ctx.h, self.h, n, _ptr(points), _ptr(u), _ptr(out),
                                     precision | (BIE_RAW if raw else 0), _stream()), "bie_eval_double")
        return out

    def velocity_at(self, points: torch.Tensor, f: torch.Tensor, u: torch.Tensor, out: torch.Tensor,
                    uinf: torch.Tensor | None = None, precision: int = BIE_FP64):
        """u_inf + (S[f] + D[u]) / 2 at fluid points [3][n]; uinf: far-field values there or None."""
        n = points.numel() // 3
        _check(lib().bie_eval_velocity(self.ctx.h, self.h, n, _ptr(points), _ptr(f), _ptr(u),
                                       _ptr(uinf) if uinf is not None else None, _ptr(out), precision, _stream()),
               "bie_eval_velocity")
        return out

    def interfacial_force(self, gamma: torch.Tensor, elasticity: float, x_s: float, out: torch.Tensor):
        """out = f = sigma (div n) n - grad sigma of the surfactant gamma (Langmuir, or linear for x_s = 0)."""
        _check(lib().bie_interfacial_force(self.ctx.h, self.h, _ptr(gamma), elasticity, x_s, _ptr(out), _stream()),
               "bie_interfacial_force")
        return out

    def rhs(self, uinf: torch.Tensor, f: torch.Tensor, out: torch.Tensor, precision: int = BIE_FP64):
        """out = 2 u_inf + S[f], the right-hand side of the boundary integral equation (S at BIE_FP64
        or BIE_DF, both FP64-grade)."""
        _check(lib().bie_rhs(self.ctx.h, self.h, _ptr(uinf), _ptr(f), _ptr(out), precision, _stream()), "bie_rhs")
        return out

    def solve(self, rhs: torch.Tensor, u: torch.Tensor, precision: int = BIE_FP64, tol: float = 1e-10,
              restart: int = 30, max_iter: int = 300, inner_tol: float = 1e-5, max_refine: int = 10,
              residual_precision: int = BIE_DF, raise_on_noconv: bool = True) -> dict:
        """Solve (lambda + 1) u - D[u] = rhs; u holds the initial guess and receives the solution."""
        o = _solve_opts(precision, tol, restart, max_iter, inner_tol, max_refine, residual_precision)
        info = bie_solve_info()
        st = lib().bie_solve(self.ctx.h, self.h, _ptr(rhs), _ptr(u), ctypes.byref(o), ctypes.byref(info), _stream())
        res = {k: getattr(info, k) for k, _ in bie_solve_info._fields_}
        if st == 4 and not raise_on_noconv:
            return res
        _check(st, "bie_solve")
        return res


def midpoint_step(ctx: "Context", p, pq, x: torch.Tensor, gamma: torch.Tensor, elasticity: float, x_s: float, lam,
                  shear: float, dt: float, precision: int = BIE_MIXED, tol: float = 1e-10, restart: int = 30,
                  max_iter: int = 300, inner_tol: float = 1e-5, max_refine: int = 10,
                  residual_precision: int = BIE_DF) -> list:
    """One midpoint step of the drop shapes x (updated in place); returns the infos of the two solves."""
    n = len(p)
    P = (ctypes.c_int * n)(*[int(v) for v in p])
    PQ = (ctypes.c_int * n)(*[int(v) for v in pq])
    L = (ctypes.c_double * n)(*[float(v) for v in lam])
    o = _solve_opts(precision, tol, restart, max_iter, inner_tol, max_refine, residual_precision)
    info = (bie_solve_info * 2)()
    _check(lib().bie_step_midpoint(ctx.h, n, P, PQ, _ptr(x), _ptr(gamma), elasticity, x_s, L, shear, dt,
                                   ctypes.byref(o), info, _stream()), "bie_step_midpoint")
    return [{k: getattr(info[i], k) for k, _ in bie_solve_info._fields_} for i in range(2)]


def _solve_opts(precision, tol, restart, max_iter, inner_tol, max_refine, residual_precision):
    o = bie_solve_opts()
    lib().bie_solve_opts_default(ctypes.byref(o))
    o.precision, o.tol, o.restart, o.max_iter, o.inner_tol, o.max_refine, o.residual_precision = (
        precision, tol, restart, max_iter, inner_tol, max_refine, residual_precision)
    return o


def surfactant_rates(ctx: "Context", p, x: torch.Tensor, u: torch.Tensor, gamma: torch.Tensor, inv_pe: float,
                     fe: torch.Tensor, fi: torch.Tensor = None):
    """fe = projection of f_E(x, u, Gamma); fi (optional) = projection of inv_pe * lap Gamma."""
    _check(lib().bie_surfactant_rates(ctx.h, len(p), _ints(p), _ptr(x), _ptr(u), _ptr(gamma), inv_pe, _ptr(fe),
                                      _ptr(fi) if fi is not None else None, _stream()), "bie_surfactant_rates")
    return fe, fi


def surfactant_implicit(ctx: "Context", p, x: torch.Tensor, b: torch.Tensor, a: float, y: torch.Tensor,
                        tol: float = 1e-13) -> int:
    """y with y - a P[lap_x y] = b (preconditioned GMRES); returns the iteration count."""
    it = ctypes.c_int(0)
    _check(lib().bie_surfactant_implicit(ctx.h, len(p), _ints(p), _ptr(x), _ptr(b), a, _ptr(y), tol,
                                         ctypes.byref(it), _stream()), "bie_surfactant_implicit")
    return it.value


def surfactant_mass(ctx: "Context", p, x: torch.Tensor, gamma: torch.Tensor) -> list:
    """Surfactant mass of each drop (regular rule on the grid of degree 2p+1)."""
    out = (ctypes.c_double * len(p))()
    _check(lib().bie_surfactant_mass(ctx.h, len(p), _ints(p), _ptr(x), _ptr(gamma), out, _stream()),
           "bie_surfactant_mass")
    return list(out)


def coupled_step(ctx: "Context", p, pq, x: torch.Tensor, gamma: torch.Tensor, u0: torch.Tensor, u0_valid: bool,
                 elasticity: float, x_s: float, lam, shear: float, inv_pe: float, dt: float, x_out: torch.Tensor,
                 gamma_out: torch.Tensor, imex1_estimate: bool = False, precision: int = BIE_MIXED,
                 tol: float = 1e-10, restart: int = 30, max_iter: int = 300, inner_tol: float = 1e-5,
                 max_refine: int = 10, residual_precision: int = BIE_DF) -> dict:
    """One step of Alg. 1 (midpoint shapes, IMEX-2 surfactant) into x_out, gamma_out; u0 holds u^t."""
    o = _solve_opts(precision, tol, restart, max_iter, inner_tol, max_refine, residual_precision)
    info = bie_coupled_info()
    _check(lib().bie_step_coupled(ctx.h, len(p), _ints(p), _ints(pq), _ptr(x), _ptr(gamma), _ptr(u0),
                                  1 if u0_valid else 0, elasticity, x_s, _doubles(lam), shear, inv_pe, dt,
                                  1 if imex1_estimate else 0, ctypes.byref(o), _ptr(x_out), _ptr(gamma_out),
                                  ctypes.byref(info), _stream()), "bie_step_coupled")
    res = {k: getattr(info, k) for k, _ in bie_coupled_info._fields_ if k != "solve"}
    res["solve"] = [{k: getattr(info.solve[i], k) for k, _ in bie_solve_info._fields_} for i in range(2)]
    return res


def next_dt(dt: float, err: float, tol: float, dt_max: float) -> float:
    """Step-size rule of Alg. 1."""
    return float(lib().bie_next_dt(dt, err, tol, dt_max))


def run_coupled(ctx: "Context", p, pq, x: torch.Tensor, gamma: torch.Tensor, elasticity: float, x_s: float, lam,
                shear: float, inv_pe: float, T: float, dt0: float, tol: float, dt_max: float,
                estimator: int = BIE_ERR_CONSERVATION, max_steps: int = 1000, precision: int = BIE_MIXED,
                solve_tol: float = 1e-10, restart: int = 30, max_iter: int = 300, inner_tol: float = 1e-5,
                max_refine: int = 10, residual_precision: int = BIE_DF, reparam: dict | None = None) -> dict:
    """Alg. 1 from 0 to T with adaptive dt; x and gamma are updated in place.  reparam: None, or the
    options of reparametrize (u_rep, p_cutoff, smooth, dtau, eps, max_iter) applied after every kept
    step."""
    o = _solve_opts(precision, solve_tol, restart, max_iter, inner_tol, max_refine, residual_precision)
    info = bie_run_info()
    ro = _reparam_opts(**reparam) if reparam is not None else None
    _check(lib().bie_run_coupled(ctx.h, len(p), _ints(p), _ints(pq), _ptr(x), _ptr(gamma), elasticity, x_s,
                                 _doubles(lam), shear, inv_pe, T, dt0, tol, dt_max, estimator, max_steps,
                                 ctypes.byref(o), ctypes.byref(ro) if ro is not None else None, ctypes.byref(info),
                                 _stream()), "bie_run_coupled")
    return {k: getattr(info, k) for k, _ in bie_run_info._fields_}


def _reparam_opts(u_rep: int = 2, p_cutoff: float = 0.05, smooth: bool = False, dtau: float = 0.5, eps: float = 1e-10,
                  max_iter: int = 200) -> bie_reparam_opts:
    o = bie_reparam_opts()
    lib().bie_reparam_opts_default(ctypes.byref(o))
    o.u_rep, o.p_cutoff, o.smooth, o.dtau, o.eps, o.max_iter = u_rep, p_cutoff, 1 if smooth else 0, dtau, eps, max_iter
    return o


def reparametrize(ctx: "Context", p, x: torch.Tensor, gamma: torch.Tensor | None = None, **opts) -> dict:
    """Angle reparametrisation (Alg. 2) of the drops' shapes x and surfactant gamma, in place; opts as
    _reparam_opts.  Returns the bie_reparam_info fields."""
    o = _reparam_opts(**opts)
    info = bie_reparam_info()
    _check(lib().bie_reparametrize(ctx.h, len(p), _ints(p), _ptr(x), _ptr(gamma) if gamma is not None else None,
                                   ctypes.byref(o), ctypes.byref(info), _stream()), "bie_reparametrize")
    return {k: getattr(info, k) for k, _ in bie_reparam_info._fields_}


def launch_count() -> int:
    """Kernels launched by libbie.so in this process."""
    return int(lib().bie_launch_count())


def debug_table(which: int, a: int, b: int = 0, c: int = 0, x: float = 0.0):
    """Host plan tables of the library (no GPU needed), as a Python list."""
    L = lib()
    n = L.bie_debug_table(which, a, b, c, x, None, 0)
    if n < 0:
        raise ValueError("bad table request")
    buf = (ctypes.c_double * n)()
    L.bie_debug_table(which, a, b, c, x, buf, n)
    return list(buf)
