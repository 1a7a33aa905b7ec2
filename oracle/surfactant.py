"""Insoluble surfactant on the drop surfaces: transport terms, the IMEX time step and the coupled
drop/surfactant step with adaptive dt (oracle; test infrastructure only).

Sec. 1 (Eq. surfactant0: convection, diffusion and stretching of Gamma; the equation of state),
Sec. 1.2 (Eq. galerkin_surfactant: the terms are formed on the grid and projected on the SH
basis), Sec. 3 (the second-order IMEX scheme, Eqs. systemforgammatpdt2 and gammatpiudt; the
first-order IMEX estimate, Eq. err_IMEX1; the conservation error, Eq. err_conservation; the
preconditioned implicit solve; Alg. 1 with its step-size rule).

Surface calculus in the parameters (theta, phi) of x, in textbook coordinate form (the paper does
not print it).  Metric g = [[G, F], [F, E]] in the order (theta, phi) with G = x_t.x_t, F = x_t.x_p,
E = x_p.x_p, W^2 = E G - F^2, inverse g^-1 = [[E, -F], [-F, G]] / W^2; summation over i, j:
    grad s = g^ij s_j x_i
    div v  = g^ij x_i . v_j
    lap s  = g^ij (s_ij - x_ij . grad s)        (the Christoffel term written with grad s)
All terms are formed on the grid of degree 2(p+1) - 1 and analysed back to degree p (Sec. 1.3).

Readings of the text:
  * The surface points move with the full velocity (dx/dt = u, Sec. 3), so Gamma is followed at
    fixed parameters.  Next to the term div(Gamma u_tan) of Eq. surfactant0 this adds
    +u_tan . grad Gamma, the rate at which tangentially moving points sample Gamma.  With it a
    rotating drop keeps any Gamma fixed (the convection test of Sec. 5), and the surfactant mass
    is conserved.
  * Stretching term.  Its printed sign clashes with the expanding-sphere test of Sec. 5
    (Gamma R^2 = Gamma(0), stretching term (div n)(u.n) = (2/R) dR/dt).  With the outward normal
    and K = -1/R on a sphere (the reading taken for the force) the term is -2 K Gamma (u.n) on the
    left-hand side.  Altogether
        f_E = -div(Gamma u_tan) + u_tan . grad Gamma + 2 K Gamma (u.n)      (= -Gamma div u),
        f_I = (1/Pe) lap Gamma.
  * The implicit solve at t + dt/2 uses the Laplacian of the surface x^(t+dt/2) (the stage at
    which Eq. systemforgammatpdt2 evaluates it).  Its preconditioner is the diagonal of the same
    operator on the sphere of the drop's mean radius R: 1 + a n(n+1)/R^2, a = dt/(2 Pe).
  * The drop update is the midpoint rule of the Butcher tableau, x^(t+dt) = x^t + dt u^(t+dt/2)
    (Alg. 1 prints x^(t+dt/2) + dt u^(t+dt/2)).  Its drop error is the embedded first-order
    (Euler) estimate of the same tableau, ||x^(t+dt) - (x^t + dt u^t)||_inf / ||x^(t+dt)||_inf.
  * Norms and mass integrals are taken on the grid: the infinity norms on the degree-p grid, the
    mass by the regular rule (Sec. 2.1) on the degree 2(p+1) - 1 grid.
  * The step size follows Alg. 1: err = max(err_drop, err_surfactant); the step is kept when
    err < tol; then dt <- min(dt_max, dt (0.9 tol/err)^(1/2)), with the last step cut to end at T.
    A kept step is followed, when asked for, by the angle reparametrisation of Sec. 4 (Alg. 2)
    of every drop's shape and surfactant, as the adaptivity box of Alg. 1 does.
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry, gmres, sh


def grid_degree(p: int) -> int:
    return 2 * (p + 1) - 1


# ----------------------------------------------------------------------------------------------
# surface calculus on the grid of degree P
# ----------------------------------------------------------------------------------------------

class Surface:
    """Derivatives, metric, normal and its derivatives of x on the degree-P grid."""

    def __init__(self, xcoef: np.ndarray, p: int, P: int):
        xcoef = np.asarray(xcoef, dtype=np.float64).reshape(3, sh.ncoef(p))
        self.p, self.P = p, P
        d = geometry.surface_fields(xcoef, p, P)
        g = geometry.forms(d)
        self.d = d
        self.x, self.xt, self.xp = d["f"], d["t"], d["p"]
        self.G = np.sum(self.xt * self.xt, axis=0)
        self.F = np.sum(self.xt * self.xp, axis=0)
        self.E = np.sum(self.xp * self.xp, axis=0)
        W2 = self.E * self.G - self.F * self.F
        self.W = np.sqrt(W2)
        self.gtt, self.gtp, self.gpp = self.E / W2, -self.F / W2, self.G / W2
        self.K = g["K"]
        c = np.cross(self.xt, self.xp, axis=0)
        ct = np.cross(d["tt"], self.xp, axis=0) + np.cross(self.xt, d["tp"], axis=0)
        cp = np.cross(d["tp"], self.xp, axis=0) + np.cross(self.xt, d["pp"], axis=0)
        self.n = c / self.W
        self.nt = ct / self.W - c * (np.sum(c * ct, axis=0) / self.W ** 3)
        self.np_ = cp / self.W - c * (np.sum(c * cp, axis=0) / self.W ** 3)
        _, w, theta, _ = sh.gauss_grid(P)
        self.J = geometry.area_density(self.W, theta)
        self.wq = (np.pi / (P + 1)) * w[:, None] * self.J  # regular rule weights times J

    def grad(self, s_t, s_p):
        a = self.gtt * s_t + self.gtp * s_p
        b = self.gtp * s_t + self.gpp * s_p
        return a * self.xt + b * self.xp

    def div(self, v_t, v_p):
        dot = lambda u, v: np.sum(u * v, axis=0)
        return (self.gtt * dot(self.xt, v_t) + self.gtp * (dot(self.xt, v_p) + dot(self.xp, v_t))
                + self.gpp * dot(self.xp, v_p))

    def lap(self, s: dict):
        gs = self.grad(s["t"], s["p"])
        dot = lambda u, v: np.sum(u * v, axis=0)
        return (self.gtt * (s["tt"] - dot(self.d["tt"], gs)) + 2.0 * self.gtp * (s["tp"] - dot(self.d["tp"], gs))
                + self.gpp * (s["pp"] - dot(self.d["pp"], gs)))

    def integral(self, s):
        return float(np.sum(self.wq * s))


def scalar_fields(coef: np.ndarray, p: int, P: int) -> dict:
    return sh.synthesize_derivs(np.asarray(coef, dtype=np.float64), p, P)


def vector_fields(coef: np.ndarray, p: int, P: int) -> dict:
    coef = np.asarray(coef, dtype=np.float64).reshape(3, sh.ncoef(p))
    comps = [sh.synthesize_derivs(coef[c], p, P) for c in range(3)]
    return {k: np.stack([comps[c][k] for c in range(3)]) for k in comps[0]}


# ----------------------------------------------------------------------------------------------
# the two right-hand sides of Eq. surfactant0 (Sec. 3: f_E explicit, f_I implicit)
# ----------------------------------------------------------------------------------------------

def f_explicit_grid(S: Surface, ucoef, gcoef, p: int) -> np.ndarray:
    """f_E = -div(Gamma u_tan) + u_tan . grad Gamma + 2 K Gamma (u.n) on the grid of S."""
    u = vector_fields(ucoef, p, S.P)
    gam = scalar_fields(gcoef, p, S.P)
    n, nt, np_ = S.n, S.nt, S.np_
    un = np.sum(u["f"] * n, axis=0)
    utan = u["f"] - un * n
    utan_t = u["t"] - (np.sum(u["t"] * n, axis=0) + np.sum(u["f"] * nt, axis=0)) * n - un * nt
    utan_p = u["p"] - (np.sum(u["p"] * n, axis=0) + np.sum(u["f"] * np_, axis=0)) * n - un * np_
    G = gam["f"]
    flux_t = gam["t"] * utan + G * utan_t
    flux_p = gam["p"] * utan + G * utan_p
    conv = S.div(flux_t, flux_p)
    frame = np.sum(utan * S.grad(gam["t"], gam["p"]), axis=0)
    stretch = 2.0 * S.K * G * un
    return -conv + frame + stretch


def f_explicit(xcoef, ucoef, gcoef, p: int) -> np.ndarray:
    """Galerkin projection (Eq. galerkin_surfactant) of f_E: degree-p coefficients."""
    P = grid_degree(p)
    return sh.analyze(f_explicit_grid(Surface(xcoef, p, P), ucoef, gcoef, p), P, p)


def lap_coef(S: Surface, gcoef, p: int) -> np.ndarray:
    """Galerkin projection of lap Gamma on the surface S: degree-p coefficients."""
    return sh.analyze(S.lap(scalar_fields(gcoef, p, S.P)), S.P, p)


def f_implicit(xcoef, gcoef, p: int, pe: float) -> np.ndarray:
    """f_I = (1/Pe) lap Gamma, projected (zero for Pe = inf)."""
    if math.isinf(pe):
        return np.zeros(sh.ncoef(p))
    return lap_coef(Surface(xcoef, p, grid_degree(p)), gcoef, p) / pe


def mass(xcoef, gcoef, p: int) -> float:
    """int_gamma Gamma dS by the regular rule on the degree 2(p+1)-1 grid."""
    S = Surface(xcoef, p, grid_degree(p))
    return S.integral(scalar_fields(gcoef, p, S.P)["f"])


# ----------------------------------------------------------------------------------------------
# the implicit system (I - a lap) y = b of Sec. 3 (Preconditioning)
# ----------------------------------------------------------------------------------------------

def degrees(p: int) -> np.ndarray:
    """Degree n of each real-packed coefficient."""
    return np.concatenate([np.full(2 * n + 1, n) for n in range(p + 1)]).astype(np.float64)


def solve_implicit(xcoef, b, p: int, a: float, precondition: bool = True, tol: float = 1e-13):
    """y with y - a lap y = b (coefficients, Galerkin), GMRES left-preconditioned by the sphere's
    diagonal 1 + a n(n+1)/R^2 (R the mean radius).  Returns (y, iterations)."""
    b = np.asarray(b, dtype=np.float64)
    if a == 0.0:
        return b.copy(), 0
    S = Surface(xcoef, p, grid_degree(p))
    R = geometry.mean_radius(np.asarray(xcoef).reshape(3, -1), p)
    nn = degrees(p)
    diag = 1.0 + a * nn * (nn + 1.0) / (R * R) if precondition else np.ones_like(nn)
    A = lambda y: (y - a * lap_coef(S, y, p)) / diag
    y, info = gmres.gmres(A, b / diag, tol=tol, restart=60, max_it=600)
    assert info["converged"]
    return y, info["iterations"]


# ----------------------------------------------------------------------------------------------
# IMEX schemes (Sec. 3) and the coupled step (Alg. 1)
# ----------------------------------------------------------------------------------------------

def imex2_half(x0, u0, xh, g0, p: int, pe: float, dt: float, precondition: bool = True):
    """First stage of the second-order IMEX step (Eq. systemforgammatpdt2):
    k0~ = f_E(x^t, u^t, Gamma^t), then Gamma_h - (dt/2) f_I(x_h, Gamma_h) = Gamma^t + (dt/2) k0~.
    Returns (Gamma_h, k0~)."""
    k0 = f_explicit(x0, u0, g0, p)
    a = 0.0 if math.isinf(pe) else 0.5 * dt / pe
    gh, _ = solve_implicit(xh, g0 + 0.5 * dt * k0, p, a, precondition)
    return gh, k0


def imex2_full(xh, uh, gh, g0, p: int, pe: float, dt: float):
    """Second stage (Eq. gammatpiudt): Gamma^(t+dt) = Gamma^t + dt (f_E(x_h, u_h, Gamma_h) + f_I(x_h, Gamma_h))."""
    return g0 + dt * (f_explicit(xh, uh, gh, p) + f_implicit(xh, gh, p, pe))


def imex2(x0, u0, xh, uh, g0, p: int, pe: float, dt: float, precondition: bool = True):
    """Both stages of the second-order IMEX step of Gamma, given the drop stages (x^t, u^t) and
    (x^(t+dt/2), u^(t+dt/2)).  Returns (Gamma_h, Gamma^(t+dt), k0~)."""
    gh, k0 = imex2_half(x0, u0, xh, g0, p, pe, dt, precondition)
    return gh, imex2_full(xh, uh, gh, g0, p, pe, dt), k0


def imex1(x1, g0, k0, p: int, pe: float, dt: float):
    """First-order IMEX estimate: Gamma_1 - dt f_I(x^(t+dt), Gamma_1) = Gamma^t + dt k0~ (Eq. err_IMEX1)."""
    a = 0.0 if math.isinf(pe) else dt / pe
    g1, _ = solve_implicit(x1, g0 + dt * k0, p, a)
    return g1


def grid_inf(coef, p: int) -> float:
    coef = np.asarray(coef).reshape(-1, sh.ncoef(p))
    return max(float(np.max(np.abs(sh.synthesize(c, p, p)))) for c in coef)


def coupled_step(xs, gs, ps, dt: float, velocity, pe: float, u0=None, imex1_estimate: bool = False):
    """One step of Alg. 1 for all drops.

    velocity(x_list, gamma_list) -> u_list (coefficients [3][(p+1)^2] per drop) is the solve of
    Eq. main_eq at those shapes and concentrations (or any prescribed field).  u0 may carry the
    velocity at (x^t, Gamma^t) from an earlier rejected attempt.
    """
    xs = [np.asarray(x, dtype=np.float64).reshape(3, -1) for x in xs]
    gs = [np.asarray(g, dtype=np.float64).reshape(-1) for g in gs]
    calls = 0
    if u0 is None:
        u0 = velocity(xs, gs)
        calls += 1
    xh = [x + 0.5 * dt * u for x, u in zip(xs, u0)]
    # Gamma at t + dt/2 needs only the explicit term at t and the Laplacian of x^(t+dt/2)
    half = [imex2_half(x, u, xm, g, p, pe, dt) for x, u, xm, g, p in zip(xs, u0, xh, gs, ps)]
    ghs = [h[0] for h in half]
    k0s = [h[1] for h in half]
    uh = velocity(xh, ghs)
    calls += 1
    x1 = [x + dt * u for x, u in zip(xs, uh)]
    g1s = [imex2_full(xm, u, gh, g, p, pe, dt) for xm, u, gh, g, p in zip(xh, uh, ghs, gs, ps)]
    err_drop = max(grid_inf(dt * (b - a), p) / grid_inf(xn, p) for a, b, xn, p in zip(u0, uh, x1, ps))
    err_cons = max(abs(mass(xn, gn, p) - mass(x, g, p)) / abs(mass(x, g, p))
                   for x, g, xn, gn, p in zip(xs, gs, x1, g1s, ps))
    out = {"x": x1, "gamma": g1s, "u0": u0, "uh": uh, "xh": xh, "gamma_h": ghs, "calls": calls,
           "err_drop": err_drop, "err_conservation": err_cons}
    if imex1_estimate:
        out["err_imex1"] = max(grid_inf(gn - imex1(xn, g, k0, p, pe, dt), p) / grid_inf(gn, p)
                               for xn, gn, g, k0, p in zip(x1, g1s, gs, k0s, ps))
    return out


def next_dt(dt: float, err: float, tol: float, dt_max: float) -> float:
    """Alg. 1: dt (0.9 tol/err)^(1/2), capped at dt_max."""
    if err <= 0.0:
        return dt_max
    return min(dt_max, dt * math.sqrt(0.9 * tol / err))


def run_adaptive(xs, gs, ps, T: float, dt0: float, tol: float, velocity, pe: float, dt_max: float,
                 estimator: str = "conservation", max_steps: int = 1000, reparam: dict | None = None):
    """Alg. 1 from t = 0 to T.  Returns the final shapes and concentrations and the step history.

    reparam: None, or the options of reparam.reparametrize (u_rep, p_cutoff, dtau, eps, i_max)
    applied to every drop after each kept step."""
    t, dt = 0.0, min(dt0, dt_max)
    xs = [np.asarray(x, dtype=np.float64).reshape(3, -1) for x in xs]
    gs = [np.asarray(g, dtype=np.float64).reshape(-1) for g in gs]
    u0 = None
    hist = []
    calls = 0
    for _ in range(max_steps):
        if t >= T * (1.0 - 1e-14):
            break
        h = min(dt, T - t)
        st = coupled_step(xs, gs, ps, h, velocity, pe, u0=u0, imex1_estimate=estimator == "imex1")
        calls += st["calls"]
        u0 = st["u0"]
        err_s = st["err_imex1"] if estimator == "imex1" else st["err_conservation"]
        err = max(st["err_drop"], err_s)
        accepted = err < tol
        hist.append({"t": t, "dt": h, "err": err, "err_drop": st["err_drop"], "err_surfactant": err_s,
                     "accepted": accepted})
        if accepted:
            t += h
            xs, gs, u0 = st["x"], st["gamma"], None
            if reparam is not None:
                from . import reparam as rp
                out = [rp.reparametrize(x, g, p, **reparam)[:2] for x, g, p in zip(xs, gs, ps)]
                xs, gs = [o[0] for o in out], [o[1] for o in out]
        dt = next_dt(h, err, tol, dt_max)
    return {"x": xs, "gamma": gs, "t": t, "dt_next": dt, "history": hist, "velocity_calls": calls}
