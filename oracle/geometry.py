"""Surface geometry and interfacial force (oracle; test infrastructure only).

Table 2 (fundamental forms, W, normal, curvatures), Sec. 1 (interfacial force, equation of
state), Sec. 1.3 (upsample, compute nonlinear terms, downsample).

Readings of the text:
  * Table 2 swaps the labels of the two curvatures; the mean curvature is
    K = (E N - 2 F M + G L) / (2 W^2) with E = x_phi.x_phi, F = x_phi.x_theta, G = x_theta.x_theta,
    L = x_phiphi.n, M = x_phitheta.n, N = x_thetatheta.n.
  * n = x_phi x x_theta / W in Table 2 points inward for theta measured from the pole; the text
    asks for the outward normal, so n = x_theta x x_phi / W.
  * Sign of the force: with K = -1/R on a sphere (outward normal) the printed
    f = 2 sigma K n - grad sigma combined with -1/(4pi) int f.G elongates a relaxing drop; the
    reading taken is f = -2 sigma K n - grad_gamma sigma (outward normal traction 2 sigma/R on a
    sphere, Marangoni term as printed).
  * Equation of state: Langmuir sigma = 1 + E ln(1 - x_s Gamma) when x_s > 0, else the linear
    limit sigma = 1 - E Gamma.
"""
from __future__ import annotations

import numpy as np

from . import sh


def surface_fields(xcoef: np.ndarray, p: int, p_grid: int) -> dict:
    """x and its first and second parameter derivatives on the degree-p_grid grid, [3][j][k] each."""
    comps = [sh.synthesize_derivs(xcoef[c], p, p_grid) for c in range(3)]
    return {k: np.stack([comps[c][k] for c in range(3)]) for k in comps[0]}


def forms(d: dict) -> dict:
    """Table 2 quantities from the derivative fields (arrays [3][...])."""
    xt, xp = d["t"], d["p"]
    E = np.sum(xp * xp, axis=0)
    F = np.sum(xp * xt, axis=0)
    G = np.sum(xt * xt, axis=0)
    W = np.sqrt(E * G - F * F)
    n = np.cross(xt, xp, axis=0) / W
    L = np.sum(d["pp"] * n, axis=0)
    M = np.sum(d["tp"] * n, axis=0)
    N = np.sum(d["tt"] * n, axis=0)
    K = (E * N - 2.0 * F * M + G * L) / (2.0 * W * W)
    KG = (L * N - M * M) / (W * W)
    return {"x": d["f"], "xt": xt, "xp": xp, "E": E, "F": F, "G": G, "W": W, "n": n, "K": K, "KG": KG}


def area_density(W: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """J = W / sin(theta) on a grid [j][k] (the smooth area density w.r.t. the unit sphere)."""
    return W / np.sin(theta)[:, None]


def sigma_of_gamma(gamma, elasticity, xs=0.0):
    if xs > 0.0:
        return 1.0 + elasticity * np.log(1.0 - xs * gamma)
    return 1.0 - elasticity * gamma


def dsigma_dgamma(gamma, elasticity, xs=0.0):
    if xs > 0.0:
        return -elasticity * xs / (1.0 - xs * gamma)
    return -elasticity * np.ones_like(gamma)


def interfacial_force(xcoef: np.ndarray, p: int, gcoef: np.ndarray, elasticity: float, xs: float = 0.0,
                      upsample: int = 2) -> np.ndarray:
    """f = -2 sigma K n - grad_gamma sigma as degree-p coefficients [3][(p+1)^2].

    Computed on the grid of degree upsample*(p+1)-1 and analysed back to degree p (Sec. 1.3).
    grad_gamma s = [(G s_phi - F s_theta) x_phi + (E s_theta - F s_phi) x_theta] / W^2.
    """
    P = upsample * (p + 1) - 1
    g = forms(surface_fields(xcoef, p, P))
    gd = sh.synthesize_derivs(gcoef, p, P)
    sig = sigma_of_gamma(gd["f"], elasticity, xs)
    ds = dsigma_dgamma(gd["f"], elasticity, xs)
    st, sp = ds * gd["t"], ds * gd["p"]
    E, F, G, W = g["E"], g["F"], g["G"], g["W"]
    grad = ((G * sp - F * st) * g["xp"] + (E * st - F * sp) * g["xt"]) / (W * W)
    f = -2.0 * sig * g["K"] * g["n"] - grad
    return np.stack([sh.analyze(f[c], P, p) for c in range(3)])


def volume(xcoef: np.ndarray, p: int, p_grid: int | None = None) -> float:
    """V = (1/3) int x.n dS by the regular rule of Sec. 2.1."""
    P = p_grid if p_grid is not None else p
    t, w, theta, phi = sh.gauss_grid(P)
    g = forms(surface_fields(xcoef, p, P))
    J = area_density(g["W"], theta)
    integrand = np.sum(g["x"] * g["n"], axis=0) * J
    return (np.pi / (P + 1)) * float(np.sum(w[:, None] * integrand)) / 3.0


def mean_radius(xcoef: np.ndarray, p: int) -> float:
    """R = (3V/(4 pi))^(1/3), the mean radius that sets h = R pi/(p+1) in Sec. 2.3."""
    return (3.0 * volume(xcoef, p, 2 * (p + 1) - 1) / (4.0 * np.pi)) ** (1.0 / 3.0)
