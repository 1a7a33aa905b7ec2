"""Near-singular (Omega_2) evaluation by interpolation along the normal line (oracle; test only).

Sec. 2.3: closest point x* on the source surface by Newton on the squared distance (Eqs. f_phi,
f_theta, newton_ite, with the Levenberg-Marquardt shift of the footnote); check points further
out on the line through x* and x0; their values by the regular rule (standard grid in Omega_0,
upsampled grid otherwise); the on-surface value at x* from the SH expansion of the source
drop's own self-interaction values; one-dimensional Lagrange interpolation in the distance.

Readings of the text (not fixed by the paper):
  * check points x_l = x* + h_j sqrt(l) e, e = (x0 - x*)/|x0 - x*|, l = 1..L (the D_l = h sqrt(l)
    family of Sec. 2.3), L = 8;
  * the seed is the nearest standard grid point; Newton runs in a rotated parametrisation that
    puts the seed on the equator (theta = pi/2, phi = 0), which avoids the coordinate poles;
    mu = 1e-8 tr(H), multiplied by 10 on a rejected step, at most 30 iterations, stop when the
    step is below 1e-14;
  * the double layer's on-surface anchor is the exterior limit PV - 4 pi u(x*) in raw-integral
    units (the jump of the double-layer identity of Sec. 2.3); the single layer is continuous.
"""
from __future__ import annotations

import numpy as np

from . import sh, wigner

L_POINTS = 8


def newton_closest(xr: np.ndarray, p: int, x0: np.ndarray, th: float = np.pi / 2, ph: float = 0.0,
                   max_it: int = 30):
    """Minimise F = |x(theta,phi) - x0|^2 / 2 over the parameters of the coefficients xr [3][.]."""

    def ev(t, f):
        d = [sh.evaluate_derivs(xr[c], p, np.array([t]), np.array([f])) for c in range(3)]
        return {k: np.array([d[c][k][0] for c in range(3)]) for k in d[0]}

    def fval(t, f):
        x = np.array([sh.evaluate(xr[c], p, np.array([t]), np.array([f]))[0] for c in range(3)])
        return 0.5 * float(np.sum((x - x0) ** 2))

    d = ev(th, ph)
    F = 0.5 * float(np.sum((d["f"] - x0) ** 2))
    mu = None
    for _ in range(max_it):
        r = d["f"] - x0
        g = np.array([r @ d["t"], r @ d["p"]])
        H = np.array([[d["t"] @ d["t"] + r @ d["tt"], d["t"] @ d["p"] + r @ d["tp"]],
                      [d["t"] @ d["p"] + r @ d["tp"], d["p"] @ d["p"] + r @ d["pp"]]])
        if mu is None:
            mu = 1e-8 * abs(np.trace(H))
        accepted = False
        for _ in range(40):
            step = -np.linalg.solve(H + mu * np.eye(2), g)
            Fn = fval(th + step[0], ph + step[1])
            if Fn <= F:
                accepted = True
                break
            mu *= 10.0
        if not accepted:
            break
        th, ph = th + step[0], ph + step[1]
        d = ev(th, ph)
        F = 0.5 * float(np.sum((d["f"] - x0) ** 2))
        if np.max(np.abs(step)) < 1e-14:
            break
    return th, ph, d["f"]


def lagrange(nodes: np.ndarray, vals: np.ndarray, x: float) -> np.ndarray:
    """Lagrange interpolant through (nodes[l], vals[:, l]) evaluated at x."""
    out = np.zeros(vals.shape[0])
    for l in range(len(nodes)):
        b = 1.0
        for k in range(len(nodes)):
            if k != l:
                b *= (x - nodes[k]) / (nodes[l] - nodes[k])
        out += b * vals[:, l]
    return out


def near_data(drops, j: int, dens_j: np.ndarray, self_raw_j: np.ndarray) -> dict:
    """What the interpolation over drop j needs for any target: the density's coefficients, its
    values on the standard and upsampled grids, and the SH coefficients of drop j's own raw
    self-rule values (the on-surface values) from self_raw_j [3][p_j+1][2p_j+2]."""
    p = drops.p[j]
    dens_j = np.asarray(dens_j).reshape(3, sh.ncoef(p))
    return {"dens": dens_j,
            "self_coef": np.stack([sh.analyze(self_raw_j[c], p, p) for c in range(3)]),
            "std_rho": drops.std[j].density(dens_j),
            "up_rho": drops.ups[j].density(dens_j)}


def near_value_at(drops, j: int, x0: np.ndarray, data: dict, kind: str) -> np.ndarray:
    """Raw integral over drop j at one point x0 of its Omega_2 (outside drop j), [3]."""
    from .layer import regular_sum
    p = drops.p[j]
    h = drops.h[j]
    xj = drops.xcoef[j]
    std_x = drops.std[j].x
    _, _, theta, phi = sh.gauss_grid(p)
    T, Ph = np.meshgrid(theta, phi, indexing="ij")
    T, Ph = T.reshape(-1), Ph.reshape(-1)
    s = int(np.argmin(np.sum((std_x - x0[:, None]) ** 2, axis=0)))
    al, be = Ph[s], T[s] - np.pi / 2
    xr = np.stack([wigner.rotate(xj[c], p, al, be) for c in range(3)])
    th, ph, xs = newton_closest(xr, p, x0)
    d0 = float(np.linalg.norm(x0 - xs))
    e = (x0 - xs) / d0
    nodes = np.concatenate([[0.0], h * np.sqrt(np.arange(1, L_POINTS + 1))])
    vals = np.zeros((3, L_POINTS + 1))
    sr = np.stack([wigner.rotate(data["self_coef"][c], p, al, be) for c in range(3)])
    anchor = np.array([sh.evaluate(sr[c], p, np.array([th]), np.array([ph]))[0] for c in range(3)])
    if kind == "D":
        ur = np.stack([wigner.rotate(data["dens"][c], p, al, be) for c in range(3)])
        u_star = np.array([sh.evaluate(ur[c], p, np.array([th]), np.array([ph]))[0] for c in range(3)])
        anchor = anchor - 4.0 * np.pi * u_star
    vals[:, 0] = anchor
    pts = xs[:, None] + e[:, None] * nodes[None, 1:]
    reg = drops.classify(pts, j)
    for l in range(L_POINTS):
        if reg[l] == 0:
            vals[:, l + 1] = regular_sum(pts[:, l:l + 1], drops.std[j], data["std_rho"], kind)[:, 0]
        else:
            vals[:, l + 1] = regular_sum(pts[:, l:l + 1], drops.ups[j], data["up_rho"], kind)[:, 0]
    return lagrange(nodes, vals, d0)


def near_values(drops, i: int, j: int, sel, dens_j: np.ndarray, kind: str, self_raw_j: np.ndarray) -> np.ndarray:
    """Raw-integral values over drop j at the Omega_2 targets sel of drop i, [3][len(sel)].

    self_raw_j: drop j's own raw self-rule values on its grid, [3][p_j+1][2p_j+2].
    """
    data = near_data(drops, j, dens_j, self_raw_j)
    out = np.zeros((3, len(sel)))
    for col, t in enumerate(sel):
        out[:, col] = near_value_at(drops, j, drops.targets[i][:, t], data, kind)
    return out
