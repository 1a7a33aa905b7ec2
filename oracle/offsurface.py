"""Layer potentials and the velocity at points off the drop surfaces (oracle; test infrastructure
only: imported by tests/, the package's smoke check and bench.py's CPU baseline, never by the
product path).

Sec. 1: the velocity can be evaluated anywhere in the domain from the surface densities once the
interface velocity is known.  The same representation that gives Eq. main_eq on the interfaces
gives, at a point x0 of the fluid (outside every drop), the factor 1 instead of (lambda_i + 1)/2:

    u(x0) = u_inf(x0) - (1/8pi) sum_j int f.G ds + sum_j ((lambda_j - 1)/8pi) int u.T.n ds
          = u_inf(x0) + (S[f](x0) + D[u](x0)) / 2,

with S and D normalised as the operators of Eq. main_eq (oracle/layer.py): S[f] = -(1/4pi) sum_j
int f.G, D[u] = (1/4pi) sum_j (lambda_j - 1) int u.T.n.  At a fluid point the double-layer integral
is an ordinary integral; its limit from outside at an interface point x is PV - 4pi u(x) in raw units,
and (1 + (lambda - 1)/2) = (lambda + 1)/2 then recovers Eq. main_eq.

Each (point, drop j) pair takes the rule of its region of Sec. 2.3: the regular rule on the standard
grid in Omega_0, on the upsampled grid in Omega_1, and in Omega_2 the interpolation along the line
through the closest surface point (oracle/near.py), whose anchor is the exterior limit.

Readings (the paper evaluates only interface points):
  * a point lies inside drop j when it is on the inner side of the tangent plane at the nearest
    point of drop j's upsampled grid; inside points are rejected (the interior representation
    and the interior limit of the interpolation are not part of the method);
  * a single-drop set builds the upsampled grid that oracle.layer.Drops leaves out for N = 1.
"""
from __future__ import annotations

import numpy as np

from . import near
from .layer import DropGrid, regular_sum

INSIDE = 3


def _ensure_upsampled(drops):
    if not drops.ups:
        drops.ups = [DropGrid(x, p, drops.up * (p + 1) - 1) for x, p in zip(drops.xcoef, drops.p)]


def classify_points(drops, pts: np.ndarray, j: int) -> np.ndarray:
    """0, 1, 2 for Omega_0/1/2 of each point [3][n] with respect to drop j, 3 inside drop j."""
    _ensure_upsampled(drops)
    up = drops.ups[j]
    codes = np.zeros(pts.shape[1], dtype=np.int64)
    for s in range(0, pts.shape[1], 256):
        diff = pts[:, s:s + 256, None] - up.x[:, None, :]
        d2 = np.sum(diff * diff, axis=0)
        k = np.argmin(d2, axis=1)
        dist = np.sqrt(d2[np.arange(len(k)), k])
        side = np.sum((pts[:, s:s + 256] - up.x[:, k]) * up.n[:, k], axis=0)
        c = np.where(dist <= drops.h[j], 2, np.where(dist <= drops.A_TILDE * drops.h[j], 1, 0))
        codes[s:s + 256] = np.where(side <= 0.0, INSIDE, c)
    return codes


def raw_layer_at(drops, pts: np.ndarray, dens_list, kind: str, j: int, codes=None) -> np.ndarray:
    """Raw integral over drop j at fluid points [3][n]: int K rho ds with K = G (kind "S") or the
    contracted stresslet u.T.n (kind "D"), [3][n]."""
    _ensure_upsampled(drops)
    codes = classify_points(drops, pts, j) if codes is None else codes
    if np.any(codes == INSIDE):
        raise ValueError(f"a point lies inside drop {j}")
    out = np.zeros((3, pts.shape[1]))
    dens = np.asarray(dens_list[j])
    for r, grid in ((0, drops.std[j]), (1, drops.ups[j])):
        sel = np.nonzero(codes == r)[0]
        if len(sel):
            out[:, sel] = regular_sum(pts[:, sel], grid, grid.density(dens), kind)
    sel = np.nonzero(codes == 2)[0]
    if len(sel):
        self_raw = drops.selfq[j].apply(dens, kind)
        data = near.near_data(drops, j, dens, self_raw.reshape(3, drops.p[j] + 1, 2 * drops.p[j] + 2))
        for col in sel:
            out[:, col] = near.near_value_at(drops, j, pts[:, col], data, kind)
    return out


def layer_at(drops, pts: np.ndarray, dens_list, kind: str, raw: bool = False) -> np.ndarray:
    """S[f](x0) (kind "S") or D[u](x0) (kind "D") at fluid points [3][n], with the weights of
    Drops.apply_single / apply_double (raw: 1/8pi for S and 1/4pi for D, every drop)."""
    out = np.zeros((3, pts.shape[1]))
    for j in range(drops.N):
        if kind == "S":
            w = 1.0 / (8.0 * np.pi) if raw else -1.0 / (4.0 * np.pi)
        else:
            w = 1.0 / (4.0 * np.pi) if raw else (drops.lam[j] - 1.0) / (4.0 * np.pi)
        if w != 0.0:
            out += w * raw_layer_at(drops, pts, dens_list, kind, j)
    return out


def velocity_at(drops, pts: np.ndarray, f_list, u_list, shear: float) -> np.ndarray:
    """u(x0) = u_inf(x0) + (S[f](x0) + D[u](x0)) / 2 at fluid points [3][n], u_inf = (shear z, 0, 0)."""
    u = 0.5 * (layer_at(drops, pts, f_list, "S") + layer_at(drops, pts, u_list, "D"))
    u[0] += shear * pts[2]
    return u
