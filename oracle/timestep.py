"""Midpoint time step of the drop shapes (oracle; test infrastructure only).

Sec. 3: the drop surfaces move with the interface velocity u, which solves Eq. main_eq for the
current shapes; the paper advances the shapes with a second-order Runge-Kutta (midpoint) rule
(Alg. 1).  Here the surfactant concentration is held fixed over the step (the transport equation
of Sec. 3 is not part of this step), so one step is

    x^{1/2} = x + (dt/2) u(x),    x^{new} = x + dt u(x^{1/2}),

with u(x) the solution of (lambda_i + 1) u_i - D[u]_i = 2 u_inf + S[f]_i for the shapes x, the far
field u_inf = (shear z, 0, 0) and the interfacial force f of the fixed surfactant (Sec. 1).  Every
piece is the oracle's own: the force (geometry.interfacial_force), the operators and right-hand side
(layer.Drops) and GMRES (gmres.gmres).
"""
from __future__ import annotations

import numpy as np

from . import geometry, gmres, layer


def velocity(xs, ps, pqs, lam, gammas, elasticity: float, xs_param: float, shear: float, up: int = 4,
             tol: float = 1e-13):
    """Interface velocity coefficients [drop][3][(p+1)^2] of Eq. main_eq for the shapes xs."""
    drops = layer.Drops(xs, ps, pqs, lam, up=up)
    f = [geometry.interfacial_force(x, p, g, elasticity, xs_param) for x, p, g in zip(drops.xcoef, ps, gammas)]
    b = drops.rhs(f, shear)
    u, info = gmres.gmres(drops.system_matvec, b, tol=tol)
    assert info["converged"]
    return drops.split(u)


def midpoint_step(xs, ps, pqs, lam, gammas, elasticity: float, xs_param: float, shear: float, dt: float,
                  up: int = 4, tol: float = 1e-13):
    """Shapes after one midpoint step of length dt (surfactant fixed)."""
    xs = [np.asarray(x, dtype=np.float64).reshape(3, -1) for x in xs]
    u0 = velocity(xs, ps, pqs, lam, gammas, elasticity, xs_param, shear, up, tol)
    xh = [x + 0.5 * dt * u for x, u in zip(xs, u0)]
    u1 = velocity(xh, ps, pqs, lam, gammas, elasticity, xs_param, shear, up, tol)
    return [x + dt * u for x, u in zip(xs, u1)]
