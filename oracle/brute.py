"""Brute-force references for the singular self-integral and for integrals at points just off the
surface (oracle; test infrastructure only).

Independent of the rotation machinery and of the singular weights of Thm 1: the integral
int K(x0 - x) rho dS over the whole surface is written in polar coordinates (theta', phi') of the
parameter sphere centred at the target, where dS = J(v) sin(theta') dtheta' dphi', J = W/sin(theta)
at the parameter point v = R s(theta', phi').  In these coordinates the weakly singular integrand is
smooth, so a Gauss-Legendre rule in theta' on [0, pi] times the trapezoid rule in phi' converges
spectrally; both are doubled until two successive values agree.  For a target just off the surface
the polar rule is centred at the nearest surface point, where the nearly singular peak sits.  The
geometry is evaluated directly from the SH series (Sec. 1.1) at the points v.
"""
from __future__ import annotations

import numpy as np

from . import sh, wigner
from .layer import stokeslet, stresslet


def _integral(xcoef, p, dens, theta_a, phi_b, kind, nt, nf, x0=None):
    t, w = np.polynomial.legendre.leggauss(nt)
    thp = 0.5 * np.pi * (t + 1.0)
    wt = 0.5 * np.pi * w
    php = 2.0 * np.pi * np.arange(nf) / nf
    T, Ph = np.meshgrid(thp, php, indexing="ij")
    s = np.stack([np.sin(T) * np.cos(Ph), np.sin(T) * np.sin(Ph), np.cos(T)])
    v = np.einsum("ab,bjk->ajk", wigner.rotation_matrix(phi_b, theta_a, 0.0), s)
    th = np.arccos(np.clip(v[2], -1.0, 1.0))
    ph = np.arctan2(v[1], v[0])
    d = [sh.evaluate_derivs(xcoef[c], p, th, ph) for c in range(3)]
    x = np.stack([d[c]["f"] for c in range(3)])
    cr = np.cross(np.stack([d[c]["t"] for c in range(3)]), np.stack([d[c]["p"] for c in range(3)]), axis=0)
    W = np.sqrt(np.sum(cr * cr, axis=0))
    n = cr / W
    J = W / np.sin(th)
    rho = np.stack([sh.evaluate(dens[c], p, th, ph) for c in range(3)])
    if x0 is None:  # the target is the surface point at the pole of the polar rule
        x0 = np.array([sh.evaluate(xcoef[c], p, np.array([theta_a]), np.array([phi_b]))[0] for c in range(3)])
    xh = x0[:, None, None] - x
    K = stokeslet(xh, rho) if kind == "S" else stresslet(xh, rho, n)
    wgt = (wt * np.sin(thp))[:, None] * (2.0 * np.pi / nf) * J
    return np.sum(K * wgt[None], axis=(1, 2))


def self_integral(xcoef, p, dens, theta_a, phi_b, kind, tol=1e-13, n0=32, nmax=512):
    """int_gamma K(x0 - x) rho(x) dS at the parameter point (theta_a, phi_b), converged in the rule size."""
    xcoef = np.asarray(xcoef).reshape(3, -1)
    dens = np.asarray(dens).reshape(3, -1)
    nt, prev = n0, None
    while nt <= nmax:
        val = _integral(xcoef, p, dens, theta_a, phi_b, kind, nt, 2 * nt)
        if prev is not None and np.max(np.abs(val - prev)) <= tol * max(1.0, np.max(np.abs(val))):
            return val
        prev = val
        nt *= 2
    raise RuntimeError("brute-force quadrature did not converge")


def _closest_parameters(xcoef, p, x0, iters=60):
    """Parameters of the surface point nearest x0: the nearest point of a fine sample (degree 4p+3
    grid), refined by Gauss-Newton on x(theta, phi) - x0 with the analytic first derivatives."""
    P = 4 * p + 3
    _, _, th, ph = sh.gauss_grid(P)
    T, F = np.meshgrid(th, ph, indexing="ij")
    X = np.stack([sh.evaluate(xcoef[c], p, T, F) for c in range(3)])
    k = int(np.argmin(np.sum((X - x0[:, None, None]) ** 2, axis=0)))
    t, f = T.ravel()[k], F.ravel()[k]
    for _ in range(iters):
        d = [sh.evaluate_derivs(xcoef[c], p, np.array([t]), np.array([f])) for c in range(3)]
        r = np.array([d[c]["f"][0] for c in range(3)]) - x0
        J = np.array([[d[c]["t"][0], d[c]["p"][0]] for c in range(3)])
        step = np.linalg.lstsq(J, -r, rcond=None)[0]
        t, f = t + step[0], f + step[1]
        if np.max(np.abs(step)) < 1e-15:
            break
    return t, f


def exterior_integral(xcoef, p, dens, x0, kind, tol=1e-12, n0=32, nmax=2048):
    """int_gamma K(x0 - x) rho(x) dS at a point x0 off the surface, with the polar rule centred at
    the surface point nearest x0 (the nearly singular peak sits at the pole), doubled until two
    successive values agree."""
    xcoef = np.asarray(xcoef).reshape(3, -1)
    dens = np.asarray(dens).reshape(3, -1)
    x0 = np.asarray(x0, dtype=np.float64)
    t, f = _closest_parameters(xcoef, p, x0)
    nt, prev = n0, None
    while nt <= nmax:
        val = _integral(xcoef, p, dens, t, f, kind, nt, 2 * nt, x0=x0)
        if prev is not None and np.max(np.abs(val - prev)) <= tol * max(1.0, np.max(np.abs(val))):
            return val
        prev = val
        nt *= 2
    raise RuntimeError("brute-force quadrature did not converge")

