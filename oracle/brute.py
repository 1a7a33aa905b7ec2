"""Brute-force reference for the singular self-integral (oracle; test infrastructure only).

Independent of the rotation machinery and of the singular weights of Thm 1: the integral
int K(x0 - x) rho dS over the whole surface is written in polar coordinates (theta', phi') of the
parameter sphere centred at the target, where dS = J(v) sin(theta') dtheta' dphi', J = W/sin(theta)
at the parameter point v = R s(theta', phi').  In these coordinates the weakly singular integrand is
smooth, so a Gauss-Legendre rule in theta' on [0, pi] times the trapezoid rule in phi' converges
spectrally; both are doubled until two successive values agree.  The geometry is evaluated
directly from the SH series (Sec. 1.1) at the points v.
"""
from __future__ import annotations

import numpy as np

from . import sh, wigner
from .layer import stokeslet, stresslet


def _integral(xcoef, p, dens, theta_a, phi_b, kind, nt, nf):
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
