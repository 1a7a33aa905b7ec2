"""Angle reparametrisation of a drop surface and its surfactant (oracle; test infrastructure only).

Sec. 4.  The spectral energy E(x) = sum_{n,m} a_nm |x_n^m|^2 (Eq. energy_rep) with the adaptive
cutoff of Eq. ncutoff_adaptive; the pseudo-velocity w = -(I - n n) grad E (Eq. pseudo_rep); the
velocity of the angles alpha = A^-1 b from the two tangential projections of the chain rule
(Eqs. system_rep, system_rep_sol); a forward Euler step of the angles; the original expansions
evaluated at the new angles and analysed on the grid (Eqs. rep_trasf1, rep_trasf2); Alg. 2 with
its stopping test on ||g||.

Readings of the text:
  * Working grid.  The surface and the surfactant are first zero-padded to degree
    P = U_rep (p+1) - 1; the energy, the cutoff and the iteration use that degree; the result is
    analysed back to degree p.
  * grad E is the L2(S^2) gradient of E as a function of x(theta, phi): grad E = 2 sum a_nm x_n^m
    Y_n^m, synthesised on the grid.  g = (I - n n) grad E with n the outward normal of the original
    surface at the current point; ||g|| is the largest Euclidean norm of g over the grid points.
  * |x_n^m| of the position vector is the Euclidean norm of its three complex coefficients, and the
    sums of Eq. energy_rep and of N_2(l) in Eq. ncutoff_adaptive run over m = -n..n (the negative
    orders from the real symmetry, |x_n^-m| = |x_n^m|).  n_cutoff = the smallest l with
    1 < l <= P and N_2(l)/N_1 < P_cutoff (P if there is none).
  * Filters: the perfect low-pass filter a_nm = 1 for n >= n_cutoff, else 0, or the smooth filter
    a_nm = n/P for n >= n_cutoff, else 0.
  * The angles of every grid point start at the grid's (theta_j, phi_k) and follow
    theta* += dtau alpha_theta, phi* += dtau alpha_phi, with A and b built from the original
    expansion's derivatives at (theta*, phi*).  An angle pair that steps across a pole is mapped
    back to theta in (0, pi) with phi shifted by pi (the same point of the sphere).
  * With this gradient the filtered modes decay at rate 2 a_n in pseudo-time, so the forward Euler
    step is stable for dtau < 1/max(a_n) (the perfect filter: dtau < 1; dtau = 1/2 removes them in
    one step in the linear setting).
"""
from __future__ import annotations

import numpy as np

from . import sh


def upsample(coef: np.ndarray, p: int, P: int) -> np.ndarray:
    """Zero-padding of real-packed coefficients [..., (p+1)^2] to degree P."""
    coef = np.asarray(coef, dtype=np.float64)
    out = np.zeros(coef.shape[:-1] + ((P + 1) ** 2,))
    out[..., : (p + 1) ** 2] = coef
    return out


def mode_norms(xcoef: np.ndarray, P: int) -> np.ndarray:
    """|x_n^m| for n <= P and m = -n..n: the norm of the three complex coefficients, [n][m+P]."""
    c = np.stack([sh.to_complex(xcoef[i], P) for i in range(3)])  # [3][n][m >= 0]
    a = np.sqrt(np.sum(np.abs(c) ** 2, axis=0))  # [n][m >= 0]
    out = np.zeros((P + 1, 2 * P + 1))
    for n in range(P + 1):
        out[n, P: P + n + 1] = a[n, : n + 1]
        out[n, P - n: P] = a[n, 1: n + 1][::-1]
    return out


def adaptive_cutoff(xcoef: np.ndarray, P: int, p_cutoff: float) -> int:
    """Eq. ncutoff_adaptive: min{l : 1 < l <= P, N_2(l) / N_1 < p_cutoff}, N_2(l) = sum_{n >= l} sum_m |x_n^m|."""
    per_n = np.sum(mode_norms(xcoef, P), axis=1)
    n1 = np.sum(per_n[1:])
    for l in range(2, P + 1):
        if np.sum(per_n[l:]) / n1 < p_cutoff:
            return l
    return P


def attenuation(P: int, ncut: int, smooth: bool) -> np.ndarray:
    """a_n for n = 0..P (the filters depend on n only)."""
    n = np.arange(P + 1, dtype=np.float64)
    a = np.where(n >= ncut, n / P if smooth else 1.0, 0.0)
    return a


def energy(xcoef: np.ndarray, P: int, a: np.ndarray) -> float:
    """Eq. energy_rep: sum_n a_n sum_{m=-n..n} |x_n^m|^2."""
    return float(np.sum(a[:, None] * mode_norms(xcoef, P) ** 2))


def _scale_degrees(coef: np.ndarray, P: int, a: np.ndarray) -> np.ndarray:
    deg = np.concatenate([np.full(2 * n + 1, n) for n in range(P + 1)])
    return coef * a[deg]


def _eval_fields(xcoef, P, th, ph):
    d = [sh.evaluate_derivs(xcoef[c], P, th, ph) for c in range(3)]
    return {k: np.stack([d[c][k] for c in range(3)]) for k in ("f", "t", "p")}


def _wrap(th, ph):
    """Map angle pairs back to theta in (0, pi) (a step across a pole shifts phi by pi)."""
    th = np.mod(th, 2 * np.pi)
    over = th > np.pi
    th = np.where(over, 2 * np.pi - th, th)
    ph = np.where(over, ph + np.pi, ph)
    return th, ph


def tangent_fields(x0: np.ndarray, P: int, th, ph):
    """x, x_theta, x_phi and the outward unit normal of the expansion x0 at the parameters (th, ph)."""
    e = _eval_fields(x0, P, th, ph)
    nrm = np.cross(e["t"], e["p"], axis=0)
    e["n"] = nrm / np.linalg.norm(nrm, axis=0)
    return e


def angle_velocity(e: dict, w: np.ndarray):
    """Eq. system_rep_sol: (dtheta/dtau, dphi/dtau) = A^-1 b with A the metric of x(theta, phi) and
    b = (w . x_theta, w . x_phi), at every point (e from tangent_fields, w [3][...])."""
    A11 = np.sum(e["t"] * e["t"], axis=0)
    A12 = np.sum(e["t"] * e["p"], axis=0)
    A22 = np.sum(e["p"] * e["p"], axis=0)
    b1 = np.sum(w * e["t"], axis=0)
    b2 = np.sum(w * e["p"], axis=0)
    det = A11 * A22 - A12 * A12
    return (A22 * b1 - A12 * b2) / det, (-A12 * b1 + A11 * b2) / det


def reparametrize(xcoef, gcoef, p: int, u_rep: int = 2, p_cutoff: float = 0.05, smooth: bool = False,
                  dtau: float = 0.5, eps: float = 1e-10, i_max: int = 200):
    """Alg. 2.  Returns (x~ [3][(p+1)^2], Gamma~ [(p+1)^2], history) after the angle iteration.

    history: per iteration the energy E (with the cutoff of that iteration), n_cutoff and ||g||.
    """
    P = u_rep * (p + 1) - 1
    x0 = upsample(np.asarray(xcoef).reshape(3, -1), p, P)
    g0 = upsample(np.asarray(gcoef).reshape(-1), p, P)
    _, _, theta, phi = sh.gauss_grid(P)
    T, F = np.meshgrid(theta, phi, indexing="ij")
    th, ph = T.copy(), F.copy()
    xt = x0.copy()  # coefficients of the current surface x~
    hist = []
    for _ in range(i_max):
        ncut = adaptive_cutoff(xt, P, p_cutoff)
        a = attenuation(P, ncut, smooth)
        # grad E = 2 sum a_n x~_n^m Y_n^m on the grid, projected on the tangent plane of the surface
        gradE = np.stack([2.0 * sh.synthesize(_scale_degrees(xt[c], P, a), P, P) for c in range(3)])
        e = tangent_fields(x0, P, th, ph)
        gvec = gradE - np.sum(gradE * e["n"], axis=0) * e["n"]
        gnorm = float(np.max(np.linalg.norm(gvec, axis=0)))
        hist.append({"energy": energy(xt, P, a), "n_cutoff": ncut, "g": gnorm})
        if gnorm < eps:
            break
        # the angles follow the pseudo-velocity w = -g on the original surface
        al_t, al_p = angle_velocity(e, -gvec)
        th, ph = _wrap(th + dtau * al_t, ph + dtau * al_p)
        # Eq. rep_trasf1: the original expansion at the new angles, analysed on the grid
        xg = np.stack([sh.evaluate(x0[c], P, th, ph) for c in range(3)])
        xt = np.stack([sh.analyze(xg[c], P, P) for c in range(3)])
    # Eq. rep_trasf2: the surfactant at the final angles; both results back to degree p
    gg = sh.evaluate(g0, P, th, ph)
    xg = np.stack([sh.evaluate(x0[c], P, th, ph) for c in range(3)])
    x_out = np.stack([sh.analyze(xg[c], P, p) for c in range(3)])
    g_out = sh.analyze(gg, P, p)
    return x_out, g_out, {"history": hist, "theta": th, "phi": ph, "P": P}
