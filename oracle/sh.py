"""Spherical-harmonic grid, basis and transforms (oracle; test infrastructure only).

Follows Sec. 1.1 (basis, truncated expansion), Sec. 2.1 (Gauss grid, regular quadrature,
discrete forward transform) and App. A (normalised Legendre recursion, derivatives).

Readings of the text:
  * the phi grid has 2p+2 points phi_k = pi k/(p+1) (Sec. 2.1);
  * the weight factor printed as pi/p in Sec. 2.1 is the phi spacing pi/(p+1) of that grid
    (with pi/p the discrete orthogonality of Sec. 2.1 fails);
  * App. A's first theta-derivative formula is used with its "cot phi" read as cot(theta);
    its second-derivative formula is garbled, so the associated Legendre equation written in
    theta is used instead.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np


def ncoef(p: int) -> int:
    return (p + 1) ** 2


@lru_cache(maxsize=None)
def gauss_legendre(n: int):
    """n Gauss-Legendre nodes (ascending) and weights, polished by Newton's method in 40-digit
    arithmetic (library double-precision nodes lose a few digits in the end weights for n > 100)."""
    import mpmath as mpm
    t0, _ = np.polynomial.legendre.leggauss(n)
    t = np.zeros(n)
    w = np.zeros(n)
    with mpm.workdps(40):
        for i, x0 in enumerate(t0):
            x = mpm.mpf(float(x0))
            for _ in range(4):
                pn, pm = mpm.legendre(n, x), mpm.legendre(n - 1, x)
                x -= pn / (n * (x * pn - pm) / (x * x - 1))
            pn, pm = mpm.legendre(n, x), mpm.legendre(n - 1, x)
            dp = n * (x * pn - pm) / (x * x - 1)
            t[i] = float(x)
            w[i] = float(2 / ((1 - x * x) * dp * dp))
    t.setflags(write=False)
    w.setflags(write=False)
    return t, w


def gauss_grid(p: int):
    """Sec. 2.1: t_j = GL nodes (ascending) with weights, theta_j = arccos t_j, phi_k = pi k/(p+1)."""
    t, w = gauss_legendre(p + 1)
    theta = np.arccos(t)
    phi = np.pi * np.arange(2 * p + 2) / (p + 1)
    return t, w, theta, phi


def legendre_normalised(p: int, x: np.ndarray) -> np.ndarray:
    """App. A recursion for P~_n^m(x), 0 <= m <= n <= p, Condon-Shortley phase included.

    Returns array [n][m][len(x)] (entries with m > n are zero).
    """
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P = np.zeros((p + 1, p + 1) + x.shape)
    P[0, 0] = math.sqrt(1.0 / (4.0 * math.pi))
    for m in range(1, p + 1):
        c = math.sqrt(1.0 + 1.0 / (2.0 * m))
        P[m, m] = -c * s * P[m - 1, m - 1]
    for m in range(0, p):
        P[m + 1, m] = math.sqrt(2.0 * m + 3.0) * x * P[m, m]
    for m in range(0, p + 1):
        for n in range(m + 2, p + 1):
            a = math.sqrt((4.0 * n * n - 1.0) / (n * n - m * m))
            b = -math.sqrt(((n - 1.0) ** 2 - m * m) / (4.0 * (n - 1.0) ** 2 - 1.0))
            P[n, m] = a * (x * P[n - 1, m] + b * P[n - 2, m])
    return P


def legendre_dtheta(p: int, theta: np.ndarray):
    """App. A: d/dtheta P~_n^m(cos theta) = alpha_n^m P~_n^{m+1} + m cot(theta) P~_n^m.

    Second derivative from the associated Legendre equation in theta:
      P'' = -cot(theta) P' + (m^2/sin^2(theta) - n(n+1)) P.
    Returns (P, dP, d2P), each [n][m][len(theta)].  theta must avoid the poles.
    """
    theta = np.asarray(theta, dtype=np.float64)
    P = legendre_normalised(p + 1, np.cos(theta))
    cot = np.cos(theta) / np.sin(theta)
    s2 = np.sin(theta) ** 2
    dP = np.zeros((p + 1, p + 1) + theta.shape)
    d2P = np.zeros_like(dP)
    for n in range(p + 1):
        for m in range(n + 1):
            alpha = math.sqrt((n - m) * (n + m + 1.0))
            up = P[n, m + 1] if m + 1 <= n else 0.0
            dP[n, m] = alpha * up + m * cot * P[n, m]
            d2P[n, m] = -cot * dP[n, m] + (m * m / s2 - n * (n + 1.0)) * P[n, m]
    return P[: p + 1, : p + 1], dP, d2P


def to_complex(coef: np.ndarray, p: int) -> np.ndarray:
    """Real-packed (index n(n+1)+m: Re for m>=0, Im of m=|m| for m<0) -> complex f_n^m, m >= 0, [n][m]."""
    c = np.zeros((p + 1, p + 1), dtype=np.complex128)
    for n in range(p + 1):
        c[n, 0] = coef[n * (n + 1)]
        for m in range(1, n + 1):
            c[n, m] = coef[n * (n + 1) + m] + 1j * coef[n * (n + 1) - m]
    return c


def from_complex(c: np.ndarray, p: int) -> np.ndarray:
    out = np.zeros(ncoef(p))
    for n in range(p + 1):
        out[n * (n + 1)] = c[n, 0].real
        for m in range(1, n + 1):
            out[n * (n + 1) + m] = c[n, m].real
            out[n * (n + 1) - m] = c[n, m].imag
    return out


def analyze(grid: np.ndarray, p_grid: int, p_out: int) -> np.ndarray:
    """Eq. back_transf_discr: f_n^m = pi/(p+1) sum_j sum_k w_j^G f(theta_j,phi_k) conj(Y_n^m), n <= p_out.

    grid: [p_grid+1][2 p_grid+2] values; returns real-packed coefficients of degree p_out.
    """
    t, w, theta, phi = gauss_grid(p_grid)
    P = legendre_normalised(p_out, t)
    c = np.zeros((p_out + 1, p_out + 1), dtype=np.complex128)
    for m in range(p_out + 1):
        e = np.exp(-1j * m * phi)
        Fm = grid @ e  # [j]
        for n in range(m, p_out + 1):
            c[n, m] = (np.pi / (p_grid + 1)) * np.sum(w * P[n, m] * Fm)
    return from_complex(c, p_out)


def _synth_from_tables(c, p, Pt, phi, dphi_order=0):
    """Sum_{n,m} f_n^m (im)^k T_n^m(theta_j) e^{im phi}, real part, using m >= 0 and the real symmetry."""
    nth = Pt.shape[2]
    out = np.zeros((nth, len(phi)))
    for m in range(p + 1):
        h = np.zeros(nth, dtype=np.complex128)
        for n in range(m, p + 1):
            h += c[n, m] * Pt[n, m]
        if dphi_order:
            h = h * (1j * m) ** dphi_order
        e = np.exp(1j * m * phi)
        term = np.outer(h, e)
        out += term.real if m == 0 else 2.0 * term.real
    return out


def synthesize(coef: np.ndarray, p: int, p_grid: int) -> np.ndarray:
    """Eq. spharm_ex evaluated on the degree-p_grid Gauss grid (zero padding when p_grid > p)."""
    t, w, theta, phi = gauss_grid(p_grid)
    P = legendre_normalised(p, t)
    return _synth_from_tables(to_complex(coef, p), p, P, phi)


def synthesize_derivs(coef: np.ndarray, p: int, p_grid: int) -> dict:
    """Values and the derivatives f_t, f_p, f_tt, f_tp, f_pp on the degree-p_grid grid (App. A)."""
    t, w, theta, phi = gauss_grid(p_grid)
    P, dP, d2P = legendre_dtheta(p, theta)
    c = to_complex(coef, p)
    return {
        "f": _synth_from_tables(c, p, P, phi),
        "t": _synth_from_tables(c, p, dP, phi),
        "p": _synth_from_tables(c, p, P, phi, 1),
        "tt": _synth_from_tables(c, p, d2P, phi),
        "tp": _synth_from_tables(c, p, dP, phi, 1),
        "pp": _synth_from_tables(c, p, P, phi, 2),
    }


def evaluate(coef: np.ndarray, p: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Eq. spharm_ex at arbitrary parameter points (theta, phi) of equal shape (direct double sum)."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    P = legendre_normalised(p, np.cos(theta))
    c = to_complex(coef, p)
    out = np.zeros(theta.shape)
    for m in range(p + 1):
        h = np.zeros(theta.shape, dtype=np.complex128)
        for n in range(m, p + 1):
            h += c[n, m] * P[n, m]
        v = (h * np.exp(1j * m * phi)).real
        out += v if m == 0 else 2.0 * v
    return out


def evaluate_derivs(coef: np.ndarray, p: int, theta: np.ndarray, phi: np.ndarray) -> dict:
    """Value and first/second parameter derivatives at arbitrary points (theta off the poles)."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    P, dP, d2P = legendre_dtheta(p, theta)
    c = to_complex(coef, p)
    res = {k: np.zeros(theta.shape) for k in ("f", "t", "p", "tt", "tp", "pp")}
    for m in range(p + 1):
        h = np.zeros(theta.shape, dtype=np.complex128)
        ht = np.zeros_like(h)
        htt = np.zeros_like(h)
        for n in range(m, p + 1):
            h += c[n, m] * P[n, m]
            ht += c[n, m] * dP[n, m]
            htt += c[n, m] * d2P[n, m]
        e = np.exp(1j * m * phi)
        fac = 1.0 if m == 0 else 2.0
        res["f"] += fac * (h * e).real
        res["t"] += fac * (ht * e).real
        res["tt"] += fac * (htt * e).real
        res["p"] += fac * (1j * m * h * e).real
        res["tp"] += fac * (1j * m * ht * e).real
        res["pp"] += fac * (-(m * m) * h * e).real
    return res
