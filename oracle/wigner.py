"""Wigner rotation of SH coefficients (oracle; test infrastructure only).  App. B.

The oracle evaluates the small-d matrix d^n(beta) = <n m'| exp(-i beta J_y) |n m> by the matrix
exponential of the real antisymmetric generator -i J_y = (J_- - J_+)/2 in the |n, m> basis,
m = -n..n (a library matrix exponential is the step).  App. B's factorial sum gives the same
matrix; it cancels catastrophically for large n, so it is used only as a pin (in extended
precision) for small n.

Rotation semantics.  For R = R_z(alpha) R_y(beta) R_z(gamma) (z-y-z Euler angles, active
rotations of R^3) the rotated expansion g(s) = f(R s) has coefficients
    g_n^{m'} = e^{i m' gamma} sum_m dd^n_{m' m}(beta) e^{i m alpha} f_n^m,
with dd^n(beta) = d^n(-beta) = d^n(beta)^T, because Y_n^m(R_y(beta) v) = sum_{m'} d^n_{m m'}(beta) Y_n^{m'}(v)
for Condon-Shortley-phased harmonics.  (App. B prints the phases with a single index m and
sums over m'; the standard form above is the reading taken.)  The pole of g sits at the
point R z = s(beta, alpha) of the original parametrisation, which is what Sec. 2.2 needs.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np
import scipy.linalg

from . import sh


@lru_cache(maxsize=None)
def _generator(n: int) -> np.ndarray:
    dim = 2 * n + 1
    Jp = np.zeros((dim, dim))
    Jm = np.zeros((dim, dim))
    for i, m in enumerate(range(-n, n + 1)):
        if m < n:
            Jp[i + 1, i] = math.sqrt((n - m) * (n + m + 1.0))
        if m > -n:
            Jm[i - 1, i] = math.sqrt((n + m) * (n - m + 1.0))
    return 0.5 * (Jm - Jp)


def small_d(n: int, beta: float) -> np.ndarray:
    """d^n_{m' m}(beta), rows m' = -n..n, columns m = -n..n."""
    return scipy.linalg.expm(beta * _generator(n))


def small_d_factorial(n: int, mp: int, m: int, beta, mpmath_mod=None):
    """App. B factorial sum for d^n_{m' m}(beta), evaluated with mpmath at 50 digits (pin only)."""
    import mpmath as mpm
    mpm.mp.dps = 50
    b = mpm.mpf(beta)
    c = mpm.cos(b / 2)
    s = mpm.sin(b / 2)
    f = mpm.factorial
    pref = (-1) ** (mp - m) * mpm.sqrt(f(n + mp) * f(n - mp) * f(n + m) * f(n - m))
    tot = mpm.mpf(0)
    for k in range(max(0, m - mp), min(n + m, n - mp) + 1):
        tot += (-1) ** k * c ** (2 * (n - k) + m - mp) * s ** (2 * k - m + mp) / (
            f(n + m - k) * f(k) * f(mp - m + k) * f(n - mp - k))
    return pref * tot


def rotate(coef: np.ndarray, p: int, alpha: float, beta: float, gamma: float = 0.0) -> np.ndarray:
    """Real-packed coefficients of g(s) = f(R_z(alpha) R_y(beta) R_z(gamma) s)."""
    c = sh.to_complex(coef, p)
    out = np.zeros_like(c)
    for n in range(p + 1):
        full = np.zeros(2 * n + 1, dtype=np.complex128)
        for m in range(0, n + 1):
            full[n + m] = c[n, m] * np.exp(1j * m * alpha)
            if m > 0:
                full[n - m] = (-1) ** m * np.conj(c[n, m]) * np.exp(-1j * m * alpha)
        dd = small_d(n, beta).T
        g = dd @ full
        for mp in range(0, n + 1):
            out[n, mp] = g[n + mp] * np.exp(1j * mp * gamma)
    return sh.from_complex(out, p)


def rotation_matrix(alpha: float, beta: float, gamma: float = 0.0) -> np.ndarray:
    """R_z(alpha) R_y(beta) R_z(gamma) as a 3x3 matrix acting on column vectors."""
    def rz(a):
        return np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])

    def ry(b):
        return np.array([[math.cos(b), 0.0, math.sin(b)], [0.0, 1.0, 0.0], [-math.sin(b), 0.0, math.cos(b)]])

    return rz(alpha) @ ry(beta) @ rz(gamma)
