"""Restarted GMRES with modified Gram-Schmidt (oracle; test infrastructure only).

Sec. 6: the second-kind system of Eq. main_eq is solved iteratively with GMRES.  Textbook
algorithm (Saad & Schultz): Arnoldi with modified Gram-Schmidt, Givens rotations on the
Hessenberg matrix, restart after m steps, stop on the relative residual ||b - A x|| / ||b||.
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, b: np.ndarray, x0: np.ndarray | None = None, tol: float = 1e-12, restart: int = 30,
          max_it: int = 300):
    """Solve A x = b.  Returns (x, info) with info = {'converged', 'iterations', 'residuals'}."""
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), {"converged": True, "iterations": 0, "residuals": [0.0]}
    hist = []
    it = 0
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm <= tol or it >= max_it:
            return x, {"converged": beta / bnorm <= tol, "iterations": it, "residuals": hist}
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(restart):
            w = matvec(V[k])
            for i in range(k + 1):
                H[i, k] = w @ V[i]
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0.0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            k_used = k + 1
            hist.append(abs(g[k + 1]) / bnorm)
            if abs(g[k + 1]) / bnorm <= tol or it >= max_it:
                break
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])
        x = x + V[:k_used].T @ y
