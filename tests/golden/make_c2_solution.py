"""Write the oracle's FP64 solution of the single-drop shear system at full size (test infrastructure).

Workload: one drop of degree p = 32 (sphere plus a seeded SH perturbation of amplitude 0.05, degrees
1..6), viscosity ratio 5, shear u_inf = (z, 0, 0), self quadrature on the grid of degree p_q = 65,
and the seeded band-limited test density as the interfacial force f.  The script calls only the
oracle (and the seeded input generators): the right-hand side b = 2 u_inf + S[f] of Eq. main_eq,
projected (Sec. 1.2), and its GMRES solution (Sec. 6) of (lambda + 1) u - D[u] = b to a relative
residual of 1e-13.  Output: tests/golden/c2_solution.npz with b, u and the residual history.

    python tests/golden/make_c2_solution.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import gmres, layer  # noqa: E402
from paper_1707_02156_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "c2_solution.npz")


def main() -> None:
    w = inputs.perturbed_drop()
    p, pq = w.p[0], w.pq[0]
    t0 = time.time()
    drops = layer.Drops([w.xcoef.reshape(3, -1)], [p], [pq], w.lam)
    b = drops.rhs([w.density], w.shear)
    print(f"rhs done in {time.time() - t0:.0f} s", flush=True)
    n_mv = [0]

    def matvec(u):
        n_mv[0] += 1
        t = time.time()
        y = drops.system_matvec(u)
        print(f"  matvec {n_mv[0]}: {time.time() - t:.0f} s", flush=True)
        return y

    u, info = gmres.gmres(matvec, b, tol=1e-13, restart=30, max_it=120)
    assert info["converged"], info
    np.savez(OUT, b=b, u=u, residuals=np.asarray(info["residuals"]), p=p, pq=pq, lam=w.lam,
             shear=w.shear)
    print(f"wrote {OUT}: {info['iterations']} iterations, final residual {info['residuals'][-1]:.2e}, "
          f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
