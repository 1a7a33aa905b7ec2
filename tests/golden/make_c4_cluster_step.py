"""Write the oracle's coupled step (Alg. 1) of a four-drop cluster cut out of the 64-drop batch
(test infrastructure).

The cluster is drop 23 of the 64-drop workload (degree 48, lambda 4.04) and its three nearest
neighbours (drops 63, 29 and 32: degrees 24, 16 and 48, surface gaps 0.63, 0.83 and 1.08), at their
positions in the batch, with its upsampling factor U = 2, clean interfaces (sigma = 1: the batch's
elasticity is 0), the constant surfactant Gamma = 1 of the batch, shear u_inf = (z, 0, 0), dt = 0.01
and Pe = 10.  The step is the oracle's own (oracle.surfactant.coupled_step with the Stokes velocity
of oracle.timestep.velocity, FP64 GMRES to 1e-13).  Output: tests/golden/c4_cluster_step.npz with the
drop ids, the velocities at t and t + dt/2, Gamma at t + dt/2, and x and Gamma at t + dt, and the
surfactant mass of each drop at t and t + dt (regular rule on the grid of degree 2p+1).

    python tests/golden/make_c4_cluster_step.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import surfactant as sf, timestep  # noqa: E402
from paper_1707_02156_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "c4_cluster_step.npz")
IDS = [23, 63, 29, 32]
DT, PE, SHEAR = 0.01, 10.0, 1.0


def cluster():
    """Shapes, surfactant, degrees and viscosity ratios of the cluster's drops, in IDS order."""
    w = inputs.config("c4")
    offs, o = [], 0
    for p in w.p:
        offs.append(o)
        o += 3 * (p + 1) ** 2
    xs, gs, ps, lam = [], [], [], []
    go = np.cumsum([0] + [(p + 1) ** 2 for p in w.p])
    for i in IDS:
        p = w.p[i]
        xs.append(w.xcoef[offs[i]:offs[i] + 3 * (p + 1) ** 2].reshape(3, -1))
        gs.append(w.gamma[go[i]:go[i + 1]].copy())
        ps.append(p)
        lam.append(w.lam[i])
    return w, xs, gs, ps, np.array(lam)


def main() -> None:
    w, xs, gs, ps, lam = cluster()
    t0 = time.time()
    n = [0]

    def velocity(x_list, g_list):
        n[0] += 1
        t = time.time()
        u = timestep.velocity(x_list, ps, ps, lam, g_list, w.elasticity, 0.0, SHEAR, up=w.up, tol=1e-13)
        print(f"velocity solve {n[0]}: {time.time() - t:.0f} s", flush=True)
        return u

    r = sf.coupled_step(xs, gs, ps, DT, velocity, PE)
    m0 = [sf.mass(x, g, p) for x, g, p in zip(xs, gs, ps)]
    m1 = [sf.mass(x, g, p) for x, g, p in zip(r["x"], r["gamma"], ps)]
    cat = lambda lst: np.concatenate([np.asarray(v).ravel() for v in lst])  # noqa: E731
    np.savez(OUT, ids=np.array(IDS), p=np.array(ps), lam=lam, dt=DT, pe=PE, shear=SHEAR, up=w.up,
             u0=cat(r["u0"]), uh=cat(r["uh"]), gamma_h=cat(r["gamma_h"]), x1=cat(r["x"]), gamma1=cat(r["gamma"]),
             mass0=np.array(m0), mass1=np.array(m1))
    cons = np.abs(np.array(m1) - np.array(m0)) / np.abs(np.array(m0))
    print(f"wrote {OUT} in {time.time() - t0:.0f} s; conservation error per drop {cons}")


if __name__ == "__main__":
    main()
