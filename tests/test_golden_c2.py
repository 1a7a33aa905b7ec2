"""Checks of the stored oracle solution of the full-size single-drop shear system
(tests/golden/c2_solution.npz, written by tests/golden/make_c2_solution.py from the oracle alone)
against invariants of the continuous problem that its construction does not enforce directly:
the right-hand side 2 u_inf + S[f] and the solution u carry no net volume flux through the drop
surface (u_inf is divergence-free, the single layer is the velocity of an incompressible flow, and
the solution of Eq. main_eq is the surface velocity of an incompressible drop)."""
import os

import numpy as np

from oracle import layer
from paper_1707_02156_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_solution.npz")


def _flux(grid, coef):
    u = grid.density(coef)
    return abs(np.sum(grid.wJ * np.sum(u * grid.n, axis=0))) / (np.sum(grid.wJ) * np.max(np.abs(u)))


def test_stored_solution_matches_its_workload_and_converged():
    z = np.load(GOLDEN)
    w = inputs.perturbed_drop()
    assert int(z["p"]) == w.p[0] and int(z["pq"]) == w.pq[0]
    assert float(z["lam"][0]) == w.lam[0] and float(z["shear"]) == w.shear
    assert z["b"].shape == z["u"].shape == (3 * (w.p[0] + 1) ** 2,)
    assert z["residuals"][-1] <= 1e-13


def test_stored_rhs_and_solution_carry_no_volume_flux():
    z = np.load(GOLDEN)
    w = inputs.perturbed_drop()
    p = w.p[0]
    g = layer.DropGrid(w.xcoef.reshape(3, -1), p, 2 * p + 1)
    assert _flux(g, z["b"]) < 1e-13
    assert _flux(g, z["u"]) < 1e-13
    # a vector that is not such a velocity field fails the same check
    rng = np.random.default_rng(0)
    assert _flux(g, z["u"] + 1e-3 * rng.standard_normal(z["u"].shape)) > 1e-8
