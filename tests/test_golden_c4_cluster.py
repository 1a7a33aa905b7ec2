"""Checks of the stored oracle coupled step of the four-drop cluster (tests/golden/c4_cluster_step.npz,
written by tests/golden/make_c4_cluster_step.py from the oracle alone) against invariants of the
continuous problem: both interface velocities carry no net volume flux through their drop's surface
(the drops are incompressible), and each drop's surfactant mass changes over the step only by the
scheme's error (the exact transport conserves it)."""
import os

import numpy as np

from oracle import layer
from paper_1707_02156_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c4_cluster_step.npz")


def test_stored_cluster_step_matches_its_workload():
    z = np.load(GOLDEN)
    w = inputs.config("c4")
    assert [w.p[int(i)] for i in z["ids"]] == [int(p) for p in z["p"]]
    assert np.allclose([w.lam[int(i)] for i in z["ids"]], z["lam"], rtol=0, atol=0)
    assert float(z["dt"]) == 0.01 and float(z["pe"]) == 10.0 and int(z["up"]) == w.up


def test_stored_velocities_carry_no_volume_flux_and_mass_is_kept():
    z = np.load(GOLDEN)
    w = inputs.config("c4")
    offs = np.cumsum([0] + [3 * (p + 1) ** 2 for p in w.p])
    dt = float(z["dt"])
    o = 0
    for i, p in zip(z["ids"], z["p"]):
        i, p = int(i), int(p)
        k = 3 * (p + 1) ** 2
        x0 = w.xcoef[offs[i]:offs[i + 1]].reshape(3, -1)
        for name, x in (("u0", x0), ("uh", x0 + 0.5 * dt * z["u0"][o:o + k].reshape(3, -1))):
            grid = layer.DropGrid(x, p, 2 * p + 1)
            u = grid.density(z[name][o:o + k])
            flux = abs(np.sum(grid.wJ * np.sum(u * grid.n, axis=0))) / (np.sum(grid.wJ) * np.max(np.abs(u)))
            assert flux < 1e-11, (i, name, flux)
        o += k
    cons = np.abs(z["mass1"] - z["mass0"]) / np.abs(z["mass0"])
    assert np.all(cons < 1e-7), cons
