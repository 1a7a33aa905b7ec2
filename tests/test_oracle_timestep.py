"""Pins of the oracle's midpoint step of the drop shapes (Sec. 3, Alg. 1, surfactant held fixed)."""
import numpy as np

from oracle import geometry, timestep
from paper_1707_02156_gb300 import inputs


def _gamma_one(p):
    g = np.zeros((p + 1) ** 2)
    g[0] = np.sqrt(4 * np.pi)  # Gamma = 1: the degree-0 coefficient of a constant
    return g


def test_volume_change_per_step_is_third_order():
    # the velocity is divergence-free (int u.n dS = 0), so a second-order step changes the volume by
    # O(dt^3): halving dt divides the change by 8
    rng = np.random.default_rng(7)
    p = 6
    x = inputs.sphere_coef(p, axes=(1.1, 0.95, 0.95)) + inputs.perturbation(rng, p, 2, 4, 0.02)
    v0 = geometry.volume(x, p, 2 * p + 1)
    dv = []
    for dt in (0.1, 0.05):
        x1 = timestep.midpoint_step([x], [p], [p], [2.0], [_gamma_one(p)], 0.2, 0.0, 1.0, dt)[0]
        dv.append(abs(geometry.volume(x1, p, 2 * p + 1) - v0) / v0)
    assert dv[1] < 2e-6
    assert 6.5 < dv[0] / dv[1] < 9.5


def test_clean_sphere_at_rest_stays_put():
    # uniform tension on a sphere gives a uniform normal traction, whose single layer vanishes
    # (S[n] = 0 on a closed surface): with no far field the velocity is zero
    p = 5
    x = inputs.sphere_coef(p, radius=0.9, centre=(0.3, -0.2, 0.1))
    x1 = timestep.midpoint_step([x], [p], [p], [3.0], [_gamma_one(p)], 0.2, 0.0, 0.0, 0.1)[0]
    assert np.max(np.abs(x1 - x)) < 1e-12
