"""Pins of the oracle's geometry (Table 2) and interfacial force (Sec. 1) against closed forms."""
import math

import numpy as np

from oracle import geometry, layer, sh
from paper_1707_02156_gb300 import inputs


def test_sphere_forms_normal_and_curvature():
    p, R = 6, 1.7
    x = inputs.sphere_coef(p, radius=R, centre=(0.2, -0.1, 0.4))
    t, w, theta, phi = sh.gauss_grid(p)
    g = geometry.forms(geometry.surface_fields(x, p, p))
    rhat = (g["x"] - np.array([0.2, -0.1, 0.4])[:, None, None]) / R
    assert np.max(np.abs(g["n"] - rhat)) < 1e-14            # outward normal
    assert np.max(np.abs(g["K"] + 1.0 / R)) < 1e-13         # mean curvature -1/R
    assert np.max(np.abs(g["KG"] - 1.0 / R ** 2)) < 1e-13   # Gaussian curvature 1/R^2
    assert np.max(np.abs(geometry.area_density(g["W"], theta) - R * R)) < 1e-13


def test_ellipsoid_volume_and_mean_radius():
    p = 4
    Q = inputs.random_rotation(np.random.default_rng(2))
    x = inputs.sphere_coef(p, centre=(1.0, 2.0, 3.0), axes=(0.7, 1.1, 1.3), rot=Q)
    assert abs(geometry.volume(x, p, 20) - 4.0 / 3.0 * math.pi * 0.7 * 1.1 * 1.3) < 1e-12
    assert abs(geometry.mean_radius(x, p) - (0.7 * 1.1 * 1.3) ** (1 / 3)) < 1e-12


def test_clean_sphere_force_is_outward_two_sigma_over_r():
    p, R = 6, 1.3
    x = inputs.sphere_coef(p, radius=R)
    gam = np.zeros((p + 1) ** 2)
    gam[0] = math.sqrt(4 * math.pi)
    f = geometry.interfacial_force(x, p, gam, elasticity=0.2)
    fg = np.stack([sh.synthesize(f[c], p, p) for c in range(3)])
    g = geometry.forms(geometry.surface_fields(x, p, p))
    sigma = 1.0 - 0.2
    assert np.max(np.abs(fg - 2.0 * sigma / R * g["n"])) < 1e-13


def test_marangoni_term_points_down_the_tension_gradient_sign_reading():
    # Unit sphere with sigma = 1 + eps z (Gamma linear in z, E < 0 sign trick avoided: use E = -eps).
    p = 6
    x = inputs.sphere_coef(p)
    gam = np.zeros((p + 1) ** 2)
    gam[0] = math.sqrt(4 * math.pi)
    gam[2] = math.sqrt(4 * math.pi / 3.0)  # Gamma = 1 + z
    eps = 0.1
    f = geometry.interfacial_force(x, p, gam, elasticity=-eps)  # sigma = 1 + eps (1 + z)
    fg = np.stack([sh.synthesize(f[c], p, p) for c in range(3)])
    g = geometry.forms(geometry.surface_fields(x, p, p))
    tang = fg - np.sum(fg * g["n"], axis=0) * g["n"]
    # -grad sigma: tangential force points towards lower z, i.e. lower tension
    zhat_t = np.array([0, 0, 1.0])[:, None, None] - g["n"][2] * g["n"]
    assert np.all(np.sum(tang * zhat_t, axis=0) <= 1e-14)
    # and its magnitude is eps sin(theta)
    _, _, theta, _ = sh.gauss_grid(p)
    assert np.max(np.abs(np.linalg.norm(tang, axis=0) - eps * np.sin(theta)[:, None])) < 1e-13


def test_rotated_geometry_matches_direct_evaluation_at_rotated_points():
    p, pq = 6, 13
    rng = np.random.default_rng(8)
    x = inputs.sphere_coef(p) + inputs.perturbation(rng, p, 1, 4, 0.15)
    q = layer.SelfQuadrature(x, p, pq)
    _, _, theta, phi = sh.gauss_grid(p)
    a = 2
    xr, nr, wJ = q.rotated_geometry(a)
    ws = layer.singular_weights(pq)
    _, _, thq, _ = sh.gauss_grid(pq)
    for b in (0, 5, 13):
        th, ph = layer.rotated_points(theta[a], phi[b], pq)
        d = [sh.evaluate_derivs(x[c], p, th, ph) for c in range(3)]
        X = np.stack([d[c]["f"] for c in range(3)])
        cr = np.cross(np.stack([d[c]["t"] for c in range(3)]), np.stack([d[c]["p"] for c in range(3)]), axis=0)
        W = np.linalg.norm(cr, axis=0)
        assert np.max(np.abs(xr[b] - X)) < 1e-13
        assert np.max(np.abs(nr[b] - cr / W)) < 1e-12
        J = W / np.sin(th)
        assert np.max(np.abs(wJ[b] - ws[:, None] * J)) < 1e-12 * np.max(np.abs(wJ[b]))


def test_interfacial_force_carries_no_net_force_or_torque():
    # f = sigma (div n) n - grad_gamma sigma is the surface divergence of the symmetric surface stress
    # sigma (I - n n): on any closed surface, for any tension field, int f dS = 0 and
    # int x x f dS = 0.  A deformed, rotated drop with a non-uniform surfactant and the Langmuir
    # equation of state; the projected force converges to zero net force and torque as p grows.
    res = []
    for p in (8, 16):
        x = inputs.sphere_coef(p, axes=(0.8, 1.0, 1.2), rot=inputs.random_rotation(np.random.default_rng(1)))
        x[:, :25] += inputs.perturbation(np.random.default_rng(2), 4, 1, 4, 0.05)
        g = np.zeros((p + 1) ** 2)
        g[:16] = 0.2 * inputs.random_bandlimited(np.random.default_rng(3), 3, 1)[0]
        g[0] += math.sqrt(4 * math.pi)
        f = geometry.interfacial_force(x, p, g, 0.3, 0.3)
        P = 4 * (p + 1) - 1
        _, w, theta, _ = sh.gauss_grid(P)
        F = np.stack([sh.synthesize(f[c], p, P) for c in range(3)])
        G = geometry.forms(geometry.surface_fields(x, p, P))
        wq = (np.pi / (P + 1)) * w[:, None] * geometry.area_density(G["W"], theta)
        scale = np.sum(np.linalg.norm(F, axis=0) * wq)
        force = np.max(np.abs(np.sum(F * wq, axis=(1, 2)))) / scale
        torque = np.max(np.abs(np.sum(np.cross(G["x"], F, axis=0) * wq, axis=(1, 2)))) / scale
        res.append(max(force, torque))
    assert res[1] < 1e-11 and res[1] < 1e-4 * res[0], res
