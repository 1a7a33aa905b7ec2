"""Pins of the off-surface evaluation of the oracle (oracle/offsurface.py): closed forms in every
region, brute-force integration on deformed drops, and the continuity of the velocity across an
interface that the paper states (Sec. 1) for a system solved with the oracle's own GMRES."""
import math

import numpy as np
import pytest

from oracle import brute, gmres, layer, offsurface, sh
from paper_1707_02156_gb300 import inputs


def _translating_sphere(xt, centre, a, cvec):
    # (1/8pi) int_sphere G . c ds at exterior points: the Stokes field of a translating sphere
    xh = xt - np.asarray(centre)[:, None]
    r = np.linalg.norm(xh, axis=0)
    xc = np.sum(xh * cvec[:, None], axis=0)
    G = cvec[:, None] / r + xh * xc / r ** 3
    dip = cvec[:, None] / r ** 3 - 3 * xh * xc / r ** 5
    return 0.5 * a * a * (G + a * a / 3.0 * dip)


def _points_off(xcoef, p, params, dists):
    pts = []
    for (t0, f0), dist in zip(params, dists):
        d = [sh.evaluate_derivs(xcoef[c], p, np.array([t0]), np.array([f0])) for c in range(3)]
        xt, xp = np.array([d[c]["t"][0] for c in range(3)]), np.array([d[c]["p"][0] for c in range(3)])
        n = np.cross(xt, xp)
        pts.append(np.array([d[c]["f"][0] for c in range(3)]) + dist * n / np.linalg.norm(n))
    return np.array(pts).T


def test_translating_sphere_field_and_double_layer_identity_in_every_region():
    # a uniform traction c on a sphere of radius a: (1/8pi) int G.c is the translating-sphere field
    # outside, and the double layer of a constant density vanishes outside (double-layer identity)
    p, a, c0 = 16, 0.9, (0.1, -0.2, 0.3)
    x = inputs.sphere_coef(p, radius=a, centre=c0)
    cvec = np.array([0.4, -1.0, 0.7])
    dens = np.zeros((3, (p + 1) ** 2))
    dens[:, 0] = cvec * math.sqrt(4 * math.pi)
    drops = layer.Drops([x], [p], [p], [2.0], up=4)
    h = drops.h[0]
    pts = _points_off(x, p, ((1.0, 0.5), (2.0, 2.5), (0.3, 4.0), (2.9, 1.0)), (0.3 * h, 0.8 * h, 3.0 * h, 9.0 * h))
    codes = offsurface.classify_points(drops, pts, 0)
    assert list(codes) == [2, 2, 1, 0]
    S = offsurface.layer_at(drops, pts, [dens], "S", raw=True)
    exact = _translating_sphere(pts, c0, a, cvec)
    D = offsurface.layer_at(drops, pts, [dens], "D", raw=True)
    # regular and upsampled rules: quadrature-exact to rounding; Omega_2: the interpolation's error
    assert np.max(np.abs(S - exact)[:, 2:]) < 1e-12 * np.max(np.abs(exact))
    assert np.max(np.abs(S - exact)[:, :2]) < 1e-5 * np.max(np.abs(exact))
    assert np.max(np.abs(D[:, 2:])) < 1e-12 and np.max(np.abs(D[:, :2])) < 1e-5


def test_inside_points_are_rejected():
    p = 8
    x = inputs.sphere_coef(p, radius=1.0)
    drops = layer.Drops([x], [p], [p], [1.0], up=2)
    pts = np.array([[0.2, 0.0, 0.0], [3.0, 0.1, 0.0], [0.0, 0.0, 0.0]]).T
    assert list(offsurface.classify_points(drops, pts, 0)) == [offsurface.INSIDE, 0, offsurface.INSIDE]
    with pytest.raises(ValueError):
        offsurface.layer_at(drops, pts, [np.zeros((3, (p + 1) ** 2))], "S")


def test_layers_converge_to_brute_force_on_two_deformed_drops():
    # shape and densities band-limited at degree 4; points near drop 1 in each of its regions, which
    # also receive the far sum of drop 0; the rules converge spectrally in p to the brute-force
    # integrals, summed with the operators' weights
    rng = np.random.default_rng(41)
    x1 = inputs.sphere_coef(4, centre=(0.0, 0.0, 0.0)) + inputs.perturbation(rng, 4, 1, 4, 0.06)
    x0 = inputs.sphere_coef(4, radius=0.6, centre=(3.2, 0.5, -0.4)) + inputs.perturbation(rng, 4, 2, 4, 0.03)
    d0, d1 = inputs.random_bandlimited(rng, 4, 3), inputs.random_bandlimited(rng, 4, 3)
    lam = [0.5, 3.0]
    pts = _points_off(x1, 4, ((1.0, 0.5), (2.0, 2.5), (0.6, 4.0)), (0.05, 0.35, 1.5))
    for kind in ("S", "D"):
        ref = np.zeros((3, 3))
        for j, (xj, dj) in enumerate(((x0, d0), (x1, d1))):
            w = -1 / (4 * math.pi) if kind == "S" else (lam[j] - 1) / (4 * math.pi)
            ref += w * np.stack([brute.exterior_integral(xj, 4, dj, pts[:, i], kind) for i in range(3)], axis=1)
        errs = []
        for p in (8, 16):
            pad = lambda c: np.pad(c, ((0, 0), (0, (p + 1) ** 2 - 25)))
            drops = layer.Drops([pad(x0), pad(x1)], [p, p], [p, p], lam, up=4)
            codes = offsurface.classify_points(drops, pts, 1)
            assert codes[0] == 2 and codes[1] == 1 and codes[2] < 2
            v = offsurface.layer_at(drops, pts, [pad(d0), pad(d1)], kind)
            errs.append(np.max(np.abs(v - ref), axis=0) / np.max(np.abs(ref)))
        # regular and upsampled rules: spectral, at the brute force's 1e-12 by p = 16; the Omega_2 point (0.05
        # off the surface): the interpolation's error (the bound of the on-surface test of the rule),
        # which falls by more than 10x from p = 8 to 16
        assert np.max(errs[1][1:]) < 1e-10, (kind, errs)
        assert errs[1][0] < 2e-3 and errs[1][0] < 0.1 * errs[0][0], (kind, errs)


def test_velocity_is_continuous_across_the_interface():
    # Sec. 1: the velocity field is continuous across the interfaces.  Solve Eq. main_eq for a
    # deformed drop in shear (lambda = 3) with the oracle's GMRES; the off-surface velocity at
    # x_g + eps n_g, extrapolated to eps = 0 (Richardson), must equal the interface velocity u(x_g).
    # A wrong sign or factor of either layer in the off-surface formula moves it by O(1).
    p, lam, shear = 10, 3.0, 1.0
    rng = np.random.default_rng(12)
    x = inputs.sphere_coef(p, axes=(1.1, 0.95, 0.9)) + inputs.perturbation(rng, p, 2, 4, 0.03)
    f = inputs.random_bandlimited(rng, p, 3, decay_pow=3.0)
    drops = layer.Drops([x], [p], [2 * p + 1], [lam], up=4)
    b = drops.rhs([f], shear)
    u, info = gmres.gmres(drops.system_matvec, b, tol=1e-13, restart=40, max_it=200)
    assert info["converged"]
    uc = drops.split(u)[0]
    params = ((0.7, 0.3), (1.9, 2.2), (2.6, 5.0))
    for (t0, f0) in params:
        ug = np.array([sh.evaluate(uc[c], p, np.array([t0]), np.array([f0]))[0] for c in range(3)])
        v = []
        for eps in (2e-3, 4e-3):
            pt = _points_off(x, p, ((t0, f0),), (eps,))
            v.append(offsurface.velocity_at(drops, pt, [f], [uc], shear)[:, 0])
        v0 = 2 * v[0] - v[1]
        # the interpolation and the O(eps^2) remainder leave about 1e-4; a wrong sign or factor is O(1)
        assert np.max(np.abs(v0 - ug)) < 1e-3 * np.max(np.abs(ug)), (v0, ug)
