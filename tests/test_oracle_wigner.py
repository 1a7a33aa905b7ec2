"""Pins of the oracle's Wigner rotation (App. B): the printed factorial sum, unitarity, and the
defining property g(s) = f(R s) checked by direct evaluation at rotated points."""

import numpy as np
import pytest

from oracle import sh, wigner
from paper_1707_02156_gb300 import inputs


@pytest.mark.parametrize("beta", [0.3, 1.2, 2.7])
def test_small_d_equals_app_b_factorial_sum(beta):
    for n in (1, 4, 9):
        d = wigner.small_d(n, beta)
        for mp in range(-n, n + 1):
            for m in range(-n, n + 1):
                ref = float(wigner.small_d_factorial(n, mp, m, beta))
                assert abs(d[mp + n, m + n] - ref) < 1e-14


def test_small_d_orthogonal_to_high_degree():
    for n in (16, 33, 48, 65):
        d = wigner.small_d(n, 0.77)
        assert np.max(np.abs(d @ d.T - np.eye(2 * n + 1))) < 1e-12


def test_rotated_expansion_is_function_at_rotated_points():
    p = 9
    rng = np.random.default_rng(11)
    f = inputs.random_bandlimited(rng, p, 1, decay_pow=0.5)[0]
    for (a, b, g) in ((0.4, 1.0, 0.0), (2.0, 2.5, 0.7), (-1.0, -0.6, 3.0)):
        fr = wigner.rotate(f, p, a, b, g)
        th = rng.uniform(0.05, 3.1, 40)
        ph = rng.uniform(0.0, 2 * np.pi, 40)
        s = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
        v = wigner.rotation_matrix(a, b, g) @ s
        th2, ph2 = np.arccos(np.clip(v[2], -1, 1)), np.arctan2(v[1], v[0])
        assert np.max(np.abs(sh.evaluate(fr, p, th, ph) - sh.evaluate(f, p, th2, ph2))) < 1e-13
        # per-degree energy is preserved
        c, cr = sh.to_complex(f, p), sh.to_complex(fr, p)
        for n in range(p + 1):
            e0 = abs(c[n, 0]) ** 2 + 2 * np.sum(np.abs(c[n, 1:n + 1]) ** 2)
            e1 = abs(cr[n, 0]) ** 2 + 2 * np.sum(np.abs(cr[n, 1:n + 1]) ** 2)
            assert abs(e0 - e1) < 1e-13 * max(1.0, e0)


def test_pole_of_rotated_surface_is_the_target():
    p = 8
    rng = np.random.default_rng(5)
    x = inputs.sphere_coef(p) + inputs.perturbation(rng, p, 1, 5, 0.1)
    _, _, theta, phi = sh.gauss_grid(p)
    for a, b in ((0, 0), (3, 7), (8, 17)):
        target = [sh.evaluate(x[c], p, np.array([theta[a]]), np.array([phi[b]]))[0] for c in range(3)]
        pole = [sh.evaluate(wigner.rotate(x[c], p, phi[b], theta[a]), p, np.array([0.0]), np.array([0.0]))[0]
                for c in range(3)]
        assert np.max(np.abs(np.array(target) - np.array(pole))) < 1e-14
