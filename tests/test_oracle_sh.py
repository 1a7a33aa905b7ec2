"""Pins of the oracle's SH grid, basis and transforms (Sec. 1.1, Sec. 2.1, App. A) against
library routines, closed forms and finite differences."""
import math

import numpy as np
import pytest
import scipy.special

from oracle import sh
from paper_1707_02156_gb300 import inputs


def test_legendre_recursion_matches_library_harmonics():
    # App. A recursion (with Condon-Shortley phase) against scipy's orthonormal Y_n^m.
    p = 12
    theta = np.linspace(0.05, 3.09, 17)
    phi = np.linspace(0.0, 6.0, 17)
    P = sh.legendre_normalised(p, np.cos(theta))
    for n in range(p + 1):
        for m in range(n + 1):
            ref = scipy.special.sph_harm_y(n, m, theta, phi)
            mine = P[n, m] * np.exp(1j * m * phi)
            assert np.max(np.abs(ref - mine)) < 1e-13, (n, m)


def test_discrete_orthogonality_needs_2p_plus_2_points_and_pi_over_p_plus_1():
    # Sec. 2.1 discrete orthogonality (Y_n^m, Y_n'^m')^p = delta delta, for all pairs up to p.
    p = 7
    t, w, theta, phi = sh.gauss_grid(p)
    assert len(phi) == 2 * p + 2
    T, F = np.meshgrid(theta, phi, indexing="ij")
    basis = []
    for n in range(p + 1):
        for m in range(-n, n + 1):
            basis.append(scipy.special.sph_harm_y(n, m, T, F))
    B = np.array(basis).reshape(len(basis), -1)
    wq = ((np.pi / (p + 1)) * np.repeat(w, 2 * p + 2)).reshape(-1)
    G = (B * wq) @ B.conj().T
    assert np.max(np.abs(G - np.eye(len(basis)))) < 1e-14
    # with the printed factor pi/p the Gram matrix is off by (p+1)/p
    assert abs(np.pi / p * (p + 1) / np.pi - 1.0) > 0.1


def test_area_of_unit_sphere_by_regular_rule():
    # int Y_0^0 dS = sqrt(4 pi) on the unit sphere (W = sin theta).
    p = 5
    g = np.full((p + 1, 2 * p + 2), 1.0 / math.sqrt(4 * math.pi))
    c = sh.analyze(g, p, p)
    assert abs(c[0] - 1.0) < 1e-15
    assert np.max(np.abs(c[1:])) < 1e-15


@pytest.mark.parametrize("p_grid", [9, 10, 19])
def test_round_trip_and_zero_padding(p_grid):
    p = 9
    rng = np.random.default_rng(3)
    f = inputs.random_bandlimited(rng, p, 1)[0]
    g = sh.synthesize(f, p, p_grid)
    back = sh.analyze(g, p_grid, p)
    assert np.max(np.abs(back - f)) < 1e-14
    # synthesis equals direct evaluation of the series at the grid points
    t, w, theta, phi = sh.gauss_grid(p_grid)
    T, F = np.meshgrid(theta, phi, indexing="ij")
    assert np.max(np.abs(sh.evaluate(f, p, T, F) - g)) < 1e-13
    # and equals scipy's harmonics summed with the complex coefficients
    c = sh.to_complex(f, p)
    ref = np.zeros(T.shape, dtype=np.complex128)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            fm = c[n, m] if m >= 0 else (-1) ** m * np.conj(c[n, -m])
            ref += fm * scipy.special.sph_harm_y(n, m, T, F)
    assert np.max(np.abs(ref.imag)) < 1e-13
    assert np.max(np.abs(ref.real - g)) < 1e-13


def test_theta_derivatives_against_finite_differences():
    # App. A first derivative (cot phi read as cot theta) and the Legendre-equation second derivative.
    p = 10
    rng = np.random.default_rng(4)
    f = inputs.random_bandlimited(rng, p, 1, decay_pow=0.0)[0]
    th = np.linspace(0.2, 2.9, 9)
    ph = np.linspace(0.1, 6.0, 9)
    d = sh.evaluate_derivs(f, p, th, ph)
    e = 1e-5
    fd_t = (sh.evaluate(f, p, th + e, ph) - sh.evaluate(f, p, th - e, ph)) / (2 * e)
    fd_p = (sh.evaluate(f, p, th, ph + e) - sh.evaluate(f, p, th, ph - e)) / (2 * e)
    fd_tt = (sh.evaluate_derivs(f, p, th + e, ph)["t"] - sh.evaluate_derivs(f, p, th - e, ph)["t"]) / (2 * e)
    fd_tp = (sh.evaluate_derivs(f, p, th, ph + e)["t"] - sh.evaluate_derivs(f, p, th, ph - e)["t"]) / (2 * e)
    fd_pp = (sh.evaluate_derivs(f, p, th, ph + e)["p"] - sh.evaluate_derivs(f, p, th, ph - e)["p"]) / (2 * e)
    scale = np.max(np.abs(d["f"])) * p * p
    for key, fd in (("t", fd_t), ("p", fd_p), ("tt", fd_tt), ("tp", fd_tp), ("pp", fd_pp)):
        assert np.max(np.abs(d[key] - fd)) < 1e-7 * scale, key


def test_laplace_beltrami_eigen_relation():
    # Sec. 3.2.1: spherical harmonics are eigenfunctions of the surface Laplacian, eigenvalue -n(n+1).
    p = 8
    theta = np.linspace(0.3, 2.8, 7)
    phi = np.linspace(0.2, 5.0, 7)
    for n in (1, 3, 8):
        for m in (0, 1, n):
            f = np.zeros((p + 1) ** 2)
            f[n * (n + 1) + m] = 1.0
            d = sh.evaluate_derivs(f, p, theta, phi)
            lap = d["tt"] + np.cos(theta) / np.sin(theta) * d["t"] + d["pp"] / np.sin(theta) ** 2
            assert np.max(np.abs(lap + n * (n + 1) * d["f"])) < 1e-11
