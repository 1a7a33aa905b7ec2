"""Pins of the oracle's angle reparametrisation (Sec. 4, Alg. 2): the adaptive cutoff and the
mode norms against hand-computed spectra and Parseval's identity, the angle velocity against
finite differences, the paper's surfactant check (a concentration linear in the position is
carried exactly), the distorted sphere that must return to its one-mode parametrisation, and the
spectral decay of the volume error with the upsampling factor."""
import math

import numpy as np
import pytest

from oracle import geometry, reparam as rp, sh


def _twisted(p, kappa, axes=(1.0, 1.0, 1.0)):
    """The surface x(theta, phi + kappa cos theta) of the ellipsoid with the given axes: the same
    surface, its latitude circles turned against each other (a distorted parametrisation)."""
    _, _, th, ph = sh.gauss_grid(p)
    T, F = np.meshgrid(th, ph, indexing="ij")
    F2 = F + kappa * np.cos(T)
    X = np.stack([axes[0] * np.sin(T) * np.cos(F2), axes[1] * np.sin(T) * np.sin(F2), axes[2] * np.cos(T)])
    return np.stack([sh.analyze(X[c], p, p) for c in range(3)])


def test_mode_norms_satisfy_parseval_on_the_unit_sphere():
    # int_{S^2} |x|^2 dOmega = sum_{n, m = -n..n} |x_n^m|^2 (orthonormal Y_n^m): pins the norm of a
    # vector coefficient and the doubling of m > 0 by the real symmetry
    p = 6
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, (p + 1) ** 2))
    P = 2 * p + 1
    t, w, theta, phi = sh.gauss_grid(P)
    X = np.stack([sh.synthesize(x[c], p, P) for c in range(3)])
    integral = (np.pi / (P + 1)) * np.sum(w[:, None] * np.sum(X * X, axis=0))
    assert abs(np.sum(rp.mode_norms(x, p) ** 2) - integral) < 1e-12 * integral


def test_adaptive_cutoff_on_a_designed_spectrum():
    # per-degree sums s_n = 1, 1/2, 1/4, 1/8, 1/16 for n = 1..5 (all in m = 0 of one component):
    # N_2(l)/N_1 = 0.4839, 0.2258, 0.0968, 0.0323 for l = 2..5
    P = 5
    x = np.zeros((3, (P + 1) ** 2))
    for n in range(1, P + 1):
        x[0, n * (n + 1)] = 0.5 ** (n - 1)
    for pc, l in ((0.5, 2), (0.3, 3), (0.1, 4), (0.05, 5), (0.01, 5)):
        assert rp.adaptive_cutoff(x, P, pc) == l, pc
    # the same weight on m = 1 counts twice (m = +-1): s_3 -> 2/4, N_2(3)/N_1 = 0.35 > 0.3
    y = x.copy()
    y[0, 3 * 4] = 0.0
    y[1, 3 * 4 + 1] = 0.25
    assert rp.adaptive_cutoff(y, P, 0.3) == 4
    # a sphere has no degree >= 2: the cutoff is 2 for any fraction
    s = _twisted(P, 0.0)
    assert rp.adaptive_cutoff(s, P, 1e-3) == 2
    # energies with the two filters
    a1, a2 = rp.attenuation(P, 3, False), rp.attenuation(P, 3, True)
    e = [0.5 ** (2 * (n - 1)) for n in range(P + 1)]
    assert rp.energy(x, P, a1) == pytest.approx(sum(e[3:]), rel=1e-14)
    assert rp.energy(x, P, a2) == pytest.approx(sum(n / P * e[n] for n in range(3, P + 1)), rel=1e-14)


def test_angle_velocity_moves_the_point_with_the_tangential_velocity():
    # chain rule (Eq. system_rep): x(theta + h a_t, phi + h a_p) - x(theta, phi) = h (I - n n) w + O(h^2)
    p = 7
    rng = np.random.default_rng(4)
    x = _twisted(p, 0.6, axes=(0.8, 1.0, 1.4))
    th = rng.uniform(0.3, 2.8, 12)
    ph = rng.uniform(0.0, 2 * np.pi, 12)
    w = rng.standard_normal((3, 12))
    e = rp.tangent_fields(x, p, th, ph)
    wt = w - np.sum(w * e["n"], axis=0) * e["n"]
    at, ap = rp.angle_velocity(e, w)
    errs = []
    for h in (1e-3, 5e-4):
        xn = np.stack([sh.evaluate(x[c], p, th + h * at, ph + h * ap) for c in range(3)])
        errs.append(np.max(np.abs((xn - e["f"]) / h - wt)))
    assert errs[1] < 1e-2 and 1.8 < errs[0] / errs[1] < 2.2   # first-order remainder O(h)


def test_distorted_sphere_returns_to_its_one_mode_parametrisation():
    # Sec. 4: a distorted grid on a sphere needs only the degree-1 modes once reparametrised, which the
    # adaptive cutoff reaches
    p = 8
    x = _twisted(p, 1.0)
    assert np.sum(rp.mode_norms(x, p)[2:]) > 1.0
    g = np.zeros((p + 1) ** 2)
    g[0] = math.sqrt(4 * math.pi)
    xo, go, info = rp.reparametrize(x, g, p, u_rep=2, p_cutoff=0.4, dtau=0.5, eps=1e-8)
    h = info["history"]
    assert h[-1]["g"] < 1e-8 and len(h) < 60
    assert all(b["energy"] <= a["energy"] * (1 + 1e-12) for a, b in zip(h, h[1:]))
    assert np.sum(rp.mode_norms(xo, p)[2:]) < 1e-6
    # still the unit sphere
    X = np.stack([sh.synthesize(xo[c], p, p) for c in range(3)])
    assert np.max(np.abs(np.linalg.norm(X, axis=0) - 1.0)) < 1e-7


def test_concentration_linear_in_the_position_is_carried_exactly():
    # Sec. 4: Gamma = 2 - x1/2 + x2 + x3/2 on a distorted ellipsoid keeps that form after the angle
    # reparametrisation.  The paper reports an error below 1e-15; measured here on the degree-p grid
    # after the round trip through the coefficients it is 1.5e-15 relative, rounding of the
    # synthesis sums, so the bound is 1e-14 (any evaluation at wrong angles errs by O(0.1))
    p = 7
    x = _twisted(p, 0.8, axes=(0.5, 0.5, 1.0))
    g = -0.5 * x[0] + x[1] + 0.5 * x[2]
    g[0] += 2.0 * math.sqrt(4 * math.pi)
    xo, go, info = rp.reparametrize(x, g, p, u_rep=2, p_cutoff=0.4, dtau=0.5, i_max=30)
    G = sh.synthesize(go, p, p)
    X = np.stack([sh.synthesize(xo[c], p, p) for c in range(3)])
    assert np.max(np.abs(G - (2.0 - 0.5 * X[0] + X[1] + 0.5 * X[2]))) < 1e-14 * np.max(np.abs(G))
    assert info["history"][-1]["energy"] < 1e-3 * info["history"][0]["energy"]


def test_volume_error_decays_spectrally_with_the_upsampling_factor():
    p = 7
    x = _twisted(p, 0.8, axes=(0.5, 0.5, 1.0))
    g = np.zeros((p + 1) ** 2)
    g[0] = math.sqrt(4 * math.pi)
    v0 = 4.0 / 3.0 * math.pi * 0.5 * 0.5 * 1.0
    errs = []
    for u in (1, 2, 3):
        xo, _, _ = rp.reparametrize(x, g, p, u_rep=u, p_cutoff=0.4, dtau=0.5, i_max=30)
        errs.append(abs(geometry.volume(xo, p, 2 * p + 1) - v0) / v0)
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 1e-3 * errs[0]


def _differential_rotation(xs, gs):
    # u = omega(z) (z^ x x) with omega = 1 + 2 z: every latitude circle of a sphere about the origin
    # turns at its own rate (tangential and surface-divergence-free), so the surface and Gamma as a
    # field on it stay as they are while the grid twists
    out = []
    for x in xs:
        p = int(round(math.sqrt(x.shape[1]))) - 1
        P = 2 * p + 1
        X = np.stack([sh.synthesize(x[c], p, P) for c in range(3)])
        om = 1.0 + 2.0 * X[2]
        U = np.stack([-om * X[1], om * X[0], np.zeros_like(X[0])])
        out.append(np.stack([sh.analyze(U[c], P, p) for c in range(3)]))
    return out


def test_reparametrisation_after_each_kept_step_removes_the_grid_twist_only():
    # Alg. 1 with Alg. 2 after every kept step: the grid energy stays low while the surface and the
    # surfactant field are those of the run without reparametrisation (mass, volume, int Gamma^2 dS)
    from oracle import surfactant as sf
    p = 8
    x = _twisted(p, 0.0)
    rng = np.random.default_rng(3)
    g = 0.2 * rp.upsample(rng.standard_normal((1, 16)), 3, p)[0]
    g[0] += math.sqrt(4 * math.pi)
    runs = {}
    for name, rep_opts in (("plain", None), ("reparam", {"u_rep": 2, "p_cutoff": 0.3, "dtau": 0.5, "i_max": 6})):
        res = sf.run_adaptive([x], [g], [p], 0.3, 0.1, 1e-3, _differential_rotation, math.inf, 0.1,
                              reparam=rep_opts)
        xo, go = res["x"][0], res["gamma"][0]
        S = sf.Surface(xo, p, sf.grid_degree(p))
        G = sf.scalar_fields(go, p, S.P)["f"]
        runs[name] = {"mass": S.integral(G), "second": S.integral(G * G), "volume": geometry.volume(xo, p, 2 * p + 1),
                      "high": float(np.sum(rp.mode_norms(xo, p)[2:] ** 2))}
    a, b = runs["plain"], runs["reparam"]
    assert a["high"] > 0.1 and b["high"] < 1e-6 * a["high"]
    for k in ("mass", "second", "volume"):
        assert abs(a[k] - b[k]) < 1e-7 * abs(a[k]), (k, a[k], b[k])
