"""Pins of the oracle's surfactant transport and coupled step (Eq. surfactant0, Sec. 3, Alg. 1)
against closed forms, geometric identities, the paper's own validation cases (Sec. 5: pure
diffusion, the expanding sphere with Gamma R^2 = Gamma(0), the rotating sphere) and the
conservation of surfactant mass."""
import math

import numpy as np
import pytest

from oracle import geometry, sh, surfactant as sf, timestep
from paper_1707_02156_gb300 import inputs


def _deformed(p, seed, amp=0.05):
    rng = np.random.default_rng(seed)
    Q = inputs.random_rotation(rng)
    x = inputs.sphere_coef(p, centre=(0.3, 0.1, -0.2), axes=(0.8, 1.0, 1.25), rot=Q)
    return x + inputs.perturbation(rng, p, 1, 5, amp), rng


def _field_coef(x, p, fn):
    """Degree-p coefficients of the vector field fn(points [3][j][k]) sampled on the surface x."""
    P = sf.grid_degree(p)
    X = geometry.surface_fields(np.asarray(x).reshape(3, -1), p, P)["f"]
    U = fn(X)
    return np.stack([sh.analyze(U[c], P, p) for c in range(3)])


def _gamma(p, rng, base=2.0):
    g = inputs.random_bandlimited(rng, p, 1)[0] * 0.3
    g[0] += base * math.sqrt(4 * math.pi)
    return g


def test_laplace_beltrami_on_a_sphere_of_radius_r():
    # Sec. 3 (Preconditioning): SH are eigenfunctions of the sphere's Laplacian, -n(n+1)/R^2.
    p, R = 8, 1.3
    P = sf.grid_degree(p)
    S = sf.Surface(inputs.sphere_coef(p, radius=R, centre=(0.2, -0.1, 0.3)), p, P)
    for n, m in ((1, 0), (1, 1), (3, 2), (8, 5)):
        y = np.zeros((p + 1) ** 2)
        y[n * (n + 1) + m] = 1.0
        if m:
            y[n * (n + 1) - m] = 0.4
        d = sf.scalar_fields(y, p, P)
        assert np.max(np.abs(d["f"])) > 0.1
        assert np.max(np.abs(S.lap(d) + n * (n + 1) / R ** 2 * d["f"])) < 1e-12


def test_surface_operators_of_the_position_vector_on_a_deformed_drop():
    # Identities of any smooth closed surface, pointwise: div x = 2, lap x = -(div n) n = 2 K n
    # (K the mean curvature of Table 2, -1/R on a sphere), div(Omega x x + V) = 0.
    p = 8
    P = sf.grid_degree(p)
    x, _ = _deformed(p, 3)
    S = sf.Surface(x, p, P)
    X = sf.vector_fields(x, p, P)
    assert np.max(np.abs(S.F)) > 0.05   # the parametrisation is not orthogonal
    assert np.max(np.abs(S.div(X["t"], X["p"]) - 2.0)) < 1e-12
    lapx = np.stack([S.lap({k: X[k][c] for k in X}) for c in range(3)])
    assert np.max(np.abs(lapx - 2.0 * S.K * S.n)) < 1e-11
    Om = np.array([0.3, -0.2, 0.7])
    rt = np.cross(Om[:, None, None], X["t"], axis=0)
    rp = np.cross(Om[:, None, None], X["p"], axis=0)
    assert np.max(np.abs(S.div(rt, rp))) < 1e-13


def test_green_identities_of_the_laplacian_on_a_deformed_drop():
    # int lap g dS = 0 and int f lap g dS = int g lap f dS on a closed surface (to quadrature error).
    p = 6
    P = 4 * (p + 1) - 1
    x, rng = _deformed(p, 4)
    S = sf.Surface(x, p, P)
    f = sf.scalar_fields(inputs.random_bandlimited(rng, p, 1)[0], p, P)
    g = sf.scalar_fields(inputs.random_bandlimited(rng, p, 1)[0], p, P)
    lf, lg = S.lap(f), S.lap(g)
    scale = S.integral(np.abs(f["f"] * lg))
    assert abs(S.integral(lg)) < 1e-10 * S.integral(np.abs(lg))
    assert abs(S.integral(f["f"] * lg) - S.integral(g["f"] * lf)) < 1e-10 * scale


def test_stretching_term_of_an_expanding_sphere():
    # Sec. 5, stretching test: u = c n on a sphere of radius R gives dGamma/dt = -(2c/R) Gamma,
    # for any Gamma (the tangential velocity is zero).
    p, R, c = 7, 1.2, 0.3
    centre = np.array([0.1, 0.4, -0.3])
    x = inputs.sphere_coef(p, radius=R, centre=tuple(centre))
    u = _field_coef(x, p, lambda X: c * (X - centre[:, None, None]) / R)
    rng = np.random.default_rng(9)
    g = _gamma(p, rng)
    fe = sf.f_explicit(x, u, g, p)
    assert np.max(np.abs(fe + 2.0 * c / R * g)) < 1e-12


def test_rigid_motion_leaves_any_concentration_unchanged():
    # Sec. 5, convection test: the points of a rigidly moving drop carry Gamma with them.
    p = 7
    x, rng = _deformed(p, 5)
    Om, V = np.array([0.4, -0.1, 0.8]), np.array([0.2, 0.0, -0.5])
    u = _field_coef(x, p, lambda X: np.cross(Om[:, None, None], X, axis=0) + V[:, None, None])
    g = _gamma(p, rng)
    assert np.max(np.abs(sf.f_explicit(x, u, g, p))) < 1e-13


def test_explicit_term_conserves_mass_at_every_instant():
    # d/dt int Gamma dS = int (dGamma/dt + Gamma div u) dS = int f_E + Gamma div u = 0 pointwise
    # in time; with the Galerkin projection it holds to truncation error for a smooth flow.
    p = 10
    x, rng = _deformed(p, 6, amp=0.03)
    u = _field_coef(x, p, lambda X: np.stack([0.5 * X[2] + 0.1 * X[0] * X[1], -0.2 * X[1], 0.3 * X[0] ** 2]))
    g = _gamma(p, rng)
    P = sf.grid_degree(p)
    S = sf.Surface(x, p, P)
    U = sf.vector_fields(u, p, P)
    G = sf.scalar_fields(g, p, P)["f"]
    rate = S.integral(sf.f_explicit_grid(S, u, g, p) + G * S.div(U["t"], U["p"]))
    assert abs(rate) < 1e-12 * S.integral(np.abs(G))
    # and the printed stretching sign breaks it
    bad = sf.f_explicit_grid(S, u, g, p) - 4.0 * S.K * G * np.sum(U["f"] * S.n, axis=0)
    assert abs(S.integral(bad + G * S.div(U["t"], U["p"]))) > 1e-4


def test_implicit_solve_preconditioned_exactly_on_a_sphere_and_equal_to_a_dense_solve():
    p, R, a = 6, 0.9, 0.05
    rng = np.random.default_rng(12)
    b = inputs.random_bandlimited(rng, p, 1)[0]
    sphere = inputs.sphere_coef(p, radius=R, centre=(0.5, 0.0, 0.1))
    y, it = sf.solve_implicit(sphere, b, p, a)
    nn = sf.degrees(p)
    assert it <= 1
    assert np.max(np.abs(y - b / (1.0 + a * nn * (nn + 1) / R ** 2))) < 1e-14
    x, _ = _deformed(p, 13)
    S = sf.Surface(x, p, sf.grid_degree(p))
    ncf = (p + 1) ** 2
    A = np.stack([e - a * sf.lap_coef(S, e, p) for e in np.eye(ncf)], axis=1)
    ref = np.linalg.solve(A, b)
    y1, it1 = sf.solve_implicit(x, b, p, a)
    y0, it0 = sf.solve_implicit(x, b, p, a, precondition=False)
    assert np.max(np.abs(y1 - ref)) < 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(y0 - ref)) < 1e-12 * np.max(np.abs(ref))
    assert it1 < it0


def test_imex2_step_of_pure_diffusion_on_a_resting_sphere():
    # Sec. 5, diffusion test.  With u = 0 the scheme is, per SH mode, the rational factor
    # (1 - a)/(1 + a), a = dt n(n+1)/(2 Pe R^2): the exact closed form of the IMEX-2 step, which
    # matches exp(-2a) to second order and decays every mode n > 0.
    p, R, pe, dt = 6, 1.1, 5.0, 0.2
    x = inputs.sphere_coef(p, radius=R)
    rng = np.random.default_rng(14)
    g = _gamma(p, rng)
    zero = np.zeros((3, (p + 1) ** 2))
    gh, g1, k0 = sf.imex2(x, zero, x, zero, g, p, pe, dt)
    nn = sf.degrees(p)
    a = dt * nn * (nn + 1) / (2.0 * pe * R * R)
    assert np.max(np.abs(k0)) < 1e-13
    assert np.max(np.abs(gh - g / (1 + a))) < 1e-13
    assert np.max(np.abs(g1 - g * (1 - a) / (1 + a))) < 1e-13


def _radial(c, centre):
    centre = np.asarray(centre, dtype=np.float64)

    def vel(xs, gs):
        out = []
        for x in xs:
            p = int(round(math.sqrt(x.shape[1]))) - 1
            out.append(_field_coef(x, p, lambda X: c * (X - centre[:, None, None])
                                   / np.linalg.norm(X - centre[:, None, None], axis=0)))
        return out
    return vel


def test_expanding_sphere_keeps_gamma_r_squared_to_second_order():
    # Sec. 5: uniform expansion R(t) = R0 + c t at infinite Peclet number gives Gamma R^2 = Gamma(0).
    p, R0, c, T = 4, 1.0, 0.5, 0.8
    x = inputs.sphere_coef(p, radius=R0)
    g = np.zeros((p + 1) ** 2)
    g[0] = math.sqrt(4 * math.pi)
    errs = []
    for nsteps in (4, 8):
        xs, gs = [x], [g]
        for _ in range(nsteps):
            st = sf.coupled_step(xs, gs, [p], T / nsteps, _radial(c, (0, 0, 0)), math.inf)
            xs, gs = st["x"], st["gamma"]
        R = geometry.mean_radius(xs[0], p)
        assert abs(R - (R0 + c * T)) < 1e-12   # the midpoint rule moves the sphere exactly
        G = gs[0][0] / math.sqrt(4 * math.pi)
        assert np.max(np.abs(gs[0][1:])) < 1e-13
        errs.append(abs(G * R * R - 1.0))
    assert errs[1] < 2e-3
    assert 3.5 < errs[0] / errs[1] < 4.5


def _shear_like(xs, gs):
    out = []
    for x in xs:
        p = int(round(math.sqrt(x.shape[1]))) - 1
        out.append(_field_coef(x, p, lambda X: np.stack([0.6 * X[2] + 0.2 * X[0] * X[1], -0.3 * X[1] + 0.1 * X[2] ** 2,
                                                          0.3 * X[2] - 0.2 * X[0] ** 2])))
    return out


def test_surfactant_mass_is_conserved_to_third_order_per_step():
    # The conservation error of Eq. err_conservation is a local error: O(dt^3) per step for the
    # second-order midpoint / IMEX-2 pair, so halving dt divides it by about 8.
    p, pe = 8, 4.0
    x, rng = _deformed(p, 21, amp=0.03)
    g = _gamma(p, rng)
    errs = []
    for dt in (0.08, 0.04):
        st = sf.coupled_step([x], [g], [p], dt, _shear_like, pe)
        errs.append(st["err_conservation"])
    assert errs[1] < 1e-5
    assert 6.0 < errs[0] / errs[1] < 10.0


def test_adaptive_run_keeps_every_accepted_step_below_tolerance():
    p, pe, tol, T = 6, 4.0, 1e-5, 0.3
    x, rng = _deformed(p, 22, amp=0.03)
    g = _gamma(p, rng)
    res = sf.run_adaptive([x], [g], [p], T, 0.2, tol, _shear_like, pe, dt_max=0.1)
    acc = [h for h in res["history"] if h["accepted"]]
    assert abs(res["t"] - T) < 1e-14
    assert all(h["err"] < tol for h in acc)
    assert any(not h["accepted"] for h in res["history"])   # the first dt = 0.1 is too long
    # the step-size rule of Alg. 1
    assert sf.next_dt(0.1, 4e-5, 1e-5, 1.0) == pytest.approx(0.1 * math.sqrt(0.9 / 4.0))
    assert sf.next_dt(0.1, 1e-9, 1e-5, 0.15) == 0.15


def test_clean_sphere_at_rest_with_uniform_surfactant_stays_put_through_the_stokes_step():
    p = 5
    x = inputs.sphere_coef(p, radius=0.9, centre=(0.3, -0.2, 0.1))
    g = np.zeros((p + 1) ** 2)
    g[0] = math.sqrt(4 * math.pi)

    def stokes(xs, gs):
        return timestep.velocity(xs, [p], [p], [3.0], gs, 0.2, 0.0, 0.0)

    st = sf.coupled_step([x], [g], [p], 0.1, stokes, 10.0)
    assert np.max(np.abs(st["x"][0] - x)) < 1e-12
    assert np.max(np.abs(st["gamma"][0] - g)) < 1e-12


def test_stokes_coupled_step_conserves_mass_and_volume_to_third_order():
    # A drop in shear with non-uniform surfactant (Marangoni stresses active): surfactant mass and
    # drop volume change by O(dt^3) per step.
    p, pe = 5, 10.0
    rng = np.random.default_rng(23)
    x = inputs.sphere_coef(p, axes=(1.1, 0.95, 0.95)) + inputs.perturbation(rng, p, 2, 4, 0.02)
    g = _gamma(p, rng, base=1.0)

    def stokes(xs, gs):
        return timestep.velocity(xs, [p], [p], [2.0], gs, 0.3, 0.0, 1.0)

    v0 = geometry.volume(x, p, 2 * p + 1)
    em, ev = [], []
    for dt in (0.1, 0.05):
        st = sf.coupled_step([x], [g], [p], dt, stokes, pe)
        em.append(st["err_conservation"])
        ev.append(abs(geometry.volume(st["x"][0], p, 2 * p + 1) - v0) / v0)
    assert 6.0 < em[0] / em[1] < 10.0
    assert 6.0 < ev[0] / ev[1] < 10.0
