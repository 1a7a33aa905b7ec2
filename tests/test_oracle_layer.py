"""Pins of the oracle's layer operators: Thm 1 on the Laplace kernel, closed forms of the Stokes
single and double layer (Eq. main_eq), brute-force quadrature, the regular and near-singular
rules at exterior points (Sec. 2.3), GMRES and the solve invariants."""
import math

import numpy as np
import pytest

from oracle import brute, geometry, gmres, layer, sh, wigner
from paper_1707_02156_gb300 import inputs


def _rand_drop(p, seed, amp=0.1, nmax=4):
    rng = np.random.default_rng(seed)
    return inputs.sphere_coef(p) + inputs.perturbation(rng, p, 1, nmax, amp), rng


def test_singular_rule_is_exact_for_laplace_on_unit_sphere():
    # Thm 1 / Funk-Hecke: int Y_n^m(s) / |s0 - s| dS = 4 pi/(2n+1) Y_n^m(s0) for n <= p_q.
    p = pq = 7
    _, _, theta, phi = sh.gauss_grid(p)
    _, _, thq, phq = sh.gauss_grid(pq)
    ws = layer.singular_weights(pq)
    P = sh.legendre_normalised(p, np.cos(thq))
    dist = 2.0 * np.sin(thq / 2.0)
    for n, m in ((0, 0), (2, 1), (5, 3), (7, 7)):
        f = np.zeros((p + 1) ** 2)
        f[n * (n + 1) + m] = 0.7
        f[n * (n + 1) - m] = -0.4 if m else 0.0
        for a, b in ((1, 0), (4, 9)):
            c = layer.rotate_batch(f[None], p, np.array([phi[b]]), theta[a])[0, 0]
            vals = layer.synth_complex(c, p, P, phq)
            Q = np.sum(ws[:, None] * vals / dist[:, None])  # J = 1 on the unit sphere
            exact = 4 * math.pi / (2 * n + 1) * sh.evaluate(f, p, np.array([theta[a]]), np.array([phi[b]]))[0]
            assert abs(Q - exact) < 1e-13


def test_single_layer_of_constant_on_sphere_radius_a():
    # S[c] = (2a/3) c on a sphere of radius a (mu = 1).
    p, a = 8, 1.6
    x = inputs.sphere_coef(p, radius=a, centre=(0.3, 0.1, -0.2))
    q = layer.SelfQuadrature(x, p, p)
    cvec = np.array([0.3, -0.7, 1.1])
    c = np.zeros((3, (p + 1) ** 2))
    c[:, 0] = cvec * math.sqrt(4 * math.pi)
    S = q.apply(c, "S") / (8 * math.pi)
    assert np.max(np.abs(S - (2 * a / 3) * cvec[:, None, None])) < 1e-14


def test_single_layer_of_normal_vanishes_and_double_layer_identity_on_deformed_drop():
    p = 8
    x, _ = _rand_drop(p, 21)
    q = layer.SelfQuadrature(x, p, 4 * (p + 1) - 1)
    g = geometry.forms(geometry.surface_fields(x, p, 4 * (p + 1) - 1))
    ncoef = np.stack([sh.analyze(g["n"][c], 4 * (p + 1) - 1, p) for c in range(3)])
    # the normal is not band-limited: use its degree-p truncation; S[n] = 0 holds to truncation error
    S = q.apply(ncoef, "S", lats=[0, 4]) / (8 * math.pi)
    assert np.max(np.abs(S[:, [0, 4]])) < 2e-3
    cvec = np.array([1.0, -2.0, 0.5])
    c = np.zeros((3, (p + 1) ** 2))
    c[:, 0] = cvec * math.sqrt(4 * math.pi)
    D = q.apply(c, "D") / (4 * math.pi)
    assert np.max(np.abs(D - cvec[:, None, None])) < 1e-10


@pytest.mark.parametrize("n", [1, 2, 4])
def test_toroidal_harmonics_are_eigenfunctions_of_single_layer(n):
    # r x grad_s Y_n is an eigenfunction of S on the unit sphere with eigenvalue 1/(2n+1).
    p = 6
    x = inputs.sphere_coef(p)
    _, _, theta, phi = sh.gauss_grid(p)
    T, F = np.meshgrid(theta, phi, indexing="ij")
    Y = np.zeros((p + 1) ** 2)
    Y[n * (n + 1) + min(n, 1)] = 1.0
    d = sh.evaluate_derivs(Y, p, T, F)
    th_hat = np.stack([np.cos(T) * np.cos(F), np.cos(T) * np.sin(F), -np.sin(T)])
    ph_hat = np.stack([-np.sin(F), np.cos(F), np.zeros_like(F)])
    X = ph_hat * d["t"] - th_hat * d["p"] / np.sin(T)
    Xc = np.stack([sh.analyze(X[c], p, p) for c in range(3)])
    q = layer.SelfQuadrature(x, p, p)
    S = q.apply(Xc, "S") / (8 * math.pi)
    assert np.max(np.abs(S - X / (2 * n + 1))) < 1e-13


@pytest.mark.parametrize("kind", ["S", "D"])
def test_singular_rule_converges_to_brute_force(kind):
    p = 8
    x, rng = _rand_drop(p, 31)
    f = inputs.random_bandlimited(rng, p, 3)
    _, _, theta, phi = sh.gauss_grid(p)
    a, b = 2, 11
    ref = brute.self_integral(x, p, f, theta[a], phi[b], kind)
    errs = []
    for pq in (p, 2 * (p + 1) - 1, 4 * (p + 1) - 1):
        v = layer.SelfQuadrature(x, p, pq).apply(f, kind, lats=[a])[:, a, b]
        errs.append(np.max(np.abs(v - ref)) / np.max(np.abs(ref)))
    assert errs[0] < 1e-2 and errs[1] < 1e-6 and errs[2] < 1e-12
    assert errs[2] < errs[1] < errs[0]


def _translating_sphere(xt, centre, a, cvec):
    xh = xt - np.asarray(centre)[:, None]
    r = np.linalg.norm(xh, axis=0)
    xc = np.sum(xh * cvec[:, None], axis=0)
    G = cvec[:, None] / r + xh * xc / r ** 3
    dip = cvec[:, None] / r ** 3 - 3 * xh * xc / r ** 5
    return 0.5 * a * a * (G + a * a / 3.0 * dip)


def test_single_layer_is_self_adjoint_on_a_deformed_drop():
    # int g . S[f] dS = int f . S[g] dS (the Stokeslet is symmetric): on a deformed drop (shape and
    # densities band-limited at degree 4) the singular rule plus the regular outer rule converge to
    # that symmetry spectrally as the grid degree grows
    rng = np.random.default_rng(31)
    x0 = inputs.sphere_coef(4) + inputs.perturbation(rng, 4, 1, 4, 0.1)
    f0, g0 = inputs.random_bandlimited(rng, 4, 3), inputs.random_bandlimited(rng, 4, 3)
    asym = []
    for p in (8, 16):
        x, f, g = (np.pad(c, ((0, 0), (0, (p + 1) ** 2 - 25))) for c in (x0, f0, g0))
        G = geometry.forms(geometry.surface_fields(x, p, p))
        _, w, theta, _ = sh.gauss_grid(p)
        wq = (np.pi / (p + 1)) * w[:, None] * geometry.area_density(G["W"], theta)
        fg = np.stack([sh.synthesize(f[c], p, p) for c in range(3)])
        gg = np.stack([sh.synthesize(g[c], p, p) for c in range(3)])
        q = layer.SelfQuadrature(x, p, 2 * (p + 1) - 1)
        a = np.sum(np.sum(gg * q.apply(f, "S"), axis=0) * wq)
        b = np.sum(np.sum(fg * q.apply(g, "S"), axis=0) * wq)
        asym.append(abs(a - b) / abs(a))
    assert asym[1] < 1e-11 and asym[1] < 1e-3 * asym[0], asym


def test_regular_rule_reproduces_translating_sphere_field_far_away():
    p, a = 10, 0.9
    x = inputs.sphere_coef(p, radius=a, centre=(0.0, 0.0, 0.0))
    cvec = np.array([0.2, 1.0, -0.4])
    c = np.zeros((3, (p + 1) ** 2))
    c[:, 0] = cvec * math.sqrt(4 * math.pi)
    src = layer.DropGrid(x, p, p)
    rng = np.random.default_rng(1)
    dirs = rng.standard_normal((3, 20))
    dirs /= np.linalg.norm(dirs, axis=0)
    pts = dirs * rng.uniform(3.0, 6.0, 20)
    S = layer.regular_sum(pts, src, src.density(c), "S") / (8 * math.pi)
    assert np.max(np.abs(S - _translating_sphere(pts, (0, 0, 0), a, cvec))) < 1e-12
    D = layer.regular_sum(pts, src, src.density(c), "D") / (4 * math.pi)
    assert np.max(np.abs(D)) < 1e-10


def test_two_drops_near_contact_closed_forms_through_all_regions():
    # Uniform traction on each of two spheres at gap 0.05: every target of drop 0 sees drop 1's
    # translating-sphere field (regions 0, 1 and 2 all occur); the double layer of a constant
    # vanishes outside its drop.
    p = 10
    w = inputs.two_drops(p=p, gap=0.05, up=4)
    xs = [w.xcoef[:3 * (p + 1) ** 2].reshape(3, -1), w.xcoef[3 * (p + 1) ** 2:].reshape(3, -1)]
    drops = layer.Drops(xs, [p, p], [p, p], [1.0, 1.0], up=4)
    reg = drops.region[(0, 1)]
    assert set(np.unique(reg)) == {0, 1, 2}
    cvec = [np.array([0.0, 0.3, 1.0]), np.array([0.5, 0.0, -0.2])]
    dens = []
    for cv in cvec:
        c = np.zeros((3, (p + 1) ** 2))
        c[:, 0] = cv * math.sqrt(4 * math.pi)
        dens.append(c)
    S = drops.apply_single_grid(dens, raw=True)[0].reshape(3, -1)
    exact = (2.0 / 3.0) * cvec[0][:, None] + _translating_sphere(drops.targets[0], (0, 0, -1.025), 1.0, cvec[1])
    err = np.abs(S - exact)
    # regular rule at d > 5h, upsampled rule at h < d <= 5h, interpolation at d <= h
    assert np.max(err[:, reg == 0]) < 1e-9
    assert np.max(err[:, reg == 1]) < 1e-12
    assert np.max(err[:, reg == 2]) < 1e-4
    D = drops.apply_double_grid(dens, raw=True)[0].reshape(3, -1)
    derr = np.abs(D - cvec[0][:, None])
    assert np.max(derr[:, reg == 0]) < 1e-7
    assert np.max(derr[:, reg == 1]) < 1e-12
    assert np.max(derr[:, reg == 2]) < 1e-6


def test_newton_closest_point_is_the_nearest_surface_point():
    # Sec. 2.3: x* minimises |x(theta, phi) - x0| over the source surface.  At x* the offset x0 - x*
    # is orthogonal to both tangents, and no point of the surface is closer (checked against 10^4
    # random surface samples by direct SH evaluation).  Targets sit 0.05 off a deformed drop, some
    # of them next to a parameter pole.
    from oracle import near
    p = 8
    x, rng = _rand_drop(p, 61, amp=0.12)
    _, _, theta, phi = sh.gauss_grid(p)
    T, F = np.meshgrid(theta, phi, indexing="ij")
    T, F = T.reshape(-1), F.reshape(-1)
    std_x = np.stack([sh.synthesize(x[c], p, p).reshape(-1) for c in range(3)])
    ts = np.arccos(rng.uniform(-1.0, 1.0, 10000))
    fs = rng.uniform(0.0, 2 * np.pi, 10000)
    samples = np.stack([sh.evaluate(x[c], p, ts, fs) for c in range(3)])
    for th0, ph0 in ((0.03, 1.0), (1.1, 0.4), (2.0, 4.0), (3.1, 2.5)):
        d = [sh.evaluate_derivs(x[c], p, np.array([th0]), np.array([ph0])) for c in range(3)]
        xs0 = np.array([d[c]["f"][0] for c in range(3)])
        nrm = np.cross([d[c]["t"][0] for c in range(3)], [d[c]["p"][0] for c in range(3)])
        x0 = xs0 + 0.05 * nrm / np.linalg.norm(nrm) + 0.02 * np.array([0.3, -0.2, 0.1])
        s = int(np.argmin(np.sum((std_x - x0[:, None]) ** 2, axis=0)))
        al, be = F[s], T[s] - np.pi / 2
        xr = np.stack([wigner.rotate(x[c], p, al, be) for c in range(3)])
        th, ph, xstar = near.newton_closest(xr, p, x0)
        dr = [sh.evaluate_derivs(xr[c], p, np.array([th]), np.array([ph])) for c in range(3)]
        xt = np.array([dr[c]["t"][0] for c in range(3)])
        xp = np.array([dr[c]["p"][0] for c in range(3)])
        off = x0 - xstar
        assert abs(off @ xt) < 1e-13 * np.linalg.norm(xt) and abs(off @ xp) < 1e-13 * np.linalg.norm(xp)
        assert np.linalg.norm(off) <= np.min(np.linalg.norm(samples - x0[:, None], axis=0)) + 1e-15
        assert np.linalg.norm(off) <= np.min(np.linalg.norm(std_x - x0[:, None], axis=0))


def test_brute_force_exterior_integral_reproduces_the_translating_sphere_field():
    # the reference used below, checked first: a uniform traction c on a sphere of radius a gives
    # the translating-sphere field at every exterior point, here 0.05 off the surface
    p, a = 6, 0.9
    x = inputs.sphere_coef(p, radius=a, centre=(0.1, -0.2, 0.3))
    cvec = np.array([0.4, -1.0, 0.7])
    c = np.zeros((3, (p + 1) ** 2))
    c[:, 0] = cvec * math.sqrt(4 * math.pi)
    for d in (np.array([1.0, 2.0, -0.5]), np.array([0.0, 0.0, 1.0])):
        pt = np.array([0.1, -0.2, 0.3]) + (a + 0.05) * d / np.linalg.norm(d)
        S = brute.exterior_integral(x, p, c, pt, "S") / (8 * math.pi)
        exact = _translating_sphere(pt[:, None], (0.1, -0.2, 0.3), a, cvec)[:, 0]
        assert np.max(np.abs(S - exact)) < 1e-11
        D = brute.exterior_integral(x, p, c, pt, "D") / (4 * math.pi)
        assert np.max(np.abs(D)) < 1e-11


def test_regular_and_upsampled_rules_converge_to_brute_force_on_a_deformed_drop():
    # Sec. 2.1 / 2.3 away from the surface, on a deformed drop: targets 0.35, 0.6 and 1.5 off the
    # surface fall in Omega_1 (upsampled rule) or Omega_0 (regular rule); both converge spectrally
    # in p to the brute-force integral (shape and density band-limited at degree 4)
    rng = np.random.default_rng(7)
    xj = inputs.sphere_coef(4) + inputs.perturbation(rng, 4, 1, 4, 0.06)
    dens = inputs.random_bandlimited(rng, 4, 3)
    pts = []
    for t0, f0, dist in ((1.0, 0.5, 0.6), (2.0, 2.5, 0.35), (0.6, 4.0, 1.5)):
        d = [sh.evaluate_derivs(xj[c], 4, np.array([t0]), np.array([f0])) for c in range(3)]
        n = np.cross([d[c]["t"][0] for c in range(3)], [d[c]["p"][0] for c in range(3)])
        pts.append(np.array([d[c]["f"][0] for c in range(3)]) + dist * n / np.linalg.norm(n))
    pts = np.array(pts).T
    for kind in ("S", "D"):
        ref = np.stack([brute.exterior_integral(xj, 4, dens, pts[:, i], kind) for i in range(3)], axis=1)
        errs = []
        for p in (8, 16):
            xp = np.zeros((3, (p + 1) ** 2))
            xp[:, :25] = xj
            dp = np.zeros((3, (p + 1) ** 2))
            dp[:, :25] = dens
            drops = layer.Drops([inputs.sphere_coef(p, radius=0.3, centre=(10.0, 0.0, 0.0)), xp], [p, p], [p, p],
                                [1.0, 1.0], up=4)
            reg = drops.classify(pts, 1)
            assert np.all(reg < 2)
            v = np.stack([layer.regular_sum(pts[:, i:i + 1], *((drops.std[1], drops.std[1].density(dp)) if reg[i] == 0
                                                              else (drops.ups[1], drops.ups[1].density(dp))), kind)[:, 0]
                          for i in range(3)], axis=1)
            errs.append(np.max(np.abs(v - ref)) / np.max(np.abs(ref)))
        assert errs[1] < 1e-12 and errs[1] < 1e-2 * errs[0], (kind, errs)


def test_near_singular_values_converge_to_brute_force_on_a_deformed_drop():
    # Sec. 2.3 on a deformed drop (no closed form): targets 0.05 off the surface, in Omega_2 for
    # every degree used.  Shape and density are band-limited at degree 4, so the exact integrals
    # (brute force) are the same at every p while the rule's resolution h = R pi/(p+1) shrinks; the
    # error of the interpolation must fall with p (about fifth order here).
    from oracle import near
    rng = np.random.default_rng(7)
    xj = inputs.sphere_coef(4) + inputs.perturbation(rng, 4, 1, 4, 0.06)
    dens = inputs.random_bandlimited(rng, 4, 3)
    pts = []
    for t0, f0 in ((1.0, 0.5), (2.0, 2.5), (0.6, 4.0)):
        d = [sh.evaluate_derivs(xj[c], 4, np.array([t0]), np.array([f0])) for c in range(3)]
        n = np.cross([d[c]["t"][0] for c in range(3)], [d[c]["p"][0] for c in range(3)])
        pts.append(np.array([d[c]["f"][0] for c in range(3)]) + 0.05 * n / np.linalg.norm(n))
    pts = np.array(pts).T
    for kind in ("S", "D"):
        ref = np.stack([brute.exterior_integral(xj, 4, dens, pts[:, i], kind) for i in range(pts.shape[1])], axis=1)
        errs = []
        for p in (8, 12, 16):
            xp = np.zeros((3, (p + 1) ** 2))
            xp[:, :25] = xj
            dp = np.zeros((3, (p + 1) ** 2))
            dp[:, :25] = dens
            far = inputs.sphere_coef(p, radius=0.3, centre=(10.0, 0.0, 0.0))
            drops = layer.Drops([far, xp], [p, p], [p, p], [1.0, 1.0], up=4)
            drops.targets[0] = pts
            assert np.all(drops.classify(pts, 1) == 2)
            v = near.near_values(drops, 0, 1, list(range(pts.shape[1])), dp, kind, drops.selfq[1].apply(dp, kind))
            errs.append(np.max(np.abs(v - ref)) / np.max(np.abs(ref)))
        assert errs[2] < errs[1] < errs[0], (kind, errs)
        assert errs[0] / errs[2] > 10 and errs[2] < 1e-3, (kind, errs)


def test_gmres_matches_direct_solve():
    rng = np.random.default_rng(0)
    n = 60
    A = np.eye(n) * 3 + rng.standard_normal((n, n)) / math.sqrt(n)
    b = rng.standard_normal(n)
    x, info = gmres.gmres(lambda v: A @ v, b, tol=1e-13, restart=12, max_it=300)
    assert info["converged"]
    assert np.max(np.abs(x - np.linalg.solve(A, b))) < 1e-11


def test_gmres_iterate_minimises_the_residual_over_the_krylov_space():
    # GMRES's defining property: after k steps from x = 0, x_k minimises ||b - A x|| over
    # span{b, A b, ..., A^(k-1) b}; here the minimum is found by least squares on an orthonormal
    # basis of that space (QR of the Krylov matrix), and the running estimates equal it.
    rng = np.random.default_rng(5)
    n = 40
    A = np.eye(n) * 2 + rng.standard_normal((n, n)) / math.sqrt(n)
    b = rng.standard_normal(n)
    for k in (3, 6, 10):
        K = np.zeros((n, k))
        v = b.copy()
        for j in range(k):
            K[:, j] = v
            v = A @ v
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
        best = np.linalg.norm(b - A @ (Q @ y)) / np.linalg.norm(b)
        x, info = gmres.gmres(lambda v: A @ v, b, tol=1e-15, restart=n, max_it=k)
        assert info["iterations"] == k
        assert abs(np.linalg.norm(b - A @ x) / np.linalg.norm(b) - best) < 1e-12
        assert abs(info["residuals"][-2] - best) < 1e-12   # the last Givens estimate


def test_solution_of_rigid_rotation_is_the_flow_for_any_viscosity_ratio():
    # u_inf = Omega x x, f = 0: rigid motions satisfy D[u] = u on the surface, so u = u_inf.
    p = 6
    x, _ = _rand_drop(p, 41, amp=0.08)
    drops = layer.Drops([x], [p], [2 * (p + 1) - 1], [3.0])
    g = geometry.forms(geometry.surface_fields(x, p, p))
    Om = np.array([0.2, -0.5, 1.0])
    uinf = np.cross(Om[:, None, None], g["x"], axis=0)
    b = 2.0 * np.concatenate([sh.analyze(uinf[c], p, p) for c in range(3)])
    u, info = gmres.gmres(drops.system_matvec, b, tol=1e-12)
    assert info["converged"]
    assert np.max(np.abs(u - b / 2.0)) < 1e-8


def test_force_free_drop_of_matched_viscosity_is_invisible():
    # A drop with the suspending fluid's viscosity (lambda = 1) and no interfacial force is not
    # there.  Alone, it moves with the undisturbed shear u_inf = (z, 0, 0).  Next to another drop it
    # leaves that drop's velocity as it is alone (the double layer of each source drop carries its
    # own lambda_j - 1, Eq. main_eq).
    p = 4
    x0, _ = _rand_drop(p, 51, amp=0.08)
    zero = np.zeros((3, (p + 1) ** 2))
    alone = layer.Drops([x0], [p], [p], [1.0])
    u, info = gmres.gmres(alone.system_matvec, alone.rhs([zero], shear=1.0), tol=1e-13)
    assert info["converged"]
    xg = geometry.surface_fields(x0, p, p)["f"]
    uinf = np.zeros((3, (p + 1) ** 2))
    uinf[0] = sh.analyze(xg[2], p, p)
    assert np.max(np.abs(u.reshape(3, -1) - uinf)) < 1e-13

    x1 = inputs.sphere_coef(p, radius=0.8, centre=(2.9, 0.0, 0.3))
    gam = np.zeros((p + 1) ** 2)
    gam[0] = math.sqrt(4 * math.pi)
    f0 = geometry.interfacial_force(x0, p, gam, elasticity=0.2)
    single = layer.Drops([x0], [p], [p], [3.0])
    u_single, info = gmres.gmres(single.system_matvec, single.rhs([f0], shear=1.0), tol=1e-13)
    assert info["converged"]
    pair = layer.Drops([x0, x1], [p, p], [p, p], [3.0, 1.0], up=2)
    u_pair, info = gmres.gmres(pair.system_matvec, pair.rhs([f0, zero], shear=1.0), tol=1e-13)
    assert info["converged"]
    u0 = pair.split(u_pair)[0].reshape(-1)
    assert np.max(np.abs(u0 - u_single)) < 1e-11 * np.max(np.abs(u_single))
    # drop 1 itself moves with the flow that drop 0 disturbs, not with u_inf
    x1g = geometry.surface_fields(x1, p, p)["f"]
    uinf1 = np.zeros((3, (p + 1) ** 2))
    uinf1[0] = sh.analyze(x1g[2], p, p)
    assert np.max(np.abs(pair.split(u_pair)[1] - uinf1)) > 1e-3


def test_volume_conservation_and_relaxation_sign_of_clean_prolate_drop():
    # Clean prolate spheroid at rest in quiescent fluid, lambda = 1: int u.n = 0 and the tips move in.
    p = 8
    x = inputs.sphere_coef(p, axes=(0.8, 0.8, 1.5))
    gam = np.zeros((p + 1) ** 2)
    gam[0] = math.sqrt(4 * math.pi)
    f = geometry.interfacial_force(x, p, gam, elasticity=0.0)
    drops = layer.Drops([x], [p], [2 * (p + 1) - 1], [1.0])
    u = drops.rhs([f], shear=0.0) / 2.0
    ug = np.stack([sh.synthesize(u.reshape(3, -1)[c], p, p) for c in range(3)])
    t, w, theta, phi = sh.gauss_grid(p)
    g = geometry.forms(geometry.surface_fields(x, p, p))
    un = np.sum(ug * g["n"], axis=0)
    J = geometry.area_density(g["W"], theta)
    flux = (np.pi / (p + 1)) * np.sum(w[:, None] * un * J)
    assert abs(flux) < 1e-5   # quadrature and truncation error at p = 8
    assert un[0, 0] < 0 and un[-1, 0] < 0        # latitudes nearest the poles (tips) move inward
    j_eq = np.argmin(np.abs(theta - np.pi / 2))
    assert un[j_eq, 0] > 0                         # the equator moves outward


def test_marangoni_flow_moves_surface_towards_high_tension():
    p = 6
    x = inputs.sphere_coef(p)
    gam = np.zeros((p + 1) ** 2)
    gam[0] = math.sqrt(4 * math.pi)
    gam[2] = math.sqrt(4 * math.pi / 3.0)
    f = geometry.interfacial_force(x, p, gam, elasticity=-0.1)   # sigma = 1 + 0.1 (1 + z)
    drops = layer.Drops([x], [p], [p], [1.0])
    u = (drops.rhs([f], shear=0.0) / 2.0).reshape(3, -1)
    ug = np.stack([sh.synthesize(u[c], p, p) for c in range(3)])
    _, _, theta, _ = sh.gauss_grid(p)
    j_eq = np.argmin(np.abs(theta - np.pi / 2))
    assert np.all(ug[2, j_eq] > 0)
