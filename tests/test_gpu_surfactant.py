"""GPU parity of the surfactant transport (Eq. surfactant0, Sec. 3, Alg. 1) with the oracle: the
explicit and diffusion rates, the preconditioned implicit solve, the surfactant mass, one coupled
step of Alg. 1 (FP64 and mixed velocity solves) and an adaptive run.

Tolerances: the rates and the mass are FP64 arithmetic on both sides (1e-12 norm-wise); the
implicit solves stop at relative residual 1e-13 on both sides, with a preconditioned operator of
condition number O(1), so the two solutions agree to about 1e-12 (1e-11 allowed); the coupled
step follows the midpoint-step parity (displacement 1e-10 with FP64 solves at tol 1e-12, 1e-7
with mixed solves at 1e-10)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sh, surfactant as sf, timestep
from paper_1707_02156_gb300 import inputs

pytestmark = pytest.mark.gpu


def _relerr(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _gamma(p, rng, base=1.0, amp=0.2):
    g = amp * inputs.random_bandlimited(rng, p, 1)[0]
    g[0] += base * math.sqrt(4 * math.pi)
    return g


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02156_gb300 import api
    c = api.Context(0, upsample=4)
    yield c
    c.close()


def _cuda(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


def _three_drops(seed):
    # degrees 6, 9, 6: two degree groups, the drops of one group not adjacent in memory
    rng = np.random.default_rng(seed)
    ps = [6, 9, 6]
    xs = [inputs.sphere_coef(p, centre=(3.0 * i, 0.0, 0.0), axes=(0.8, 1.0, 1.2), rot=inputs.random_rotation(rng))
          + inputs.perturbation(rng, p, 1, 5, 0.05) for i, p in enumerate(ps)]
    us = [0.5 * inputs.random_bandlimited(rng, p, 3) for p in ps]
    gs = [_gamma(p, rng) for p in ps]
    return ps, xs, us, gs, rng


def test_rates_match_oracle(ctx):
    from paper_1707_02156_gb300 import api
    ps, xs, us, gs, _ = _three_drops(1)
    inv_pe = 0.25
    x, u, g = _cuda(inputs.pack_drops(xs)), _cuda(inputs.pack_drops(us)), _cuda(np.concatenate(gs))
    fe, fi = torch.zeros_like(g), torch.zeros_like(g)
    api.surfactant_rates(ctx, ps, x, u, g, inv_pe, fe, fi)
    ref_e = np.concatenate([sf.f_explicit(a, b, c, p) for a, b, c, p in zip(xs, us, gs, ps)])
    ref_i = np.concatenate([sf.f_implicit(a, c, p, 1.0 / inv_pe) for a, c, p in zip(xs, gs, ps)])
    assert _relerr(fe.cpu().numpy(), ref_e) < 1e-12
    assert _relerr(fi.cpu().numpy(), ref_i) < 1e-12
    fe2 = torch.zeros_like(g)
    api.surfactant_rates(ctx, ps, x, u, g, 0.0, fe2, None)
    assert torch.equal(fe2, fe)


def test_rigid_rotation_rate_vanishes_on_the_gpu(ctx):
    # the rotating-drop test of Sec. 5 on the device path: f_E = 0 for u = Omega x x + V
    from paper_1707_02156_gb300 import api
    ps, xs, _, gs, _ = _three_drops(2)
    Om, V = np.array([0.4, -0.1, 0.8]), np.array([0.2, 0.0, -0.5])
    us = []
    for x, p in zip(xs, ps):
        q = sf.Surface(x, p, sf.grid_degree(p))
        U = np.cross(Om[:, None, None], q.x, axis=0) + V[:, None, None]
        us.append(np.stack([sh.analyze(U[c], q.P, p) for c in range(3)]))
    x, u, g = _cuda(inputs.pack_drops(xs)), _cuda(inputs.pack_drops(us)), _cuda(np.concatenate(gs))
    fe = torch.zeros_like(g)
    api.surfactant_rates(ctx, ps, x, u, g, 0.0, fe, None)
    assert float(fe.abs().max()) < 1e-12


def test_implicit_solve_matches_oracle(ctx):
    from paper_1707_02156_gb300 import api
    ps, xs, _, _, rng = _three_drops(3)
    a = 0.03
    bs = [inputs.random_bandlimited(rng, p, 1)[0] for p in ps]
    x, b = _cuda(inputs.pack_drops(xs)), _cuda(np.concatenate(bs))
    y = torch.zeros_like(b)
    it = api.surfactant_implicit(ctx, ps, x, b, a, y)
    ref = np.concatenate([sf.solve_implicit(xx, bb, p, a)[0] for xx, bb, p in zip(xs, bs, ps)])
    assert _relerr(y.cpu().numpy(), ref) < 1e-11
    assert 1 <= it <= 60
    # on a sphere the preconditioner is the operator: one iteration, the closed form per degree
    p, R = 6, 0.9
    xsph = _cuda(inputs.sphere_coef(p, radius=R, centre=(0.5, 0.0, 0.1)))
    bsph = _cuda(bs[0])
    ysph = torch.zeros_like(bsph)
    it = api.surfactant_implicit(ctx, [p], xsph, bsph, a, ysph)
    nn = sf.degrees(p)
    assert it <= 1
    assert np.max(np.abs(ysph.cpu().numpy() - bs[0] / (1.0 + a * nn * (nn + 1) / R ** 2))) < 1e-13
    # a = 0 copies the right-hand side
    y0 = torch.zeros_like(b)
    assert api.surfactant_implicit(ctx, ps, x, b, 0.0, y0) == 0
    assert torch.equal(y0, b)


def test_mass_matches_oracle(ctx):
    from paper_1707_02156_gb300 import api
    ps, xs, _, gs, _ = _three_drops(4)
    m = api.surfactant_mass(ctx, ps, _cuda(inputs.pack_drops(xs)), _cuda(np.concatenate(gs)))
    ref = [sf.mass(x, g, p) for x, g, p in zip(xs, gs, ps)]
    assert np.max(np.abs(np.array(m) - ref) / np.abs(ref)) < 1e-13


def _pair(seed):
    rng = np.random.default_rng(seed)
    ps = [5, 6]
    xs = [inputs.sphere_coef(5, axes=(1.1, 0.95, 1.0), rot=inputs.random_rotation(rng)) +
          inputs.perturbation(rng, 5, 2, 4, 0.02),
          inputs.sphere_coef(6, centre=(2.4, 0.3, 0.2), radius=0.9) + inputs.perturbation(rng, 6, 2, 4, 0.02)]
    gs = [_gamma(p, rng, amp=0.1) for p in ps]
    return ps, xs, gs


def test_coupled_step_matches_oracle(ctx):
    from paper_1707_02156_gb300 import api
    ps, xs, gs = _pair(5)
    lam, E, shear, pe, dt = [0.5, 3.0], 0.2, 1.0, 10.0, 0.05

    def stokes(xx, gg):
        return timestep.velocity(xx, ps, ps, lam, gg, E, 0.0, shear, up=4)

    ref = sf.coupled_step(xs, gs, ps, dt, stokes, pe, imex1_estimate=True)
    disp_ref = np.concatenate([(a - b).ravel() for a, b in zip(ref["x"], xs)])
    dg_ref = np.concatenate([a - b for a, b in zip(ref["gamma"], gs)])
    x, g = _cuda(inputs.pack_drops(xs)), _cuda(np.concatenate(gs))
    for prec, tol in ((0, 1e-10), (1, 1e-7)):
        u0, x1, g1 = torch.zeros_like(x), torch.zeros_like(x), torch.zeros_like(g)
        info = api.coupled_step(ctx, ps, ps, x, g, u0, False, E, 0.0, lam, shear, 1.0 / pe, dt, x1, g1,
                                imex1_estimate=True, precision=prec, tol=1e-12 if prec == 0 else 1e-10)
        assert info["velocity_solves"] == 2 and all(s["converged"] for s in info["solve"])
        assert _relerr((x1 - x).cpu().numpy(), disp_ref) < tol, prec
        assert _relerr((g1 - g).cpu().numpy(), dg_ref) < tol, prec
        # the estimates are small differences of nearby quantities: they carry the solves' errors
        # relative to the step's change, hence looser bounds than the state itself
        for key in ("err_drop", "err_conservation", "err_imex1"):
            rel = 1e-3 if prec == 0 else 5e-2
            assert abs(info[key] - ref[key]) < rel * ref[key], (prec, key, info[key], ref[key])
        if prec == 0:
            # a retry with the same u^t (as after a rejected attempt) solves once and lands on the same step
            x2, g2 = torch.zeros_like(x), torch.zeros_like(g)
            info2 = api.coupled_step(ctx, ps, ps, x, g, u0, True, E, 0.0, lam, shear, 1.0 / pe, dt, x2, g2,
                                     precision=0, tol=1e-12)
            assert info2["velocity_solves"] == 1 and info2["err_imex1"] == -1.0
            assert _relerr((x2 - x).cpu().numpy(), (x1 - x).cpu().numpy()) < 1e-11
            assert _relerr((g2 - g).cpu().numpy(), (g1 - g).cpu().numpy()) < 1e-11


def test_adaptive_run_conserves_mass_and_keeps_steps_below_tolerance(ctx):
    from paper_1707_02156_gb300 import api
    rng = np.random.default_rng(6)
    p = 5
    x0 = inputs.sphere_coef(p, axes=(1.1, 0.95, 0.95)) + inputs.perturbation(rng, p, 2, 4, 0.02)
    g0 = _gamma(p, rng, amp=0.1)
    x, g = _cuda(x0), _cuda(g0)
    m0 = api.surfactant_mass(ctx, [p], x, g)[0]
    T, tol = 0.1, 1e-4
    res = api.run_coupled(ctx, [p], [p], x, g, 0.2, 0.0, [2.0], 1.0, 0.1, T, 0.1, tol, 0.05, precision=0,
                          solve_tol=1e-12)
    assert abs(res["t"] - T) < 1e-14
    assert res["steps_accepted"] >= 2 and res["err_max_accepted"] < tol
    assert res["velocity_solves"] == 2 * res["steps_accepted"] + res["steps_rejected"]
    m1 = api.surfactant_mass(ctx, [p], x, g)[0]
    assert abs(m1 - m0) / m0 < res["steps_accepted"] * tol
    assert api.next_dt(0.1, 4e-5, 1e-5, 1.0) == pytest.approx(sf.next_dt(0.1, 4e-5, 1e-5, 1.0), rel=1e-15)
