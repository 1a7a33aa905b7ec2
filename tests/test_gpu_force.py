"""GPU parity of the interfacial force (Sec. 1, Table 2, Sec. 1.3) and of the full physical solve of
two surfactant-covered drops near contact in shear (right-hand side 2 u_inf + S[f], Eq. main_eq)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import geometry, gmres, layer
from paper_1707_02156_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02156_gb300 import api, build
    build.build()
    return api.Context(0, upsample=4)


def _relerr(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("x_s", [0.0, 0.3])
def test_interfacial_force_matches_oracle(ctx, x_s):
    rng = np.random.default_rng(7)
    ps = [6, 10]
    xs = [inputs.sphere_coef(6, centre=(0, 0, 0)) + inputs.perturbation(rng, 6, 1, 4, 0.08),
          inputs.sphere_coef(10, centre=(3.0, 0, 0), axes=(0.9, 1.1, 1.0)) + inputs.perturbation(rng, 10, 2, 6, 0.05)]
    gams = []
    for p in ps:
        g = 0.2 * inputs.random_bandlimited(rng, p, 1)
        g[0, 0] = math.sqrt(4 * math.pi)
        gams.append(g)
    geo = ctx.geometry(ps, ps, torch.tensor(inputs.pack_drops(xs), device="cuda"), [1.0, 2.0])
    out = torch.zeros(sum(3 * (p + 1) ** 2 for p in ps), dtype=torch.float64, device="cuda")
    geo.interfacial_force(torch.tensor(inputs.pack_drops(gams), device="cuda"), 0.2, x_s, out)
    torch.cuda.synchronize()
    ref = inputs.pack_drops([geometry.interfacial_force(x, p, g[0], 0.2, x_s) for x, p, g in zip(xs, ps, gams)])
    assert _relerr(out.cpu().numpy(), ref) < FP64_TOL


def test_two_surfactant_drops_near_contact_solve(ctx):
    # the near-contact workload at reduced degree: Gamma = 1 + 0.3 Y_2^0, sigma = 1 - 0.2 Gamma,
    # shear (z, 0, 0), lambda = 0.5, gap 0.05: force, right-hand side and both solves on the GPU
    p = 8
    w = inputs.two_drops(p=p, gap=0.05, up=4, lam=0.5)
    nc = 3 * (p + 1) ** 2
    xs = [w.xcoef[:nc].reshape(3, -1), w.xcoef[nc:].reshape(3, -1)]
    gs = [w.gamma[:nc // 3], w.gamma[nc // 3:]]
    drops = layer.Drops(xs, [p, p], [p, p], w.lam, up=4)
    fs = [geometry.interfacial_force(x, p, g, w.elasticity) for x, g in zip(xs, gs)]
    uinf = [np.zeros((3, (p + 1) ** 2)) for _ in range(2)]
    for u, x in zip(uinf, xs):
        u[0] = w.shear * x[2]
    b = 2 * inputs.pack_drops(uinf) + np.concatenate([s.ravel() for s in drops.apply_single(fs)])
    u_ref, info = gmres.gmres(drops.system_matvec, b, tol=1e-13)
    assert info["converged"]
    geo = ctx.geometry([p, p], [p, p], torch.tensor(w.xcoef, device="cuda"), w.lam)
    f = torch.zeros(2 * nc, dtype=torch.float64, device="cuda")
    geo.interfacial_force(torch.tensor(w.gamma, device="cuda"), w.elasticity, 0.0, f)
    rhs = torch.zeros_like(f)
    geo.rhs(torch.tensor(inputs.pack_drops(uinf), device="cuda"), f, rhs)
    torch.cuda.synchronize()
    assert _relerr(rhs.cpu().numpy(), b) < FP64_TOL
    for prec, tol in ((0, 1e-11), (1, 1e-8)):
        u = torch.zeros_like(rhs)
        res = geo.solve(rhs, u, precision=prec, tol=1e-12 if prec == 0 else 1e-10)
        assert res["converged"]
        torch.cuda.synchronize()
        assert _relerr(u.cpu().numpy(), u_ref) < tol, (prec, res)
