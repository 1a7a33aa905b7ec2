"""GPU parity of the C-ABI library against the FP64 oracle: transforms, rotation, and the
single-drop layer operators and solve.  FP64 path: 1e-12 relative; mixed path: 2e-6 relative
for one apply (FP32 rotation, synthesis and pair sums), 1e-8 after refinement in the solve."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gmres, layer, sh, wigner
from paper_1707_02156_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 2e-6  # FP32 rounding of the single-drop applies: measured 5.9e-8 .. 5.3e-7 relative; about 4x the largest
DF_TOL = 1e-11  # double-float: about 44 bits per operation


@pytest.fixture(scope="module", params=[(False, True), (True, True), (False, False)],
                ids=["projected", "direct", "projected-cuda-core-rotation"])
def ctx(request):
    # projected self form with the mixed rotation on the tensor cores (default), the direct form, and
    # the projected form with the mixed rotation on the CUDA cores
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02156_gb300 import api, build
    build.build()
    direct, tc = request.param
    return api.Context(0, self_direct=direct, tensor_rotation=tc)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relerr(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_sh_analyze_synthesize_match_oracle(ctx):
    rng = np.random.default_rng(0)
    ps = [3, 9, 16]
    pouts = [3, 20, 33]
    coefs = [inputs.random_bandlimited(rng, p, 2, decay_pow=0.5) for p in ps]
    c = dev(np.concatenate([x.ravel() for x in coefs]))
    ng = sum(2 * (q + 1) * (2 * q + 2) for q in pouts)
    g = torch.zeros(ng, dtype=torch.float64, device="cuda")
    ctx.sh_synthesize(ps, pouts, 2, c, g)
    gh = host(g)
    o = 0
    for p, q, x in zip(ps, pouts, coefs):
        for comp in range(2):
            n = (q + 1) * (2 * q + 2)
            ref = sh.synthesize(x[comp], p, q)
            assert relerr(gh[o:o + n], ref) < FP64_TOL
            o += n
    # analysis on the native grids (degree p) back to coefficients
    gp = torch.zeros(sum(2 * (p + 1) * (2 * p + 2) for p in ps), dtype=torch.float64, device="cuda")
    ctx.sh_synthesize(ps, ps, 2, c, gp)
    back = torch.zeros_like(c)
    ctx.sh_analyze(ps, 2, gp, back)
    assert relerr(host(back), host(c)) < FP64_TOL


def test_rotate_matches_oracle(ctx):
    rng = np.random.default_rng(1)
    ps = [5, 16, 32]
    coefs = [inputs.random_bandlimited(rng, p, 3, decay_pow=0.5) for p in ps]
    eul = [(0.3, 1.1, -0.4), (2.0, 2.9, 0.0), (-1.2, 0.05, 1.7)]
    c = dev(np.concatenate([x.ravel() for x in coefs]))
    out = torch.zeros_like(c)
    ctx.rotate(ps, 3, c, eul, out)
    oh = host(out)
    o = 0
    for p, x, e in zip(ps, coefs, eul):
        for comp in range(3):
            n = (p + 1) ** 2
            assert relerr(oh[o:o + n], wigner.rotate(x[comp], p, *e)) < FP64_TOL
            o += n


def _single(ctx, w):
    return ctx.geometry(w.p, w.pq, dev(w.xcoef), w.lam)


@pytest.mark.parametrize("kind", ["S", "D"])
def test_self_apply_sphere_p16_matches_oracle(ctx, kind):
    # lambda = 1 makes the scaled double layer vanish, so the double layer is compared raw
    w = inputs.single_sphere(16)
    geo = _single(ctx, w)
    p = 16
    drops = layer.Drops([w.xcoef.reshape(3, -1)], [p], [p], w.lam)
    if kind == "S":
        ref = drops.apply_single([w.density])[0].ravel()
    else:
        ref = drops.apply_double([w.density], raw=True)[0].ravel()
    f = dev(w.density)
    out = torch.zeros_like(f)
    for prec, tol in ((0, FP64_TOL), (1, MIXED_TOL)):
        if kind == "S":
            geo.apply_single(f, out, precision=prec)
        else:
            geo.apply_double(f, out, precision=prec, raw=True)
        assert relerr(host(out), ref) < tol, (kind, prec)


@pytest.mark.parametrize("kind", ["S", "D"])
def test_self_apply_perturbed_upsampled_quadrature_matches_oracle(ctx, kind):
    # several tiles of targets, a ragged last rotation chunk, p_q = 2p+1
    p = 11
    w = inputs.perturbed_drop(p=p, lam=5.0)
    geo = _single(ctx, w)
    drops = layer.Drops([w.xcoef.reshape(3, -1)], [p], [2 * p + 1], w.lam)
    f = dev(w.density)
    out = torch.zeros_like(f)
    ref = (drops.apply_single if kind == "S" else drops.apply_double)([w.density])[0].ravel()
    # FP64, mixed, and double-float (the self term's rotation and contraction on the FP32 pipes)
    for prec, tol in ((0, FP64_TOL), (1, MIXED_TOL), (2, DF_TOL)):
        (geo.apply_single if kind == "S" else geo.apply_double)(f, out, precision=prec)
        assert relerr(host(out), ref) < tol, (kind, prec)


def test_self_apply_full_size_sampled_targets(ctx):
    # the bench workload (p = 32, p_q = 65): grid values at sampled latitudes against the oracle
    w = inputs.perturbed_drop()
    p, pq = w.p[0], w.pq[0]
    geo = _single(ctx, w)
    f = dev(w.density)
    out = torch.zeros(3 * (p + 1) * (2 * p + 2), dtype=torch.float64, device="cuda")
    q = layer.SelfQuadrature(w.xcoef.reshape(3, -1), p, pq)
    lats = [0, 13, 32]
    lam = w.lam[0]
    for kind in ("S", "D"):
        fn = geo.apply_single if kind == "S" else geo.apply_double
        wt = -1 / (4 * math.pi) if kind == "S" else (lam - 1) / (4 * math.pi)
        ref = wt * q.apply(w.density, kind, lats=lats)
        for prec, tol in ((0, FP64_TOL), (1, MIXED_TOL)):
            fn(f, out, precision=prec, grid_out=True)
            g = host(out).reshape(3, p + 1, 2 * p + 2)
            assert relerr(g[:, lats, :], ref[:, lats, :]) < tol, (kind, prec)


def test_solve_fp64_and_mixed_match_oracle(ctx):
    p = 8
    w = inputs.perturbed_drop(p=p, lam=5.0)
    geo = _single(ctx, w)
    drops = layer.Drops([w.xcoef.reshape(3, -1)], [p], [2 * p + 1], w.lam)
    uinf = np.zeros((3, (p + 1) ** 2))
    uinf[0] = w.xcoef.reshape(3, -1)[2]  # u_inf = (z, 0, 0)
    b = 2 * uinf.ravel() + drops.apply_single([w.density])[0].ravel()
    u_ref, info = gmres.gmres(drops.system_matvec, b, tol=1e-13)
    assert info["converged"]
    rhs = dev(b)
    for prec, tol in ((0, 1e-11), (1, 1e-8)):
        u = torch.zeros_like(rhs)
        res = geo.solve(rhs, u, precision=prec, tol=1e-12 if prec == 0 else 1e-10)
        assert res["converged"]
        assert relerr(host(u), u_ref) < tol, (prec, res)
