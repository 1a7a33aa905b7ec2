"""GPU parity of the multi-drop layer operators (Sec. 2.1, 2.3) against the FP64 oracle: drops of
uneven degree and viscosity ratio at gaps where both the regular (Omega_0) and the upsampled (Omega_1)
rules occur; exact region counts; and the solve."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gmres, layer
from paper_1707_02156_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 5e-6  # FP32 rounding of multi-drop applies: measured 5.8e-8 .. 1.3e-6 relative; about 4x the largest
DF_TOL = 1e-11  # 2^-44 per operation, grown over ~10^4-term sums with magnitudes up to the 1/r peak


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02156_gb300 import api, build
    build.build()
    return api.Context(0, upsample=3)


def _batch(seed=5):
    """Four drops of degrees 6, 8, 10, 7 (sphere / perturbed / ellipsoid), gaps 0.6-1.5."""
    rng = np.random.default_rng(seed)
    spec = [(6, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)), (8, (2.6, 0.2, 0.1), (0.9, 1.1, 1.0)),
            (10, (-0.3, 2.7, 0.4), (1.0, 0.8, 1.2)), (7, (1.2, 1.4, 2.6), (1.1, 1.0, 0.9))]
    xs, fs, ps = [], [], []
    for p, c, ax in spec:
        x = inputs.sphere_coef(p, centre=c, axes=ax, rot=inputs.random_rotation(rng))
        x = x + inputs.perturbation(rng, p, 2, 4, 0.04)
        xs.append(x)
        fs.append(inputs.random_bandlimited(rng, p, 3))
        ps.append(p)
    lam = np.array([0.5, 3.0, 1.7, 4.2])
    return ps, xs, fs, lam


def _relerr(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def batch(ctx):
    ps, xs, fs, lam = _batch()
    drops = layer.Drops(xs, ps, ps, lam, up=3)
    geo = ctx.geometry(ps, ps, torch.tensor(inputs.pack_drops(xs), device="cuda"), lam)
    return ps, xs, fs, lam, drops, geo


def test_region_counts_match_oracle(batch):
    ps, xs, fs, lam, drops, geo = batch
    far = up = near = 0
    for (i, j), reg in drops.region.items():
        ng_j = (ps[j] + 1) * (2 * ps[j] + 2)
        nu_j = (3 * (ps[j] + 1)) * (6 * (ps[j] + 1))
        far += int(np.sum(reg == 0)) * ng_j
        up += int(np.sum(reg == 1)) * nu_j
        near += int(np.sum(reg == 2))
    assert up > 0 and far > 0 and near == 0
    assert geo.info["far_pairs"] == far
    assert geo.info["up_pairs"] == up
    assert geo.info["near_targets"] == near


@pytest.mark.parametrize("kind", ["S", "D"])
def test_multidrop_apply_matches_oracle(batch, kind):
    ps, xs, fs, lam, drops, geo = batch
    ref = (drops.apply_single if kind == "S" else drops.apply_double)(fs)
    ref = np.concatenate([r.ravel() for r in ref])
    f = torch.tensor(inputs.pack_drops(fs), device="cuda")
    out = torch.zeros_like(f)
    fn = geo.apply_single if kind == "S" else geo.apply_double
    # BIE_DF: inter-drop pair sums in double-float (about 44 bits), everything else FP64
    for prec, tol in ((0, FP64_TOL), (1, MIXED_TOL), (2, DF_TOL)):
        fn(f, out, precision=prec)
        torch.cuda.synchronize()
        assert _relerr(out.cpu().numpy(), ref) < tol, (kind, prec)
    # grid values, per target, before the projection
    gref = (drops.apply_single_grid if kind == "S" else drops.apply_double_grid)(fs)
    gref = np.concatenate([r.ravel() for r in gref])
    gout = torch.zeros(gref.size, dtype=torch.float64, device="cuda")
    fn(f, gout, precision=0, grid_out=True)
    torch.cuda.synchronize()
    assert _relerr(gout.cpu().numpy(), gref) < FP64_TOL


def test_multidrop_solve_matches_oracle(batch):
    ps, xs, fs, lam, drops, geo = batch
    uinf = [np.zeros((3, (p + 1) ** 2)) for p in ps]
    for u, x in zip(uinf, xs):
        u[0] = x[2]  # u_inf = (z, 0, 0)
    b = 2 * inputs.pack_drops(uinf) + np.concatenate([r.ravel() for r in drops.apply_single(fs)])
    u_ref, info = gmres.gmres(drops.system_matvec, b, tol=1e-13)
    assert info["converged"]
    rhs = torch.tensor(b, device="cuda")
    # FP64 GMRES; mixed with double-float residuals (the default); mixed with FP64 residuals
    for prec, resid, tol in ((0, 2, 1e-11), (1, 2, 1e-8), (1, 0, 1e-8)):
        u = torch.zeros_like(rhs)
        res = geo.solve(rhs, u, precision=prec, tol=1e-12 if prec == 0 else 1e-10, residual_precision=resid)
        assert res["converged"]
        torch.cuda.synchronize()
        assert _relerr(u.cpu().numpy(), u_ref) < tol, (prec, resid, res)


def test_overlapping_drops_are_rejected(ctx):
    from paper_1707_02156_gb300 import api
    p = 6
    xs = [inputs.sphere_coef(p), inputs.sphere_coef(p, centre=(1.5, 0, 0))]
    with pytest.raises(api.BIEError) as e:
        ctx.geometry([p, p], [p, p], torch.tensor(inputs.pack_drops(xs), device="cuda"), [1.0, 1.0])
    assert e.value.status == 6


def test_graph_replay_matches_eager_launches_bit_for_bit():
    # an apply captured into a CUDA graph (second call onwards) must give the eager result exactly
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02156_gb300 import api
    ps, xs, fs, lam = _batch(seed=9)
    x = torch.tensor(inputs.pack_drops(xs), device="cuda")
    f = torch.tensor(inputs.pack_drops(fs), device="cuda")
    outs = {}
    for graphs in (False, True):
        ctx = api.Context(0, upsample=3, use_graphs=graphs)
        geo = ctx.geometry(ps, ps, x, lam)
        res = []
        for prec in (0, 1):
            for call in range(3):  # eager, captured, replayed
                out = torch.zeros_like(f)
                geo.apply_double(f * (1.0 + 0.5 * call), out, precision=prec)
                torch.cuda.synchronize()
                res.append(out.cpu().numpy())
        outs[graphs] = res
        geo.close()
        ctx.close()
    for a, b in zip(outs[False], outs[True]):
        assert np.array_equal(a, b)


def test_more_degree_groups_than_one_launch_holds():
    # ten drops of ten different degrees: the self term and the Galerkin projection of all groups run
    # as one launch of at most eight groups, so this takes two launches of each
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02156_gb300 import api
    rng = np.random.default_rng(21)
    ps = list(range(3, 13))
    xs, fs = [], []
    for i, p in enumerate(ps):
        c = (3.0 * (i % 4), 3.0 * ((i // 4) % 3), 3.0 * (i // 12))
        x = inputs.sphere_coef(p, centre=c, axes=(1.0, 0.9, 1.1), rot=inputs.random_rotation(rng))
        xs.append(x + inputs.perturbation(rng, p, 1, 3, 0.03))
        fs.append(inputs.random_bandlimited(rng, p, 3))
    lam = np.linspace(0.5, 3.0, len(ps))
    drops = layer.Drops(xs, ps, ps, lam, up=3)
    ctx = api.Context(0, upsample=3)
    geo = ctx.geometry(ps, ps, torch.tensor(inputs.pack_drops(xs), device="cuda"), lam)
    f = torch.tensor(inputs.pack_drops(fs), device="cuda")
    out = torch.zeros_like(f)
    for kind in ("S", "D"):
        ref = np.concatenate([r.ravel() for r in (drops.apply_single if kind == "S" else drops.apply_double)(fs)])
        for prec, tol in ((0, FP64_TOL), (1, MIXED_TOL)):
            (geo.apply_single if kind == "S" else geo.apply_double)(f, out, precision=prec)
            torch.cuda.synchronize()
            assert _relerr(out.cpu().numpy(), ref) < tol, (kind, prec)
    geo.close()
    ctx.close()


def test_double_float_rhs_matches_fp64(batch):
    # b = 2 u_inf + S[f] with the single layer in double-float (inter-drop pairs) and in FP64
    ps, xs, fs, lam, drops, geo = batch
    f = torch.tensor(inputs.pack_drops(fs), device="cuda")
    uinf = torch.zeros_like(f)
    b64, bdf = torch.zeros_like(f), torch.zeros_like(f)
    geo.rhs(uinf, f, b64, precision=0)
    geo.rhs(uinf, f, bdf, precision=2)
    torch.cuda.synchronize()
    assert _relerr(bdf.cpu().numpy(), b64.cpu().numpy()) < DF_TOL


def test_double_float_single_drop_matches_fp64():
    # one drop: the self term alone, in double-float arithmetic against FP64
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02156_gb300 import api
    rng = np.random.default_rng(3)
    p = 9
    x = inputs.sphere_coef(p) + inputs.perturbation(rng, p, 1, 4, 0.05)
    f = torch.tensor(inputs.random_bandlimited(rng, p, 3).ravel(), device="cuda")
    ctx = api.Context(0)
    geo = ctx.geometry([p], [p], torch.tensor(x.ravel(), device="cuda"), [2.0])
    a, b = torch.zeros_like(f), torch.zeros_like(f)
    geo.apply_double(f, a, precision=0)
    geo.apply_double(f, b, precision=2)
    torch.cuda.synchronize()
    assert _relerr(b.cpu().numpy(), a.cpu().numpy()) < DF_TOL
    geo.close()
    ctx.close()


def test_interleaved_degree_groups_match_oracle(ctx):
    # five drops whose degrees alternate (6, 8, 6, 8, 6): each degree group's drops are separated in
    # memory by drops of the other degree, as in a batch of seeded random degrees.  The singular
    # rule's rotated geometry of every drop must use that drop's own targets (a set-up that read the
    # targets of a group's later drops from the slots after its first drop gave O(1) errors on them).
    rng = np.random.default_rng(17)
    ps = [6, 8, 6, 8, 6]
    centres = [(0.0, 0.0, 0.0), (2.7, 0.0, 0.3), (5.3, 0.4, 0.0), (0.2, 2.8, 0.5), (2.9, 2.6, -0.4)]
    xs, fs = [], []
    for p, c in zip(ps, centres):
        x = inputs.sphere_coef(p, centre=c, axes=(1.0, 0.9, 1.1), rot=inputs.random_rotation(rng))
        xs.append(x + inputs.perturbation(rng, p, 2, 4, 0.04))
        fs.append(inputs.random_bandlimited(rng, p, 3))
    lam = np.array([0.5, 2.0, 3.5, 1.5, 4.0])
    drops = layer.Drops(xs, ps, ps, lam, up=3)
    geo = ctx.geometry(ps, ps, torch.tensor(inputs.pack_drops(xs), device="cuda"), lam)
    f = torch.tensor(inputs.pack_drops(fs), device="cuda")
    for kind in ("S", "D"):
        ref = (drops.apply_single_grid if kind == "S" else drops.apply_double_grid)(fs)
        ref = np.concatenate([r.ravel() for r in ref])
        out = torch.zeros(ref.size, dtype=torch.float64, device="cuda")
        fn = geo.apply_single if kind == "S" else geo.apply_double
        for prec, tol in ((0, FP64_TOL), (1, MIXED_TOL), (2, DF_TOL)):
            fn(f, out, precision=prec, grid_out=True)
            torch.cuda.synchronize()
            o = out.cpu().numpy()
            # every drop on its own, so that a fault confined to some drops cannot hide in the norm
            off = 0
            for p in ps:
                n = 3 * (p + 1) * (2 * p + 2)
                assert _relerr(o[off:off + n], ref[off:off + n]) < tol, (kind, prec, p, off)
                off += n
    geo.close()
