"""GPU parity of the layer potentials and the velocity at points off the surfaces (bie_eval_single,
bie_eval_double, bie_eval_velocity) with the FP64 oracle (oracle/offsurface.py): points in all three
regions of two drops 0.05 apart (some in the gap, near both), a single deformed drop, a point set
that spans two 32768-point chunks with a ragged last tile, and points inside a drop.

Bars: FP64 1e-12 at points in Omega_0/1 of every drop (both sides run the same rules in FP64), 1e-9 at
points in Omega_2 of some drop, double-float 1e-11 / 1e-9, mixed 5e-6 (FP32 pair sums and self term,
FP64 check points: the bar of the on-surface multi-drop applies).  The Omega_2 bar is the near rule's
conditioning: the closest point is found by Newton to a step of 1e-14 and the interpolation through
(0, h sqrt(l)) amplifies by about 2e3, so a 1e-15 relative change of a point moves the oracle's own
value there by up to 9.5e-11 (measured on the 8-degree sphere of the two-chunk case)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import layer, offsurface, sh
from paper_1707_02156_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
DF_TOL = 1e-11
NEAR_TOL = 1e-9
MIXED_TOL = 5e-6


def _relerr(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _check(out, ref, near, tol):
    """Relative error within tol at the points off every drop's Omega_2, within NEAR_TOL (or tol if
    larger) at the points in some drop's Omega_2, each relative to the largest value of the set."""
    out, ref = np.asarray(out).reshape(3, -1), np.asarray(ref).reshape(3, -1)
    scale = np.max(np.abs(ref))
    far = ~near
    if np.any(far):
        e = max(_relerr(out[:, far], ref[:, far]), np.max(np.abs(out[:, far] - ref[:, far])) / scale)
        assert e < tol, ("far", e, tol)
    if np.any(near):
        e = np.max(np.abs(out[:, near] - ref[:, near])) / scale
        assert e < max(tol, NEAR_TOL), ("near", e)


def _near(drops, pts):
    return np.any(np.stack([offsurface.classify_points(drops, pts, j) == 2 for j in range(drops.N)]), axis=0)


def _points_off(xcoef, p, params, dists):
    """Points at signed distances along the outward normals of the surface at (theta, phi) params."""
    pts = []
    for (t0, f0), dist in zip(params, dists):
        d = [sh.evaluate_derivs(xcoef[c], p, np.array([t0]), np.array([f0])) for c in range(3)]
        xt, xp = np.array([d[c]["t"][0] for c in range(3)]), np.array([d[c]["p"][0] for c in range(3)])
        n = np.cross(xt, xp)
        pts.append(np.array([d[c]["f"][0] for c in range(3)]) + dist * n / np.linalg.norm(n))
    return np.array(pts).T


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02156_gb300 import api, build
    build.build()
    c = api.Context(0, upsample=4)
    yield c
    c.close()


@pytest.fixture(scope="module")
def pair(ctx):
    p = 10
    w = inputs.two_drops(p=p, gap=0.05, up=4, lam=0.5)
    nc = 3 * (p + 1) ** 2
    xs = [w.xcoef[:nc].reshape(3, -1), w.xcoef[nc:].reshape(3, -1)]
    fs = [w.density[:nc].reshape(3, -1), w.density[nc:].reshape(3, -1)]
    drops = layer.Drops(xs, [p, p], [p, p], w.lam, up=4)
    h = drops.h[1]
    # drop 0 sits above drop 1 (centres at z = +-1.025): points off drop 1's lower and side parts and
    # off drop 0's upper part, in each region
    dists = [0.3 * h, 0.7 * h, 2.0 * h, 4.0 * h, 9.0 * h]
    low = [(2.5, 0.3), (1.6, 2.0), (2.0, 4.0), (2.8, 1.0), (1.3, 5.0)]
    high = [(0.4, 1.0), (1.2, 3.0), (0.9, 5.0)]
    pts = np.concatenate([_points_off(xs[1], p, low, dists), _points_off(xs[0], p, high, dists[:3])], axis=1)
    # the midpoint of the gap: Omega_2 of both drops
    gap = 0.5 * (drops.std[0].x.mean(axis=1) + drops.std[1].x.mean(axis=1))
    pts = np.concatenate([pts, gap[:, None]], axis=1)
    for j in range(2):
        assert np.all(offsurface.classify_points(drops, pts, j) != offsurface.INSIDE)
    geo = ctx.geometry([p, p], [p, p], torch.tensor(w.xcoef, device="cuda"), w.lam)
    yield p, w, xs, fs, drops, geo, pts
    geo.close()


@pytest.mark.parametrize("kind", ["S", "D"])
def test_two_drops_every_region_matches_oracle(pair, kind):
    p, w, xs, fs, drops, geo, pts = pair
    codes = np.stack([offsurface.classify_points(drops, pts, j) for j in range(2)])
    assert set(codes.ravel()) == {0, 1, 2}
    ref = offsurface.layer_at(drops, pts, fs, kind)
    f = torch.tensor(w.density, device="cuda")
    P = torch.tensor(np.ascontiguousarray(pts), device="cuda")
    out = torch.zeros_like(P)
    fn = geo.eval_single if kind == "S" else geo.eval_double
    near = _near(drops, pts)
    for prec, tol in ((0, FP64_TOL), (2, DF_TOL), (1, MIXED_TOL)):
        out.fill_(1.0)
        fn(P, f, out, precision=prec)
        torch.cuda.synchronize()
        _check(out.cpu().numpy(), ref, near, tol)
    # raw normalisation: the plain integrals, 1/8pi and 1/4pi
    ref_raw = offsurface.layer_at(drops, pts, fs, kind, raw=True)
    fn(P, f, out, precision=0, raw=True)
    torch.cuda.synchronize()
    _check(out.cpu().numpy(), ref_raw, near, FP64_TOL)


def test_velocity_at_points_matches_oracle(pair):
    p, w, xs, fs, drops, geo, pts = pair
    rng = np.random.default_rng(8)
    us = [0.3 * inputs.random_bandlimited(rng, p, 3) for _ in range(2)]
    shear = 1.0
    ref = offsurface.velocity_at(drops, pts, fs, us, shear)
    f = torch.tensor(w.density, device="cuda")
    u = torch.tensor(np.concatenate([a.ravel() for a in us]), device="cuda")
    P = torch.tensor(np.ascontiguousarray(pts), device="cuda")
    uinf = torch.zeros_like(P)
    uinf[0] = shear * P[2]
    out = torch.zeros_like(P)
    near = _near(drops, pts)
    for prec, tol in ((0, FP64_TOL), (1, MIXED_TOL)):
        geo.velocity_at(P, f, u, out, uinf=uinf, precision=prec)
        torch.cuda.synchronize()
        _check(out.cpu().numpy(), ref, near, tol)


def test_single_deformed_drop_matches_oracle(ctx):
    # a one-drop geometry has no inter-drop data until the first evaluation builds it
    p = 12
    rng = np.random.default_rng(21)
    x = inputs.sphere_coef(p, axes=(1.1, 0.9, 1.0)) + inputs.perturbation(rng, p, 2, 5, 0.04)
    f = inputs.random_bandlimited(rng, p, 3)
    drops = layer.Drops([x], [p], [p], [3.0], up=4)
    h = drops.h[0]
    params = [(0.4, 1.0), (1.3, 4.0), (2.2, 2.0), (2.8, 5.5), (1.0, 3.0), (1.8, 0.2)]
    pts = _points_off(x, p, params, (0.2 * h, 0.9 * h, 1.5 * h, 3.5 * h, 6.0 * h, 20.0 * h))
    geo = ctx.geometry([p], [p], torch.tensor(x.ravel(), device="cuda"), [3.0])
    P = torch.tensor(np.ascontiguousarray(pts), device="cuda")
    fd = torch.tensor(f.ravel(), device="cuda")
    out = torch.zeros_like(P)
    near = _near(drops, pts)
    for kind, fn in (("S", geo.eval_single), ("D", geo.eval_double)):
        ref = offsurface.layer_at(drops, pts, [f], kind)
        fn(P, fd, out, precision=0)
        torch.cuda.synchronize()
        _check(out.cpu().numpy(), ref, near, FP64_TOL)
    geo.close()


def test_two_chunks_with_a_ragged_tail_match_oracle(ctx):
    # 32768 + 237 points around a sphere (most in Omega_0, some in Omega_1, a few in Omega_2 in the
    # second chunk): the chunk boundary, the last tile of 109 points and the pseudo-drop layout
    p = 8
    x = inputs.sphere_coef(p, radius=1.0, centre=(0.2, -0.1, 0.3))
    rng = np.random.default_rng(4)
    f = inputs.random_bandlimited(rng, p, 3)
    drops = layer.Drops([x], [p], [p], [2.0], up=4)  # the context's upsampling factor
    n = 32768 + 237
    d = rng.standard_normal((3, n))
    d /= np.linalg.norm(d, axis=0)
    r = rng.uniform(1.6, 6.0, n)
    r[-12:] = 1.0 + np.linspace(0.02, 0.3, 12)  # close to the unit sphere: Omega_2 and Omega_1
    pts = np.array([0.2, -0.1, 0.3])[:, None] + d * r
    codes = offsurface.classify_points(drops, pts, 0)
    assert np.sum(codes == 2) >= 3 and np.sum(codes == 1) >= 3 and not np.any(codes == offsurface.INSIDE)
    ref = offsurface.layer_at(drops, pts, [f], "D")
    geo = ctx.geometry([p], [p], torch.tensor(x.ravel(), device="cuda"), [2.0])
    P = torch.tensor(np.ascontiguousarray(pts), device="cuda")
    out = torch.zeros_like(P)
    geo.eval_double(P, torch.tensor(f.ravel(), device="cuda"), out, precision=0)
    torch.cuda.synchronize()
    _check(out.cpu().numpy(), ref, codes == 2, FP64_TOL)
    geo.close()


def test_points_inside_a_drop_and_empty_sets(pair):
    from paper_1707_02156_gb300 import api
    p, w, xs, fs, drops, geo, pts = pair
    f = torch.tensor(w.density, device="cuda")
    centre = drops.std[1].x.mean(axis=1)
    P = torch.tensor(np.ascontiguousarray(np.concatenate([pts, centre[:, None]], axis=1)), device="cuda")
    out = torch.zeros_like(P)
    with pytest.raises(api.BIEError):
        geo.eval_single(P, f, out)
    empty = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    geo.eval_single(empty, f, empty)
    with pytest.raises(api.BIEError):
        geo.eval_single(P[:, :4].contiguous(), f, out[:, :4].contiguous(), precision=0 | 0x1000)
