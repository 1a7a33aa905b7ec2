"""GPU parity of the near-singular (Omega_2) step of Sec. 2.3 against the FP64 oracle: two drops at
gap 0.05, where targets fall in all three regions; closest-point Newton, check points, anchors and
Lagrange interpolation all run on the GPU."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import layer
from paper_1707_02156_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 5e-6  # FP32 rounding of multi-drop applies: measured 5.8e-8 .. 1.3e-6 relative; about 4x the largest


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02156_gb300 import api, build
    build.build()
    ctx = api.Context(0, upsample=4)
    p = 10
    w = inputs.two_drops(p=p, gap=0.05, up=4, lam=0.5)
    nc = 3 * (p + 1) ** 2
    xs = [w.xcoef[:nc].reshape(3, -1), w.xcoef[nc:].reshape(3, -1)]
    fs = [w.density[:nc].reshape(3, -1), w.density[nc:].reshape(3, -1)]
    drops = layer.Drops(xs, [p, p], [p, p], w.lam, up=4)
    geo = ctx.geometry([p, p], [p, p], torch.tensor(w.xcoef, device="cuda"), w.lam)
    return p, w, xs, fs, drops, geo


def _relerr(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_near_region_counts(setup):
    p, w, xs, fs, drops, geo = setup
    near = sum(int(np.sum(r == 2)) for r in drops.region.values())
    assert near > 0
    assert geo.info["near_targets"] == near


@pytest.mark.parametrize("kind", ["S", "D"])
def test_near_contact_apply_matches_oracle(setup, kind):
    p, w, xs, fs, drops, geo = setup
    gref = (drops.apply_single_grid if kind == "S" else drops.apply_double_grid)(fs)
    gref = np.concatenate([r.ravel() for r in gref])
    f = torch.tensor(w.density, device="cuda")
    out = torch.zeros(gref.size, dtype=torch.float64, device="cuda")
    fn = geo.apply_single if kind == "S" else geo.apply_double
    for prec, tol in ((0, FP64_TOL), (1, MIXED_TOL)):
        fn(f, out, precision=prec, grid_out=True)
        torch.cuda.synchronize()
        assert _relerr(out.cpu().numpy(), gref) < tol, (kind, prec)
    cref = (drops.apply_single if kind == "S" else drops.apply_double)(fs)
    cref = np.concatenate([r.ravel() for r in cref])
    cout = torch.zeros_like(f)
    fn(f, cout, precision=0)
    torch.cuda.synchronize()
    assert _relerr(cout.cpu().numpy(), cref) < FP64_TOL


def test_near_contact_translating_sphere_field(setup):
    # uniform traction c_j on each sphere: S_raw at drop 0's targets = (2/3) c_0 + translating-sphere
    # field of drop 1; closed form, independent of the oracle
    p, w, xs, fs, drops, geo = setup
    cvec = [np.array([0.0, 0.3, 1.0]), np.array([0.5, 0.0, -0.2])]
    dens = np.zeros((2, 3, (p + 1) ** 2))
    for d in range(2):
        dens[d, :, 0] = cvec[d] * math.sqrt(4 * math.pi)
    out = torch.zeros(2 * 3 * (p + 1) * (2 * p + 2), dtype=torch.float64, device="cuda")
    geo.apply_single(torch.tensor(dens.ravel(), device="cuda"), out, raw=True, grid_out=True)
    torch.cuda.synchronize()
    S0 = out.cpu().numpy()[:3 * (p + 1) * (2 * p + 2)].reshape(3, -1)
    xt = drops.targets[0]
    xh = xt - np.array([0, 0, -1.025])[:, None]
    r = np.linalg.norm(xh, axis=0)
    c = cvec[1]
    xc = np.sum(xh * c[:, None], axis=0)
    field = 0.5 * (c[:, None] / r + xh * xc / r ** 3 + (c[:, None] / r ** 3 - 3 * xh * xc / r ** 5) / 3.0)
    exact = (2.0 / 3.0) * cvec[0][:, None] + field
    reg = drops.region[(0, 1)]
    err = np.abs(S0 - exact)
    assert np.max(err[:, reg == 0]) < 1e-9
    assert np.max(err[:, reg == 1]) < 1e-12
    assert np.max(err[:, reg == 2]) < 1e-4
