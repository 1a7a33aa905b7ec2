"""Full-size solve parity: the device solve of the single-drop shear system (p = 32, p_q = 65,
lambda = 5, u_inf = (z, 0, 0), the seeded density as interfacial force) against the oracle's FP64
GMRES solution stored by tests/golden/make_c2_solution.py.

Bars: the right-hand side 2 u_inf + S[f] at 1e-12 (FP64) and 1e-11 (double-float); the FP64 solve
(tol 1e-12; the system's condition number is below 10, so the solution error is below 1e-11) at
1e-11; the mixed solve (FP32 inner GMRES inside refinement with double-float residuals, tol 1e-10)
at 1e-8."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1707_02156_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_solution.npz")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02156_gb300 import api, build
    build.build()
    return api.Context(0)


def relerr(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_full_size_single_drop_solve_matches_oracle(ctx):
    z = np.load(GOLDEN)
    w = inputs.perturbed_drop()
    assert int(z["p"]) == w.p[0] and int(z["pq"]) == w.pq[0] and float(z["lam"][0]) == w.lam[0]
    x = torch.tensor(w.xcoef, device="cuda")
    geo = ctx.geometry(w.p, w.pq, x, w.lam)
    nco = geo.info["ncoef"]
    uinf = torch.zeros(nco, dtype=torch.float64, device="cuda")
    uinf.view(3, -1)[0] = x.view(3, -1)[2] * w.shear  # u_inf = (z, 0, 0) is band-limited: z's coefficients
    f = torch.tensor(w.density, device="cuda")
    b64, bdf = torch.zeros_like(uinf), torch.zeros_like(uinf)
    geo.rhs(uinf, f, b64, precision=0)
    geo.rhs(uinf, f, bdf, precision=2)
    torch.cuda.synchronize()
    assert relerr(b64.cpu().numpy(), z["b"]) < 1e-12
    assert relerr(bdf.cpu().numpy(), z["b"]) < 1e-11
    u = torch.zeros_like(uinf)
    info = geo.solve(b64, u, precision=0, tol=1e-12)
    torch.cuda.synchronize()
    assert info["converged"]
    assert relerr(u.cpu().numpy(), z["u"]) < 1e-11, info
    u.zero_()
    info = geo.solve(bdf, u, precision=1, tol=1e-10, residual_precision=2)
    torch.cuda.synchronize()
    assert info["converged"]
    assert relerr(u.cpu().numpy(), z["u"]) < 1e-8, info
    geo.close()
