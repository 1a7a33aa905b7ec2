"""GPU parity of the midpoint step of the drop shapes (Sec. 3, Alg. 1, surfactant held fixed)
against the oracle's step: two deformed drops in shear, with surfactant and different viscosity
ratios; FP64 solves and mixed solves with double-float residuals."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import timestep
from paper_1707_02156_gb300 import inputs

pytestmark = pytest.mark.gpu


def _relerr(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_midpoint_step_matches_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02156_gb300 import api
    rng = np.random.default_rng(11)
    ps = [6, 7]
    xs = [inputs.sphere_coef(6, axes=(1.1, 0.95, 1.0), rot=inputs.random_rotation(rng)) +
          inputs.perturbation(rng, 6, 2, 4, 0.02),
          inputs.sphere_coef(7, centre=(2.4, 0.3, 0.2), radius=0.9) + inputs.perturbation(rng, 7, 2, 4, 0.02)]
    gam = []
    for p in ps:
        g = 0.1 * inputs.random_bandlimited(rng, p, 1)[0]
        g[0] += np.sqrt(4 * np.pi)  # Gamma = 1 + small variation
        gam.append(g)
    lam, E, shear, dt = [0.5, 3.0], 0.2, 1.0, 0.05
    ref = timestep.midpoint_step(xs, ps, ps, lam, gam, E, 0.0, shear, dt, up=4)
    disp_ref = np.concatenate([(r - x).ravel() for r, x in zip(ref, xs)])
    ctx = api.Context(0, upsample=4)
    g_dev = torch.tensor(np.concatenate(gam), device="cuda")
    for prec, tol in ((0, 1e-10), (1, 1e-7)):
        x = torch.tensor(inputs.pack_drops(xs), device="cuda")
        x0 = x.clone()
        infos = api.midpoint_step(ctx, ps, ps, x, g_dev, E, 0.0, lam, shear, dt, precision=prec,
                                  tol=1e-12 if prec == 0 else 1e-10)
        assert all(i["converged"] for i in infos)
        disp = (x - x0).cpu().numpy()
        assert _relerr(disp, disp_ref) < tol, (prec, _relerr(disp, disp_ref))
    ctx.close()
