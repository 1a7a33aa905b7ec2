"""GPU parity of one coupled step (Alg. 1) of the four-drop cluster around drop 23 of the 64-drop
batch (degrees 48, 24, 16, 48, at their batch positions) with the oracle's step stored by
tests/golden/make_c4_cluster_step.py: both velocity solves, the explicit rates, the implicit stage,
the new shapes and surfactant, and the surfactant masses.

The two degree-48 drops of the cluster are not adjacent in memory (drops 0 and 3 of the cluster), the
layout under which the singular rule's set-up once read a drop's targets from the wrong slots.

Bars: FP64 solves at tol 1e-12 (the step's velocities and displacements to 1e-9 relative, through
the dt = 0.01 difference of the positions), the rates and masses FP64 arithmetic on both sides
(1e-12, 1e-13), the implicit solve 1e-11; mixed solves (tol 1e-10) to 1e-7 on the displacement."""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import surfactant as sf
from paper_1707_02156_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c4_cluster_step.npz")


def _relerr(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02156_gb300 import api, build
    build.build()
    z = np.load(GOLDEN)
    w = inputs.config("c4")
    offs = np.cumsum([0] + [3 * (p + 1) ** 2 for p in w.p])
    goffs = np.cumsum([0] + [(p + 1) ** 2 for p in w.p])
    ids = [int(i) for i in z["ids"]]
    ps = [w.p[i] for i in ids]
    assert ps == [int(v) for v in z["p"]] and int(z["up"]) == w.up
    x = np.concatenate([w.xcoef[offs[i]:offs[i + 1]] for i in ids])
    g = np.concatenate([w.gamma[goffs[i]:goffs[i + 1]] for i in ids])
    lam = [w.lam[i] for i in ids]
    ctx = api.Context(0, upsample=w.up)
    yield api, ctx, z, ps, x, g, lam, w
    ctx.close()


def _step(api, ctx, z, ps, x, g, lam, w, precision):
    xd, gd = torch.tensor(x, device="cuda"), torch.tensor(g, device="cuda")
    u0, x1, g1 = torch.zeros_like(xd), torch.zeros_like(xd), torch.zeros_like(gd)
    api.coupled_step(ctx, ps, ps, xd, gd, u0, False, w.elasticity, 0.0, lam, float(z["shear"]), 1.0 / float(z["pe"]),
                     float(z["dt"]), x1, g1, precision=precision, tol=1e-12 if precision == 0 else 1e-10)
    m1 = api.surfactant_mass(ctx, ps, x1, g1)
    torch.cuda.synchronize()
    return u0.cpu().numpy(), x1.cpu().numpy(), g1.cpu().numpy(), np.array(m1)


def test_cluster_coupled_step_fp64_matches_oracle(case):
    api, ctx, z, ps, x, g, lam, w = case
    dt = float(z["dt"])
    u0, x1, g1, m1 = _step(api, ctx, z, ps, x, g, lam, w, 0)
    assert _relerr(u0, z["u0"]) < 1e-10                       # velocity solve at (x^t, Gamma^t)
    assert _relerr((x1 - x) / dt, z["uh"]) < 1e-9             # the solve at t + dt/2, through x^{t+dt}
    assert _relerr(g1 - g, z["gamma1"] - g) < 1e-9            # the surfactant change of the step
    assert _relerr(m1, z["mass1"]) < 1e-13
    cons_gpu = np.abs(m1 - z["mass0"]) / np.abs(z["mass0"])
    cons_ref = np.abs(z["mass1"] - z["mass0"]) / np.abs(z["mass0"])
    assert np.all(np.abs(cons_gpu - cons_ref) < 1e-12), (cons_gpu, cons_ref)
    assert np.max(cons_gpu) < 1e-7


def test_cluster_rates_and_implicit_stage_match_oracle(case):
    # the explicit rate at (x^t, u^t, Gamma^t) and the implicit stage to Gamma^{t+dt/2}, with the
    # oracle's velocity u^t as input on both sides
    api, ctx, z, ps, x, g, lam, w = case
    dt, pe = float(z["dt"]), float(z["pe"])
    xd, gd = torch.tensor(x, device="cuda"), torch.tensor(g, device="cuda")
    ud = torch.tensor(z["u0"], device="cuda")
    fe = torch.zeros_like(gd)
    api.surfactant_rates(ctx, ps, xd, ud, gd, 0.0, fe, None)
    torch.cuda.synchronize()
    ref, o, og = [], 0, 0
    for p in ps:
        k = (p + 1) ** 2
        ref.append(sf.f_explicit(x[o:o + 3 * k].reshape(3, -1), z["u0"][o:o + 3 * k].reshape(3, -1), g[og:og + k], p))
        o += 3 * k
        og += k
    assert _relerr(fe.cpu().numpy(), np.concatenate(ref)) < 1e-12
    xh = xd + 0.5 * dt * ud
    rhs = gd + 0.5 * dt * fe
    gh = torch.zeros_like(gd)
    api.surfactant_implicit(ctx, ps, xh, rhs, 0.5 * dt / pe, gh)
    torch.cuda.synchronize()
    assert _relerr(gh.cpu().numpy(), z["gamma_h"]) < 1e-11


def test_cluster_coupled_step_mixed_matches_oracle(case):
    api, ctx, z, ps, x, g, lam, w = case
    dt = float(z["dt"])
    u0, x1, g1, m1 = _step(api, ctx, z, ps, x, g, lam, w, 1)
    assert _relerr((x1 - x) / dt, z["uh"]) < 1e-7
    assert _relerr(g1 - g, z["gamma1"] - g) < 1e-7
