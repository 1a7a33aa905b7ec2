"""Checkpoint and resume of a coupled run (host side): the archive round-trips the state exactly,
and a run split at a checkpoint reproduces the uninterrupted run (the oracle's Alg. 1 with a
prescribed flow)."""
import math

import numpy as np
import pytest

from oracle import surfactant as sf
from paper_1707_02156_gb300 import checkpoint, inputs


def _flow(xs, gs):
    out = []
    for x in xs:
        p = int(round(math.sqrt(x.shape[1]))) - 1
        P = 2 * p + 1
        X = np.stack([sf.sh.synthesize(x[c], p, P) for c in range(3)])
        U = np.stack([0.6 * X[2] + 0.2 * X[0] * X[1], -0.3 * X[1], 0.3 * X[2] - 0.2 * X[0] ** 2])
        out.append(np.stack([sf.sh.analyze(U[c], P, p) for c in range(3)]))
    return out


def test_round_trip_is_exact(tmp_path):
    rng = np.random.default_rng(1)
    p = [3, 5]
    x = np.concatenate([rng.standard_normal(3 * (q + 1) ** 2) for q in p])
    g = np.concatenate([rng.standard_normal((q + 1) ** 2) for q in p])
    f = str(tmp_path / "state.npz")
    checkpoint.save(f, p=p, pq=[7, 11], lam=[0.5, 2.0], x=x, gamma=g, t=0.125, dt_next=0.03125, shear=1.0,
                    elasticity=0.2, inv_pe=0.1)
    s = checkpoint.load(f)
    assert s["p"].tolist() == p and s["pq"].tolist() == [7, 11] and s["lam"].tolist() == [0.5, 2.0]
    assert np.array_equal(s["x"], x) and np.array_equal(s["gamma"], g)
    assert s["t"] == 0.125 and s["dt_next"] == 0.03125
    assert s["params"] == {"shear": 1.0, "elasticity": 0.2, "inv_pe": 0.1}
    with pytest.raises(ValueError):
        checkpoint.save(f, p=p, pq=p, lam=[1, 1], x=x[:-1], gamma=g, t=0.0, dt_next=0.1)
    # per-drop arrays of the wrong length, and self-rule degrees outside p <= p_q <= 2p+1
    for bad in ({"pq": [7], "lam": [1, 1]}, {"pq": [7, 11], "lam": [1.0]}, {"pq": [2, 11], "lam": [1, 1]},
                {"pq": [8, 11], "lam": [1, 1]}):
        with pytest.raises(ValueError):
            checkpoint.save(f, p=p, x=x, gamma=g, t=0.0, dt_next=0.1, **bad)
    # an archive written by other means is checked on load too
    np.savez(f, p=np.array(p), pq=np.array([7]), lam=np.array([0.5, 2.0]), x=x, gamma=g, t=0.0, dt_next=0.1,
             params=np.array("{}"))
    with pytest.raises(ValueError):
        checkpoint.load(f)


def test_resumed_run_reproduces_the_uninterrupted_run(tmp_path):
    # cut the run where the uninterrupted run itself lands after its second kept step: the first
    # part takes the same steps, and the resumed part continues with the proposed step size
    p, pe, tol, T = 6, 4.0, 1e-5, 0.08
    rng = np.random.default_rng(22)
    x = inputs.sphere_coef(p, axes=(0.9, 1.0, 1.15)) + inputs.perturbation(rng, p, 1, 4, 0.03)
    g = 0.2 * inputs.random_bandlimited(rng, p, 1)[0]
    g[0] += 2.0 * math.sqrt(4 * math.pi)
    # dt0 small enough that no attempt before the cut is shortened by the end of the first part
    full = sf.run_adaptive([x], [g], [p], T, 0.004, tol, _flow, pe, 0.05)
    kept = [h for h in full["history"] if h["accepted"]]
    assert len(kept) >= 4
    t_cut = kept[1]["t"] + kept[1]["dt"]
    first = sf.run_adaptive([x], [g], [p], t_cut, 0.004, tol, _flow, pe, 0.05)
    f = str(tmp_path / "cut.npz")
    checkpoint.save(f, p=[p], pq=[p], lam=[1.0], x=first["x"][0], gamma=first["gamma"][0], t=first["t"],
                    dt_next=first["dt_next"], inv_pe=1.0 / pe)
    s = checkpoint.load(f)
    rest = sf.run_adaptive([s["x"].reshape(3, -1)], [s["gamma"]], [p], T - s["t"], s["dt_next"], tol, _flow,
                           pe, 0.05)
    assert abs(s["t"] + rest["t"] - T) < 1e-14
    assert len([h for h in rest["history"] if h["accepted"]]) == len(kept) - 2
    assert np.max(np.abs(rest["x"][0] - full["x"][0])) < 1e-12
    assert np.max(np.abs(rest["gamma"][0] - full["gamma"][0])) < 1e-12
