"""Checkpoint and resume of a coupled drop/surfactant run (Alg. 1), host side.

The state of a run is, per drop, the SH coefficients of the shape and of the surfactant, the
degrees p and p_q and the viscosity ratio, together with the time reached and the step size that
the rule of Alg. 1 proposes next.  Everything built per geometry (tables, projected kernel
factors, work lists) is rebuilt from the shapes when the run resumes.  The archive is a NumPy
.npz file; the run's physical parameters travel with it as a JSON string.

Resume a run of run_coupled (bie_run_coupled) from a state saved after it returned: upload x and
gamma, then call it again with dt0 = dt_next and T = T_end - t.
"""
from __future__ import annotations

import json

import numpy as np


def _host(a) -> np.ndarray:
    if hasattr(a, "detach"):  # a torch tensor on any device
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)


def _check(p, pq, lam, x, gamma) -> None:
    """Raise ValueError unless the per-drop arrays agree: one p_q and one lambda per drop,
    p <= p_q <= 2p+1 (the self-rule degrees bie_geometry_setup accepts), and coefficient arrays of
    3 (p+1)^2 and (p+1)^2 entries per drop."""
    if p.ndim != 1 or len(p) == 0 or np.any(p < 1):
        raise ValueError("p must list one degree >= 1 per drop")
    if len(pq) != len(p) or len(lam) != len(p):
        raise ValueError("pq and lam must have one entry per drop")
    if np.any(pq < p) or np.any(pq > 2 * p + 1):
        raise ValueError("each p_q must satisfy p <= p_q <= 2p+1")
    nc = (p + 1) ** 2
    if x.size != 3 * int(nc.sum()) or gamma.size != int(nc.sum()):
        raise ValueError("coefficient arrays do not match the degrees")


def save(path: str, *, p, pq, lam, x, gamma, t: float, dt_next: float, **params) -> None:
    """Write the state of a run.  x: [drop][3][(p+1)^2] coefficients, gamma: [drop][(p+1)^2]
    (flat, host or device arrays); params: the run's scalars (elasticity, shear, 1/Pe, ...).
    Raises ValueError if the per-drop arrays do not agree (see _check)."""
    p = np.atleast_1d(np.asarray(p, dtype=np.int64))
    pq = np.atleast_1d(np.asarray(pq, dtype=np.int64))
    lam = np.atleast_1d(np.asarray(lam, dtype=np.float64))
    x, gamma = _host(x), _host(gamma)
    _check(p, pq, lam, x, gamma)
    np.savez(path, p=p, pq=pq, lam=lam, x=x, gamma=gamma, t=np.float64(t), dt_next=np.float64(dt_next),
             params=np.array(json.dumps(params)))


def load(path: str) -> dict:
    """The state written by save: numpy arrays and the run's parameters.  The per-drop arrays are
    checked as in save (ValueError on a mismatch)."""
    with np.load(path, allow_pickle=False) as z:
        out = {k: z[k] for k in ("p", "pq", "lam", "x", "gamma")}
        out["t"] = float(z["t"])
        out["dt_next"] = float(z["dt_next"])
        out["params"] = json.loads(str(z["params"]))
    _check(out["p"], out["pq"], out["lam"], out["x"], out["gamma"])
    return out
