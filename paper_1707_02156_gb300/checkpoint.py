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


def save(path: str, *, p, pq, lam, x, gamma, t: float, dt_next: float, **params) -> None:
    """Write the state of a run.  x: [drop][3][(p+1)^2] coefficients, gamma: [drop][(p+1)^2]
    (flat, host or device arrays); params: the run's scalars (elasticity, shear, 1/Pe, ...)."""
    p = np.asarray(p, dtype=np.int64)
    nc = (p + 1) ** 2
    x, gamma = _host(x), _host(gamma)
    if x.size != 3 * int(nc.sum()) or gamma.size != int(nc.sum()):
        raise ValueError("coefficient arrays do not match the degrees")
    np.savez(path, p=p, pq=np.asarray(pq, dtype=np.int64), lam=np.asarray(lam, dtype=np.float64), x=x,
             gamma=gamma, t=np.float64(t), dt_next=np.float64(dt_next), params=np.array(json.dumps(params)))


def load(path: str) -> dict:
    """The state written by save: numpy arrays and the run's parameters."""
    with np.load(path, allow_pickle=False) as z:
        out = {k: z[k] for k in ("p", "pq", "lam", "x", "gamma")}
        out["t"] = float(z["t"])
        out["dt_next"] = float(z["dt_next"])
        out["params"] = json.loads(str(z["params"]))
    return out
