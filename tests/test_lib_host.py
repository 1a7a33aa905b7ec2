"""CPU checks of the C-ABI library: it loads, exports every symbol declared in include/bie.h, and its
host-side plan tables agree with the oracle (no GPU needed)."""
import os
import re

import numpy as np
import pytest

from oracle import layer, sh, wigner
from paper_1707_02156_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return api.lib()


def test_exports_match_header(L):
    hdr = open(os.path.join(ROOT, "include", "bie.h")).read()
    names = set(re.findall(r"\b(bie_[a-z_0-9]+)\s*\(", hdr))
    assert names, "no declarations found"
    for n in sorted(names):
        assert hasattr(L, n), n
    assert names == set(api.EXPORTS), sorted(names ^ set(api.EXPORTS))


def test_gauss_legendre_nodes(L):
    for P in (0, 5, 16, 65, 131):
        v = np.array(api.debug_table(0, P))
        t, w = v[:P + 1], v[P + 1:]
        tr, wr = sh.gauss_legendre(P + 1)
        assert np.max(np.abs(t - tr)) <= 2.3e-16
        assert np.max(np.abs(w - wr) / wr) <= 4.5e-16


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_legendre_tables_match_oracle(L, kind):
    p, P = 12, 25
    v = np.array(api.debug_table(1, p, kind, P))
    _, _, theta, _ = sh.gauss_grid(P)
    tabs = sh.legendre_dtheta(p, theta)
    ref = tabs[kind]
    i = 0
    for m in range(p + 1):
        for n in range(m, p + 1):
            assert np.max(np.abs(v[i:i + P + 1] - ref[n, m])) < 1e-12 * max(1, n * n), (m, n)
            i += P + 1


def test_wigner_small_d_matches_oracle(L):
    for n in (0, 1, 7, 32, 48):
        for beta in (0.05, 1.3, 3.05, -0.7):
            v = np.array(api.debug_table(2, n, x=beta)).reshape(2 * n + 1, 2 * n + 1)
            assert np.max(np.abs(v - wigner.small_d(n, beta))) < 2e-13


def test_singular_weights_match_oracle(L):
    for pq in (8, 33, 65):
        v = np.array(api.debug_table(3, pq))
        assert np.max(np.abs(v - layer.singular_weights(pq))) < 1e-14


def test_null_arguments_are_rejected_before_any_device_work(L):
    # every entry point checks its handles and pointers first: BIE_EINVAL (1), no CUDA call made
    import ctypes
    EINVAL = 1
    o = api.bie_solve_opts()
    L.bie_solve_opts_default(ctypes.byref(o))
    info = api.bie_solve_info()
    p = (ctypes.c_int * 1)(8)
    lam = (ctypes.c_double * 1)(1.0)
    assert L.bie_apply_single(None, None, None, None, 0, None) == EINVAL
    assert L.bie_apply_double(None, None, None, None, 0, None) == EINVAL
    assert L.bie_rhs(None, None, None, None, None, 0, None) == EINVAL
    assert L.bie_eval_single(None, None, 4, None, None, None, 0, None) == EINVAL
    assert L.bie_eval_double(None, None, 4, None, None, None, 0, None) == EINVAL
    assert L.bie_eval_velocity(None, None, 4, None, None, None, None, None, 0, None) == EINVAL
    assert L.bie_solve(None, None, None, None, ctypes.byref(o), ctypes.byref(info), None) == EINVAL
    assert L.bie_step_midpoint(None, 1, p, p, None, None, 0.2, 0.0, lam, 1.0, 0.01, ctypes.byref(o), None,
                               None) == EINVAL
    # surfactant entry points
    x = ctypes.c_void_p(16)
    cinfo = api.bie_coupled_info()
    rinfo = api.bie_run_info()
    assert L.bie_surfactant_rates(None, 1, p, x, x, x, 0.1, x, None, None) == EINVAL
    assert L.bie_surfactant_rates(None, 1, p, None, x, x, 0.1, x, None, None) == EINVAL
    assert L.bie_surfactant_implicit(None, 1, p, x, x, 0.1, x, 1e-13, None, None) == EINVAL
    assert L.bie_surfactant_mass(None, 1, p, x, x, None, None) == EINVAL
    assert L.bie_step_coupled(None, 1, p, p, x, x, x, 0, 0.2, 0.0, lam, 1.0, 0.1, 0.01, 0, ctypes.byref(o), x, x,
                              ctypes.byref(cinfo), None) == EINVAL
    assert L.bie_run_coupled(None, 1, p, p, x, x, 0.2, 0.0, lam, 1.0, 0.1, 1.0, 0.1, 1e-5, 0.1, 0, 10,
                             ctypes.byref(o), None, ctypes.byref(rinfo), None) == EINVAL
    # angle reparametrisation: null handles, then options out of range
    ro = api.bie_reparam_opts()
    L.bie_reparam_opts_default(ctypes.byref(ro))
    assert (ro.u_rep, ro.p_cutoff, ro.smooth, ro.dtau, ro.eps, ro.max_iter) == (2, 0.05, 0, 0.5, 1e-10, 200)
    pinfo = api.bie_reparam_info()
    assert L.bie_reparametrize(None, 1, p, x, x, ctypes.byref(ro), ctypes.byref(pinfo), None) == EINVAL
    assert L.bie_reparametrize(ctypes.c_void_p(16), 1, p, None, x, ctypes.byref(ro), ctypes.byref(pinfo),
                               None) == EINVAL
    for field, bad in (("u_rep", 0), ("p_cutoff", 1.0), ("dtau", 0.0), ("eps", -1.0)):
        r2 = api.bie_reparam_opts()
        L.bie_reparam_opts_default(ctypes.byref(r2))
        setattr(r2, field, bad)
        assert L.bie_reparametrize(ctypes.c_void_p(16), 1, p, x, x, ctypes.byref(r2), ctypes.byref(pinfo),
                                   None) == EINVAL, field
    # status strings
    assert L.bie_strerror(0) == b"ok"
    assert L.bie_strerror(EINVAL) == b"invalid argument"


def test_step_size_rule_matches_oracle(L):
    # Alg. 1: dt (0.9 tol/err)^(1/2), capped at dt_max; dt_max when err is zero
    from oracle import surfactant as sf
    for dt, err, tol, dt_max in ((0.1, 4e-5, 1e-5, 1.0), (0.02, 1e-9, 1e-6, 0.05), (0.3, 2e-3, 1e-4, 1.0),
                                 (0.1, 0.0, 1e-5, 0.2)):
        assert api.next_dt(dt, err, tol, dt_max) == pytest.approx(sf.next_dt(dt, err, tol, dt_max), rel=1e-15)
