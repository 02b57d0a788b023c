"""CUDA path against the FP64 oracle on identical seeded configurations.

Tolerances: FP64 forces and energies 1e-10 relative (infinity norm over all
beads for forces); mixed precision (FP32 springs and pairs) 1e-5 relative.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_common import amplitude, make_system, rel_inf
from workloads import beads, momenta

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-5

# (N, P, d, beta, xi): single tile, exact tiles, ragged tails, several tiles
EXCH_CASES = [(1, 4, 2, 1.0, 1.0), (2, 3, 2, 1.0, 0.5), (5, 8, 2, 2.0, 1.0), (31, 4, 2, 1.5, 1.0),
              (32, 4, 2, 1.5, 0.7), (33, 6, 3, 1.0, 1.0), (64, 5, 1, 2.0, 1.0), (100, 8, 2, 3.0, 1.0),
              (257, 4, 2, 2.0, 0.3), (300, 6, 2, 1.0, 1.0), (130, 4, 2, 2.0, 0.0), (200, 4, 2, 1.0, 1e-3)]


@pytest.mark.parametrize("arith", ["df", "fp64"])
@pytest.mark.parametrize("table", ["store", "recompute"])
@pytest.mark.parametrize("N,P,d,beta,xi", EXCH_CASES)
def test_exchange_forces_and_potential(N, P, d, beta, xi, table, arith):
    import paper_2404_02628_gb300 as pkg
    r = beads(N, P, d, 100 + N)
    mode = pkg.TABLE_STORE if table == "store" else pkg.TABLE_RECOMPUTE
    ar = pkg.XARITH_DF if arith == "df" else pkg.XARITH_FP64
    S = make_system(N, P, d, beta, 0.0, 0.0, 0.5, xi, r, table_mode=mode, exchange_arith=ar)
    F, V = S.exchange_forces()
    Fo, info = oracle.forces(r, beta, xi, 0.0, 0.0, 0.5)
    assert rel_inf(F, Fo) < TOL64
    assert abs(V - info["V_xi"]) < TOL64 * abs(info["V_xi"])
    est = S.estimators()
    assert abs(est["V_xi_bwd"] - info["V_xi_bwd"]) < TOL64 * abs(info["V_xi"])
    assert abs(est["spring"] - info["spring"]) < TOL64 * abs(info["spring"])
    S.close()


@pytest.mark.parametrize("N,P,d", [(40, 8, 2), (300, 4, 2), (129, 4, 3)])
def test_first_launch_with_force_workers(N, P, d):
    """The forces formed when the buffers are bound -- the first recursion
    launch on a workspace that still holds another system's factors and
    operators -- match the oracle with force workers in the launch: no item
    reads a factor tile, operator or band tile before this launch wrote it."""
    import paper_2404_02628_gb300 as pkg
    beta, xi, g, s = 2.0, 1.0, 3.0, 0.5
    # leave another configuration's workspace in the allocator's cache
    T = make_system(N, P, d, 3.0, 1.0, 1.0, s, 0.5, beads(N, P, d, 7))
    T.step(2)
    T.close()
    del T
    r = beads(N, P, d, 130 + N)
    S = make_system(N, P, d, beta, 1.0, g, s, xi, r)
    assert S.tuning()["force_blocks"] > 0
    Fo, _ = oracle.forces(r, beta, xi, 1.0, amplitude(g, s), s)
    assert rel_inf(S.forces_array(), Fo) < TOL64
    S.close()


@pytest.mark.parametrize("W", [2, 3, 4, 5])
@pytest.mark.parametrize("N,xi", [(700, 1.0), (450, 0.5)])
def test_exchange_band_widths(N, xi, W):
    """The double-float recursion gives the same forces for every look-ahead width."""
    P, d, beta = 4, 2, 2.0
    r = beads(N, P, d, 150 + N)
    S = make_system(N, P, d, beta, 0.0, 0.0, 0.5, xi, r, exch_band=W)
    F, V = S.exchange_forces()
    Fo, info = oracle.forces(r, beta, xi, 0.0, 0.0, 0.5)
    assert rel_inf(F, Fo) < TOL64
    assert abs(V - info["V_xi"]) < TOL64 * abs(info["V_xi"])
    S.close()


@pytest.mark.parametrize("N,P,d", [(1, 4, 2), (50, 8, 2), (129, 4, 3), (300, 4, 1)])
def test_interaction_fp64(N, P, d):
    beta, g, s, om = 2.0, 3.0, 0.5, 1.3
    r = beads(N, P, d, 200 + N)
    S = make_system(N, P, d, beta, om, g, s, 1.0, r)
    F, U = S.interaction_forces()
    Uo, Fo, vir = oracle.interaction(r, om, amplitude(g, s), s)
    assert rel_inf(F, Fo) < TOL64
    assert abs(U - Uo / P) < TOL64 * abs(Uo / P)
    S.close()


@pytest.mark.parametrize("N,P,d", [(50, 8, 2), (300, 4, 2), (129, 4, 3)])
def test_interaction_mixed(N, P, d):
    import paper_2404_02628_gb300 as pkg
    beta, g, s, om = 2.0, 3.0, 0.5, 1.0
    r = beads(N, P, d, 300 + N)
    S = make_system(N, P, d, beta, om, g, s, 1.0, r, precision=pkg.PREC_MIXED)
    F, U = S.interaction_forces()
    Uo, Fo, vir = oracle.interaction(r, om, amplitude(g, s), s)
    assert rel_inf(F, Fo) < TOLMIX
    assert abs(U - Uo / P) < TOLMIX * abs(Uo / P)
    S.close()


@pytest.mark.parametrize("N,P,d,beta,xi,g", [(16, 32, 2, 2.0, 1.0, 0.0), (100, 8, 2, 3.0, 1.0, 3.0),
                                             (70, 6, 2, 1.0, 0.4, 1.0)])
def test_total_forces_and_estimators(N, P, d, beta, xi, g):
    s, om = 0.5, 1.0
    r = beads(N, P, d, 400 + N)
    p = momenta(N, P, d, beta, 400 + N)
    S = make_system(N, P, d, beta, om, g, s, xi, r, p)
    V = S.forces()
    F = S.forces_array()
    A = amplitude(g, s)
    Fo, info = oracle.forces(r, beta, xi, om, A, s)
    assert rel_inf(F, Fo) < TOL64
    assert abs(V - (info["V_xi"] + info["U_over_P"])) < TOL64 * abs(V)
    est = S.estimators()
    st = oracle.MDState(r, p, 4)
    oe = oracle.estimators(st, beta, xi, om, A, s, beta / P)
    for k in ("E_prim", "E_vir", "V_xi", "U_over_P", "kinetic", "spring", "virial", "H_conserved"):
        assert abs(est[k] - oe[k]) < TOL64 * max(1.0, abs(oe[k])), (k, est[k], oe[k])
    S.close()


@pytest.mark.parametrize("thermostat", [1, 0])
def test_md_steps_match_oracle(thermostat):
    N, P, d, beta, xi, g, s = 40, 8, 2, 2.0, 1.0, 3.0, 0.5
    r = beads(N, P, d, 501)
    p = momenta(N, P, d, beta, 501)
    S = make_system(N, P, d, beta, 1.0, g, s, xi, r, p, thermostat=thermostat)
    nsteps = 5
    S.step(nsteps)
    st = oracle.MDState(r, p, 4)
    oest = oracle.md_run(st, beta, xi, 1.0, amplitude(g, s), s, 0.01, beta / P, nsteps,
                         thermostat=bool(thermostat))
    assert rel_inf(S.positions(), st.r) < 1e-11
    assert rel_inf(S.momenta(), st.p) < 1e-10
    est = S.estimators()
    for k in ("E_prim", "E_vir", "H_conserved"):
        o = oest[-1, oracle.ESTIMATE_FIELDS.index(k)]
        assert abs(est[k] - o) < 1e-9 * abs(o), (k, est[k], o)
    assert est["step"] == nsteps
    S.close()


def test_graph_and_eager_steps_are_bitwise_equal():
    N, P, d, beta = 70, 8, 2, 2.0
    r = beads(N, P, d, 601)
    p = momenta(N, P, d, beta, 601)
    A = make_system(N, P, d, beta, 1.0, 3.0, 0.5, 0.8, r, p)
    B = make_system(N, P, d, beta, 1.0, 3.0, 0.5, 0.8, r, p)
    A.step(20, graph=True)
    B.step(20, graph=False)
    assert np.array_equal(A.positions(), B.positions())
    assert np.array_equal(A.momenta(), B.momenta())
    A.close()
    B.close()


def test_checkpoint_resume_bitwise():
    N, P, d, beta = 50, 8, 2, 2.0
    r = beads(N, P, d, 701)
    p = momenta(N, P, d, beta, 701)
    A = make_system(N, P, d, beta, 1.0, 3.0, 0.5, 1.0, r, p)
    A.step(40)
    B = make_system(N, P, d, beta, 1.0, 3.0, 0.5, 1.0, r, p)
    B.step(20)
    blob = B.get_state()
    B.close()
    C = make_system(N, P, d, beta, 1.0, 3.0, 0.5, 1.0, r, p)
    C.set_state(blob)
    C.step(20)
    assert np.array_equal(A.positions(), C.positions())
    assert np.array_equal(A.momenta(), C.momenta())
    assert C.estimators()["step"] == 40
    A.close()
    C.close()


def test_bounded_wait_reports_timeout_and_context_survives():
    """A one-poll wait limit makes the recursion's cross-block waits give up
    (their flags are not set yet); the call returns PIMD_ETIMEOUT and a fresh
    context on the same device still works."""
    import paper_2404_02628_gb300 as pkg
    N, P, d, beta = 2000, 4, 2, 2.0
    r = beads(N, P, d, 801)
    with pytest.raises(pkg.PimdError) as ei:
        S = make_system(N, P, d, beta, 0.0, 0.0, 0.5, 1.0, r, spin_limit=1)
        S.forces()
    assert ei.value.status == pkg.PIMD_ETIMEOUT
    T = make_system(64, P, d, beta, 0.0, 0.0, 0.5, 1.0, beads(64, P, d, 802))
    F, V = T.exchange_forces()
    Fo, info = oracle.forces(beads(64, P, d, 802), beta, 1.0, 0.0, 0.0, 0.5)
    assert rel_inf(F, Fo) < TOL64
    T.close()


def test_nonfinite_is_reported():
    import paper_2404_02628_gb300 as pkg
    N, P, d = 20, 4, 2
    r = beads(N, P, d, 901)
    r[3, 1, 0] = np.nan
    S = make_system(N, P, d, 2.0, 1.0, 0.0, 0.5, 1.0, r)
    with pytest.raises(pkg.PimdError) as ei:
        S.estimators()
    assert ei.value.status == pkg.PIMD_ENONFINITE
    S.close()
