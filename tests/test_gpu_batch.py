"""Batched replicas (uneven N, beta, xi) against the FP64 oracle, replica by replica.

Every replica of a batch must give what the oracle gives for that system on
its own: FP64 forces and energies to 1e-10 relative, mixed precision (FP32
springs and pairs) to 1e-5.
"""
import numpy as np
import pytest

import oracle
from gpu_common import amplitude, rel_inf
from workloads import beads, momenta

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-5

# (N, beta, xi): one particle, ragged and exact tiles, xi = 0, tiny xi, several chunks
REPLICAS = [(1, 1.0, 1.0), (31, 2.0, 0.0), (33, 3.0, 0.6), (100, 1.5, 1.0), (257, 2.0, 0.2),
            (64, 4.0, 1e-3), (200, 1.0, 1.0), (32, 2.5, 1.0)]


def make_batch(reps, P, d, omega, g, s, seed, **cfg):
    import paper_2404_02628_gb300 as pkg
    Ns = [n for n, _, _ in reps]
    betas = [b for _, b, _ in reps]
    xis = [x for _, _, x in reps]
    rs = [beads(n, P, d, seed + 7 * q) for q, n in enumerate(Ns)]
    ps = [momenta(n, P, d, b, seed + 7 * q) for q, (n, b) in enumerate(zip(Ns, betas))]
    B = pkg.Batch(Ns, P, d, betas, xis, omega, g, s, rs=rs, ps=ps, **cfg)
    return B, rs, ps


@pytest.mark.parametrize("P,d,g", [(4, 2, 0.0), (6, 3, 3.0), (5, 1, 1.0)])
def test_batch_forces_match_oracle(P, d, g):
    s, omega = 0.5, 1.0
    B, rs, _ = make_batch(REPLICAS, P, d, omega, g, s, 900)
    est = B.estimators()
    A = amplitude(g, s)
    for q, (N, beta, xi) in enumerate(REPLICAS):
        Fo, info = oracle.forces(rs[q], beta, xi, omega, A, s)
        assert rel_inf(B.forces_array(q), Fo) < TOL64, q
        assert abs(est[q]["V_xi"] - info["V_xi"]) < TOL64 * max(1.0, abs(info["V_xi"])), q
        assert abs(est[q]["V_xi_bwd"] - info["V_xi_bwd"]) < TOL64 * max(1.0, abs(info["V_xi"])), q
        assert abs(est[q]["U_over_P"] - info["U_over_P"]) < TOL64 * max(1.0, abs(info["U_over_P"])), q
        assert abs(est[q]["spring"] - info["spring"]) < TOL64 * abs(info["spring"]), q
    B.close()


@pytest.mark.parametrize("N,xi", [(700, 1.0), (1000, 0.5), (2047, 1.0)])
def test_batch_many_chunks(N, xi):
    """Large replicas: the self-contained recursion streams many tile chunks per block."""
    P, d, beta = 4, 2, 2.0
    reps = [(N, beta, xi), (45, 1.0, 1.0)]
    B, rs, _ = make_batch(reps, P, d, 0.0, 0.0, 0.5, 950)
    for q, (n, b, x) in enumerate(reps):
        Fo, info = oracle.forces(rs[q], b, x, 0.0, 0.0, 0.5)
        assert rel_inf(B.forces_array(q), Fo) < TOL64, q
    B.close()


def test_batch_matches_single_system():
    """A replica in a batch and the same system on its own give the same forces."""
    import paper_2404_02628_gb300 as pkg
    P, d, g, s = 8, 2, 3.0, 0.5
    B, rs, _ = make_batch(REPLICAS[2:6], P, d, 1.0, g, s, 980)
    for q, (N, beta, xi) in enumerate(REPLICAS[2:6]):
        S = pkg.System(N, P, d, beta, 1.0, g, s, xi, r=rs[q])
        S.forces()
        assert rel_inf(B.forces_array(q), S.forces_array()) < 1e-11, q
        S.close()
    B.close()


@pytest.mark.parametrize("thermostat", [1, 0])
def test_batch_md_matches_oracle(thermostat):
    P, d, g, s, dt, nsteps = 8, 2, 3.0, 0.5, 0.01, 5
    reps = [(40, 2.0, 1.0), (17, 1.0, 0.5), (70, 3.0, 0.0)]
    B, rs, ps = make_batch(reps, P, d, 1.0, g, s, 990, thermostat=thermostat)
    B.step(nsteps)
    est = B.estimators()
    for q, (N, beta, xi) in enumerate(reps):
        st = oracle.MDState(rs[q], ps[q], 4)
        oest = oracle.md_run(st, beta, xi, 1.0, amplitude(g, s), s, dt, beta / P, nsteps,
                             thermostat=bool(thermostat))
        assert rel_inf(B.positions(q), st.r) < 1e-11, q
        assert rel_inf(B.momenta(q), st.p) < 1e-10, q
        for k in ("E_prim", "E_vir", "H_conserved"):
            o = oest[-1, oracle.ESTIMATE_FIELDS.index(k)]
            assert abs(est[q][k] - o) < 1e-9 * abs(o), (q, k, est[q][k], o)
        assert est[q]["step"] == nsteps
    B.close()


def test_batch_graph_and_eager_bitwise():
    P, d = 8, 2
    A, _, _ = make_batch(REPLICAS[:5], P, d, 1.0, 3.0, 0.5, 1010)
    C, _, _ = make_batch(REPLICAS[:5], P, d, 1.0, 3.0, 0.5, 1010)
    A.step(10, graph=True)
    C.step(10, graph=False)
    for q in range(5):
        assert np.array_equal(A.positions(q), C.positions(q))
        assert np.array_equal(A.momenta(q), C.momenta(q))
    A.close()
    C.close()


def test_batch_mixed_precision():
    import paper_2404_02628_gb300 as pkg
    P, d, g, s = 32, 2, 3.0, 0.5
    reps = [(300, 1.0, 0.0), (150, 2.0, 0.4), (512, 3.0, 1.0), (40, 4.0, 0.8)]
    B, rs, _ = make_batch(reps, P, d, 1.0, g, s, 1020, precision=pkg.PREC_MIXED)
    for q, (N, beta, xi) in enumerate(reps):
        Fo, _ = oracle.forces(rs[q], beta, xi, 1.0, amplitude(g, s), s)
        assert rel_inf(B.forces_array(q), Fo) < TOLMIX, q
    B.close()


def test_batch_fp32_thermostat_tracks_fp64():
    """nhc_fp32 (mixed mode): 20 steps stay within 1e-4 of the FP64 thermostat run."""
    import paper_2404_02628_gb300 as pkg
    P, d, g, s = 16, 2, 3.0, 0.5
    reps = [(120, 1.0, 1.0), (60, 3.0, 0.4)]
    A, _, _ = make_batch(reps, P, d, 1.0, g, s, 1030, precision=pkg.PREC_MIXED)
    C, _, _ = make_batch(reps, P, d, 1.0, g, s, 1030, precision=pkg.PREC_MIXED, nhc_fp32=1)
    A.step(20)
    C.step(20)
    ea, ec = A.estimators(), C.estimators()
    for q in range(len(reps)):
        assert rel_inf(C.momenta(q), A.momenta(q)) < 1e-4, q
        assert rel_inf(C.positions(q), A.positions(q)) < 1e-6, q
        assert abs(ec[q]["H_conserved"] - ea[q]["H_conserved"]) < 1e-5 * abs(ea[q]["H_conserved"]), q
    A.close()
    C.close()
