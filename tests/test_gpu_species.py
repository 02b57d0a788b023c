"""Several species on the GPU (Sec. II, closing paragraph): one exchange
recursion per species, trap and pairs between all particles.  Forces,
potential and estimators against the oracle's species composition; a long
run of two ideal species against the sum of their exact energies."""
import numpy as np
import pytest

import oracle
from gpu_common import amplitude, rel_inf
from oracle import exact
from workloads import beads, momenta

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("counts,P,d,beta,xi,g", [([37, 63], 8, 2, 2.0, 1.0, 3.0), ([1, 128, 128], 4, 2, 1.5, 0.5, 1.0),
                                                 ([32, 32], 6, 3, 1.0, 0.5, 0.0), ([20, 50], 4, 1, 2.0, 0.0, 2.0),
                                                 ([300, 700], 8, 2, 3.0, 1.0, 1.0)])
@pytest.mark.parametrize("prec,arith", [(0, 0), (0, 1), (1, 0)])
def test_species_forces_and_estimators_match_oracle(counts, P, d, beta, xi, g, prec, arith):
    import paper_2404_02628_gb300 as pkg
    N, s = sum(counts), 0.5
    r = beads(N, P, d, 2600 + N)
    S = pkg.System(N, P, d, beta, 1.0, g, s, xi, r=r, species=counts, precision=prec, exchange_arith=arith)
    V = S.forces()
    F = S.forces_array()
    est = S.estimators()
    S.close()
    Fo, info = oracle.forces_species(r, counts, beta, xi, 1.0, amplitude(g, s), s)
    tol = 1e-10 if prec == 0 else 1e-5
    assert rel_inf(F, Fo) < tol
    assert abs(est["V_xi"] - info["V_xi"]) < 1e-10 * max(1.0, abs(info["V_xi"]))
    assert abs(est["V_xi_bwd"] - info["V_xi"]) < 1e-10 * max(1.0, abs(info["V_xi"]))
    assert abs(est["spring"] - info["spring"]) < 1e-10 * max(1.0, abs(info["spring"]))
    Vo = info["V_xi"] + info["U_over_P"]
    assert abs(V - Vo) < tol * max(1.0, abs(Vo))


def test_species_exchange_forces_and_autotune(tmp_path):
    import paper_2404_02628_gb300 as pkg
    counts, P, d, beta, xi, g, s = [150, 250], 8, 2, 2.0, 0.8, 2.0, 0.5
    N = sum(counts)
    r = beads(N, P, d, 2700)
    S = pkg.System(N, P, d, beta, 1.0, g, s, xi, r=r, species=counts)
    t = S.autotune(str(tmp_path / "tune.txt"))
    assert t["force_blocks"] == 0  # several species: springs and pairs as kernels of their own
    S.forces()
    Fo, info = oracle.forces_species(r, counts, beta, xi, 1.0, amplitude(g, s), s)
    assert rel_inf(S.forces_array(), Fo) < 1e-10
    Fx, Vx = S.exchange_forces()
    Fxo, ix = oracle.forces_species(r, counts, beta, xi, 0.0, 0.0, s)
    assert rel_inf(Fx, Fxo) < 1e-10
    assert abs(Vx - ix["V_xi"]) < 1e-10 * abs(ix["V_xi"])
    S.step(3)  # graph-captured steps run with several recursions
    x = S.positions()
    F3, _ = oracle.forces_species(x, counts, beta, xi, 1.0, amplitude(g, s), s)
    assert rel_inf(S.forces_array(), F3) < 1e-10
    S.close()


def test_two_species_long_run_matches_exact():
    """16 trapped ideal bosons as two species of 8 (spin-unpolarised), P = 32,
    beta = 2, FP64: E_prim and E_vir average to 2 E_8 = 16.919 (one species
    of 16 would give 16.455, distinguishable particles 21.000)."""
    import paper_2404_02628_gb300 as pkg
    N, P, d, beta = 16, 32, 2, 2.0
    r = beads(N, P, d, 2800)
    p = momenta(N, P, d, beta, 2800)
    S = pkg.System(N, P, d, beta, 1.0, 0.0, 0.5, 1.0, r=r, p=p, species=[8, 8], precision=pkg.PREC_FP64)
    S.step(10000)
    n_samples, stride = 30000, 10
    Ep = np.empty(n_samples)
    Ev = np.empty(n_samples)
    for i in range(n_samples):
        S.step(stride)
        est = S.estimators()
        Ep[i], Ev[i] = est["E_prim"], est["E_vir"]
    S.close()
    E_exact = 2 * exact.energy(8, beta, P=P, d=d, xi=1.0)
    for series in (Ev, Ep):
        blocks = series.reshape(20, -1).mean(axis=1)
        mean, se = blocks.mean(), blocks.std(ddof=1) / np.sqrt(20)
        print("two species: %.4f +- %.4f, exact %.4f" % (mean, se, E_exact))
        assert se < 0.03 * E_exact
        assert abs(mean - E_exact) < 4 * se
