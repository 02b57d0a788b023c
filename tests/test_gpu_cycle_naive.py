"""The O(N^3 P) debug evaluation of the cycle energies (one GPU thread per
E^[u,v], straight from the ring-of-springs definition, Sec. III) against the
oracle's quadratic iteration of Sec. III -- two independent routes to the
same table -- from tiny N to the benchmarked size N = 1600, P = 32."""
import numpy as np
import pytest

import oracle
from workloads import beads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,P,d,beta", [(1, 2, 2, 1.0), (7, 3, 1, 1.3), (33, 5, 3, 0.7), (257, 8, 2, 2.0),
                                        (1600, 32, 2, 3.0)])
def test_naive_cycle_energies_match_oracle_iteration(N, P, d, beta):
    import paper_2404_02628_gb300 as pkg
    r = beads(N, P, d, 2500 + N)
    S = pkg.System(N, P, d, beta, 1.0, 0.0, 0.5, 1.0, r=r)
    E = S.cycle_energies_naive()
    S.close()
    Eo = oracle.cycle_energies(r, beta)
    iu = np.triu_indices(N)
    scale = np.maximum(1.0, np.abs(Eo[iu]))
    assert float(np.max(np.abs(E[iu] - Eo[iu]) / scale)) < 1e-11
    assert not np.any(np.tril(E, -1))  # below the diagonal nothing is written
