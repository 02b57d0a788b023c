"""Seeded initial state on the GPU (pimd_init_state / pimd_batch_init_state)
against the oracle's generator (oracle/rng.py): same counters, same streams.

Both sides draw the same splitmix64 words (bit-exact integer work); the
normal deviates then differ only by the rounding of log, sqrt and cos, so
beads and momenta agree to 1e-13 absolute (|z| < 9).  The forces computed
after the draw match the oracle's forces of the drawn beads (1e-10).
"""
import numpy as np
import pytest

import oracle
from oracle import rng
from gpu_common import amplitude, rel_inf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,P,d,beta,seed", [(1, 4, 2, 1.0, 0), (37, 8, 2, 2.0, 5), (300, 6, 3, 0.7, 2**63 + 11),
                                             (1600, 32, 2, 3.0, 3)])
def test_init_state_matches_oracle(N, P, d, beta, seed):
    import paper_2404_02628_gb300 as pkg
    g, s, xi = 3.0, 0.5, 1.0
    S = pkg.System(N, P, d, beta, 1.0, g, s, xi)
    S.init_state(seed)
    r_o, p_o = rng.init_state(N, P, d, beta, seed)
    assert np.abs(S.positions() - r_o).max() < 1e-13
    assert np.abs(S.momenta() - p_o).max() < 1e-13
    assert S.estimators()["step"] == 0
    if N <= 300:
        Fo, _ = oracle.forces(r_o, beta, xi, 1.0, amplitude(g, s), s)
        assert rel_inf(S.forces_array(), Fo) < 1e-10
    # padding columns are zero
    assert float(S.r[:, :, N:].abs().max() if S.n_pad > N else 0.0) == 0.0
    S.step(3)
    assert np.isfinite(S.positions()).all()
    S.close()


def test_init_state_is_deterministic():
    import paper_2404_02628_gb300 as pkg
    A = pkg.System(50, 8, 2, 2.0, 1.0, 3.0, 0.5, 1.0)
    B = pkg.System(50, 8, 2, 2.0, 1.0, 3.0, 0.5, 1.0)
    A.init_state(77)
    B.init_state(77)
    A.step(10)
    B.step(10)
    assert np.array_equal(A.positions(), B.positions())
    B.init_state(78)
    assert not np.array_equal(A.positions(), B.positions())
    A.close()
    B.close()


def test_batch_init_state_matches_oracle():
    import paper_2404_02628_gb300 as pkg
    Ns, P, d = [40, 7, 129], 8, 2
    betas, xis = [1.0, 2.0, 3.0], [1.0, 0.0, 0.5]
    B = pkg.Batch(Ns, P, d, betas, xis, 1.0, 3.0, 0.5)
    B.init_state(2024)
    for q, N in enumerate(Ns):
        r_o, p_o = rng.init_state(N, P, d, betas[q], rng.replica_seed(2024, q))
        assert np.abs(B.positions(q) - r_o).max() < 1e-13
        assert np.abs(B.momenta(q) - p_o).max() < 1e-13
        Fo, _ = oracle.forces(r_o, betas[q], xis[q], 1.0, amplitude(3.0, 0.5), 0.5)
        assert rel_inf(B.forces_array(q), Fo) < 1e-10
    B.step(2)
    B.close()
