"""Autotuner: every candidate launch shape gives the same forces, a tuned
system still matches the oracle, and the cache round-trips."""
import numpy as np
import pytest

import oracle
from gpu_common import amplitude, rel_inf
from workloads import beads

pytestmark = pytest.mark.gpu


def test_autotune_keeps_oracle_parity_and_caches(tmp_path):
    import paper_2404_02628_gb300 as pkg
    N, P, d, beta, xi, g, s = 700, 8, 2, 2.0, 1.0, 3.0, 0.5
    r = beads(N, P, d, 1700)
    cache = str(tmp_path / "tune.txt")
    S = pkg.System(N, P, d, beta, 1.0, g, s, xi, r=r)
    t = S.autotune(cache)
    assert 2 <= t["exch_band"] <= 5 and t["pair_block"] in (64, 128, 256)
    Fo, _ = oracle.forces(r, beta, xi, 1.0, amplitude(g, s), s)
    assert rel_inf(S.forces_array(), Fo) < 1e-10
    S.step(3)  # the step graph is captured with the tuned shapes
    S.close()
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and "W=%d;pair_t=%d" % (t["exch_band"], t["pair_block"]) in lines[0]
    S2 = pkg.System(N, P, d, beta, 1.0, g, s, xi, r=r)
    assert S2.autotune(cache) == t           # read back, not re-timed
    assert len(open(cache).read().splitlines()) == 1
    S2.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-6)])
def test_every_candidate_gives_the_same_forces(tmp_path, prec, tol):
    import paper_2404_02628_gb300 as pkg
    N, P, d, beta, xi, g, s = 500, 6, 2, 1.5, 0.8, 3.0, 0.5
    r = beads(N, P, d, 1710)
    ref = None
    for W in (2, 3, 4, 5):
        for T in (64, 128, 256):
            S = pkg.System(N, P, d, beta, 1.0, g, s, xi, r=r, precision=prec)
            key_probe = str(tmp_path / ("probe_%d_%d.txt" % (W, T)))
            S.autotune(key_probe)  # learn the cache key of this problem
            key = open(key_probe).read().split("|")[0]
            forced = str(tmp_path / ("forced_%d_%d.txt" % (W, T)))
            open(forced, "w").write("%s|W=%d;pair_t=%d\n" % (key, W, T))
            assert S.autotune(forced) == {"exch_band": W, "pair_block": T}
            F = S.forces_array()
            S.close()
            if ref is None:
                ref = F
            else:
                assert rel_inf(F, ref) < tol, (W, T)


def test_batch_autotune_keeps_oracle_parity(tmp_path):
    import paper_2404_02628_gb300 as pkg
    reps = [(300, 1.0, 1.0), (77, 2.0, 0.0), (512, 3.0, 0.5)]
    P, d, g, s = 8, 2, 3.0, 0.5
    Ns = [n for n, _, _ in reps]
    rs = [beads(n, P, d, 1720 + q) for q, n in enumerate(Ns)]
    B = pkg.Batch(Ns, P, d, [b for _, b, _ in reps], [x for _, _, x in reps], 1.0, g, s, rs=rs)
    cache = str(tmp_path / "btune.txt")
    B.autotune(cache)
    assert open(cache).read().count("pair_t=") == 1
    for q, (N, beta, xi) in enumerate(reps):
        Fo, _ = oracle.forces(rs[q], beta, xi, 1.0, amplitude(g, s), s)
        assert rel_inf(B.forces_array(q), Fo) < 1e-10, q
    B.step(2)
    B.autotune(cache)  # cache hit
    assert open(cache).read().count("pair_t=") == 1
    B.close()
