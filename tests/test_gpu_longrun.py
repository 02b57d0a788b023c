"""Long-run check: MD averages of the energy estimators on the GPU against the
exact canonical energy of non-interacting trapped bosons.

N = 16, d = 2, P = 32, beta = 2, omega = 1, FP64, massive NHC (M = 4),
dt = 0.01, beads ~ N(0,1) (seed 1).  The exact finite-P energy comes from the
recursion Z_N = (1/N) sum_k xi^(k-1) z_P(k) Z_{N-k} (oracle.exact, pinned to
the N! permutation sum in the oracle tests): 16.4554 for xi = 1 and 21.0002 for
xi = 0, so the two settings differ by 28 % and a wrong exchange weight, a wrong
temperature or a broken thermostat shows far outside the error bars.  Averages
use blocks of the sampled series; the check is |mean - exact| < 4 standard
errors of the block means, with the standard error itself below 3 % of E (200k steps).
For xi = 0 the radial bead density averaged over the run is also checked, bin
by bin (5 standard errors), against the exact Gaussian density of a bead of a
distinguishable trapped ring polymer.
"""
import numpy as np
import pytest

from oracle import exact
from workloads import beads, momenta

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("xi", [1.0, 0.0])
def test_long_run_energy_matches_exact(xi):
    import paper_2404_02628_gb300 as pkg
    N, P, d, beta = 16, 32, 2, 2.0
    r = beads(N, P, d, 1)
    p = momenta(N, P, d, beta, 1)
    S = pkg.System(N, P, d, beta, 1.0, 0.0, 0.5, xi, r=r, p=p, precision=pkg.PREC_FP64, nhc_len=4, dt=0.01)
    S.step(10000)  # equilibration, discarded
    n_samples, stride = 20000, 10
    Ep = np.empty(n_samples)
    Ev = np.empty(n_samples)
    nbins, r_max, nblk = 24, 4.0, 20
    hist = [S.torch.zeros(nbins, dtype=S.torch.float64, device="cuda") for _ in range(nblk)]
    for i in range(n_samples):
        S.step(stride)
        S.density(nbins, r_max, hist[i * nblk // n_samples])
        est = S.estimators()
        Ep[i], Ev[i] = est["E_prim"], est["E_vir"]
    S.close()
    if xi == 0.0:
        # distinguishable particles: every bead is an isotropic Gaussian of
        # variance exact.bead_variance per coordinate, so the averaged
        # density must match the exact shell probabilities per volume
        var = exact.bead_variance(beta, P)
        rho = np.stack([h.cpu().numpy() for h in hist]) / (n_samples // nblk)
        dr = r_max / nbins
        for b in range(nbins):
            V = np.pi * (((b + 1) * dr) ** 2 - (b * dr) ** 2)
            ref = exact.shell_probability(b * dr, (b + 1) * dr, var, d) / V
            if ref * V < 1e-3:
                continue
            mean, se = rho[:, b].mean(), rho[:, b].std(ddof=1) / np.sqrt(nblk)
            assert abs(mean - ref) < 5 * se + 1e-3 * ref, (b, mean, ref, se)
    E_exact = exact.energy(N, beta, P=P, d=d, xi=xi)
    for series in (Ev, Ep):
        blocks = series.reshape(20, -1).mean(axis=1)
        mean = blocks.mean()
        se = blocks.std(ddof=1) / np.sqrt(len(blocks))
        assert se < 0.03 * E_exact, (se, E_exact)
        assert abs(mean - E_exact) < 4 * se, (mean, se, E_exact)
        print(f"xi={xi}: mean {mean:.4f} +- {se:.4f}, exact {E_exact:.4f}")


def test_batch_fp32_thermostat_long_run_matches_exact():
    """The batched workload's FP32 thermostat (nhc_fp32, mixed precision) over
    long runs of ideal trapped particles (g = 0) at the batched workload's
    temperatures and exchange parameters: each replica's block-averaged E_prim
    and E_vir agree with the exact finite-P energy for its (beta, xi) within 4
    standard errors."""
    import paper_2404_02628_gb300 as pkg
    N, P, d = 16, 32, 2
    reps = [(1.0, 0.0), (2.0, 1.0), (3.0, 0.4), (4.0, 0.8), (2.0, 0.6), (3.0, 1.0)]
    rs = [beads(N, P, d, 2100 + q) for q in range(len(reps))]
    ps = [momenta(N, P, d, b, 2100 + q) for q, (b, _) in enumerate(reps)]
    B = pkg.Batch([N] * len(reps), P, d, [b for b, _ in reps], [x for _, x in reps], 1.0, 0.0, 0.5, rs=rs, ps=ps,
                  precision=pkg.PREC_MIXED, nhc_len=4, dt=0.01, nhc_fp32=1)
    B.step(10000)
    n_samples, stride = 20000, 10
    Ep = np.empty((n_samples, len(reps)))
    Ev = np.empty((n_samples, len(reps)))
    for i in range(n_samples):
        B.step(stride)
        est = B.estimators()
        Ep[i] = [e["E_prim"] for e in est]
        Ev[i] = [e["E_vir"] for e in est]
    B.close()
    for q, (beta, xi) in enumerate(reps):
        E_exact = exact.energy(N, beta, P=P, d=d, xi=xi)
        for series in (Ev[:, q], Ep[:, q]):
            blocks = series.reshape(20, -1).mean(axis=1)
            mean = blocks.mean()
            se = blocks.std(ddof=1) / np.sqrt(len(blocks))
            print(f"beta={beta} xi={xi}: mean {mean:.4f} +- {se:.4f}, exact {E_exact:.4f}")
            assert se < 0.05 * E_exact, (q, se, E_exact)
            assert abs(mean - E_exact) < 4 * se, (q, mean, se, E_exact)
