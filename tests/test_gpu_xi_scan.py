"""xi scan of ideal trapped fictitious particles on the GPU and its
extrapolation to fermions (Sec. I, Sec. IV D).

N = 4, d = 2, P = 12, beta = 1 (the paper's fictitious-particle example,
without the interaction so that exact results exist), xi in {0, 0.2, ..., 1},
four replicas per xi in one batch.  Each MD energy must match the exact
finite-P energy of its xi (oracle.exact, the cycle recursion) within 4
standard errors; the quadratic extrapolation of the MD energies must match
the same extrapolation of the exact energies within 4 of its standard
errors.  The exact fermion energy (xi = -1) is printed beside it: the gap
between the two is the quadratic model's error, not the simulation's."""
import numpy as np
import pytest

from oracle import exact, xifit

pytestmark = pytest.mark.gpu


def test_xi_scan_matches_exact_and_extrapolates():
    from paper_2404_02628_gb300.xi_scan import extrapolate, xi_scan
    N, P, d, beta = 4, 12, 2, 1.0
    xis = [0.0, 0.2, 0.4, 0.6, 0.8, 1.0]
    scan = xi_scan(N, P, d, beta, xis, replicas=4, equil_steps=10000, samples=20000, stride=10, seed=42)
    E_exact = [exact.energy(N, beta, P=P, d=d, xi=x) for x in xis]
    for name in ("E_prim", "E_vir"):
        e = scan[name]
        for k, x in enumerate(xis):
            print("%s xi=%.1f: %.4f +- %.4f, exact %.4f" % (name, x, e["E"][k], e["sigma"][k], E_exact[k]))
            assert e["sigma"][k] < 0.05 * E_exact[k]
            assert abs(e["E"][k] - E_exact[k]) < 4 * e["sigma"][k], (name, x)
        fit = extrapolate(scan, name)
        ref, _, _, _ = xifit.extrapolate(xis, E_exact, e["sigma"], 2, -1.0)
        ef = exact.energy(N, beta, P=P, d=d, xi=-1.0)
        print("%s: E(-1) = %.4f +- %.4f (chi2 %.2f / %d); same fit of exact E(xi): %.4f; exact fermions %.4f"
              % (name, fit["value"], fit["sigma"], fit["chi2"], fit["dof"], ref, ef))
        assert abs(fit["value"] - ref) < 4 * fit["sigma"]
