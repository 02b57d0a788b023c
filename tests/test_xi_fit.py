"""pimd_xi_extrapolate (host arithmetic of the C ABI, no GPU) against the
oracle's weighted least squares, exact polynomials, and the exact energies of
ideal trapped fictitious particles (Sec. I, Sec. IV D)."""
import numpy as np
import pytest

from oracle import exact, xifit


@pytest.fixture(scope="module")
def pkg():
    import paper_2404_02628_gb300 as p
    p.load()
    return p


def test_reference_fit_matches_numpy_polyfit():
    rng = np.random.default_rng(3)
    xi = np.linspace(0, 1, 6)
    sig = 0.05 + 0.1 * rng.random(6)
    E = 3.0 - 1.2 * xi + 0.4 * xi ** 2 + sig * rng.standard_normal(6)
    v, vs, chi2, coef = xifit.extrapolate(xi, E, sig, 2, -1.0)
    c_np, cov_np = np.polyfit(xi, E, 2, w=1.0 / sig, cov="unscaled")
    assert np.allclose(coef[::-1], c_np, rtol=1e-12, atol=1e-12)
    p = np.array([1.0, -1.0, 1.0])[::-1]
    assert abs(v - np.polyval(c_np, -1.0)) < 1e-12
    assert abs(vs - np.sqrt(p @ cov_np @ p)) < 1e-12


@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_library_fit_recovers_exact_polynomials(pkg, degree):
    xi = np.linspace(0.0, 1.0, 7)
    c = np.array([2.0, -0.7, 0.3, 0.11])[:degree + 1]
    E = np.polynomial.polynomial.polyval(xi, c)
    v, vs, chi2, coef = pkg.pimd_xi_extrapolate(xi, E, np.full(7, 0.1), degree, -1.0)
    assert np.allclose(coef, c, atol=1e-12)
    assert abs(v - np.polynomial.polynomial.polyval(-1.0, c)) < 1e-12
    assert chi2 < 1e-20


def test_library_fit_matches_reference(pkg):
    rng = np.random.default_rng(11)
    for degree in (1, 2, 3):
        xi = np.sort(rng.random(9))
        sig = 0.02 + 0.2 * rng.random(9)
        E = 5.0 + rng.standard_normal(9)
        got = pkg.pimd_xi_extrapolate(xi, E, sig, degree, -1.0)
        ref = xifit.extrapolate(xi, E, sig, degree, -1.0)
        for a, b in zip(got[:3], ref[:3]):
            assert abs(a - b) <= 1e-10 * max(1.0, abs(b)), (degree, got, ref)
        assert np.allclose(got[3], ref[3], rtol=1e-9, atol=1e-9)


def test_library_fit_rejects_underdetermined(pkg):
    with pytest.raises(pkg.PimdError):
        pkg.pimd_xi_extrapolate([0.5, 0.5, 0.5], [1.0, 2.0, 3.0], [1.0, 1.0, 1.0], 2, -1.0)
    with pytest.raises(pkg.PimdError):
        pkg.pimd_xi_extrapolate([0.0, 1.0], [1.0, 2.0], [1.0, 0.0], 1, -1.0)


def test_quadratic_extrapolation_of_exact_ideal_energies():
    """Ideal trapped particles (N=4, d=2, P=12): the quadratic fit of the exact
    E(xi) over xi in {0, 0.2, ..., 1} reaches the exact fermion energy
    (the same recursion at xi = -1) within 0.5 % at weak degeneracy (beta=0.5)
    and misses it by more at strong degeneracy (beta=2): the extrapolation's
    model error, which the MD scan cannot remove."""
    xi = np.linspace(0.0, 1.0, 6)
    for beta, lo, hi in ((0.5, 0.0, 0.005), (2.0, 0.05, 1.0)):
        E = [exact.energy(4, beta, P=12, d=2, xi=x) for x in xi]
        v, _, _, _ = xifit.extrapolate(xi, E, np.ones(6), 2, -1.0)
        ef = exact.energy(4, beta, P=12, d=2, xi=-1.0)
        assert lo <= abs(v - ef) / ef < hi, (beta, v, ef)


def test_exact_fermion_energy_from_the_recursion_is_the_permutation_sum():
    """exact.energy at xi = -1 (the cycle recursion with sign (-1)^(k-1)) equals
    -d ln Z / d beta of the N! permutation sum with signs (-1)^{N_p} (Sec. II),
    N = 3, by central differences in beta."""
    import itertools
    import math

    def z1(k, beta, P):
        th = P * math.asinh(beta / (2 * P))
        return (2 * math.sinh(k * th)) ** -2

    def Z(beta, P=12, N=3):
        tot = 0.0
        for perm in itertools.permutations(range(N)):
            seen, cyc, swaps = [False] * N, [], 0
            for i in range(N):
                if not seen[i]:
                    L, j = 0, i
                    while not seen[j]:
                        seen[j] = True
                        j = perm[j]
                        L += 1
                    cyc.append(L)
                    swaps += L - 1
            tot += (-1.0) ** swaps * math.prod(z1(L, beta, P) for L in cyc)
        return tot / math.factorial(N)

    beta, h = 0.8, 1e-5
    E_perm = -(math.log(Z(beta + h)) - math.log(Z(beta - h))) / (2 * h)
    assert abs(exact.energy(3, beta, P=12, d=2, xi=-1.0) - E_perm) < 1e-6 * abs(E_perm)
