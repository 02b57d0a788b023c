"""Pins of the several-species oracle (Sec. II, closing paragraph: coexisting
spins, one exchange recursion per species) against things other than itself
(no GPU): finite differences of its potential, the one-species oracle, the
distinguishable limit, and the N! x M! permutation sum of the partition
function of two trapped ideal species."""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import exact
from workloads import beads


def _V_total(r, counts, beta, xi, om, A, s):
    _, info = oracle.forces_species(r, counts, beta, xi, om, A, s)
    return info["V_xi"] + info["U_over_P"]


@pytest.mark.parametrize("counts,xi,A", [([3, 4], 1.0, 0.0), ([2, 2, 3], 0.6, 1.5), ([1, 5], 0.0, 0.8)])
def test_species_forces_match_finite_differences(counts, xi, A):
    N, P, d, beta, om, s = sum(counts), 4, 2, 1.3, 1.0, 0.7
    r = beads(N, P, d, 600 + N)
    F, _ = oracle.forces_species(r, counts, beta, xi, om, A, s)
    rng = np.random.default_rng(5)
    h = 1e-4
    for _ in range(16):
        l, j, c = int(rng.integers(N)), int(rng.choice([0, P - 1, 1])), int(rng.integers(d))
        vals = []
        for k in (-2, -1, 1, 2):
            x = r.copy()
            x[l, j, c] += k * h
            vals.append(_V_total(x, counts, beta, xi, om, A, s))
        fd = -(vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)
        assert abs(F[l, j, c] - fd) < 1e-7 * max(1.0, abs(fd)), (l, j, c, F[l, j, c], fd)


def test_one_species_is_the_plain_oracle():
    r = beads(9, 5, 3, 61)
    F1, i1 = oracle.forces_species(r, [9], 1.1, 0.7, 1.0, 2.0, 0.5)
    F2, i2 = oracle.forces(r, 1.1, 0.7, 1.0, 2.0, 0.5)
    assert np.array_equal(F1, F2)
    assert i1["V_xi"] == i2["V_xi"]


def test_distinguishable_forces_do_not_depend_on_the_split():
    """xi = 0: no exchange at all, so every split gives the same forces; the
    potentials differ only by the constant sum_k ln(n_k!)/beta."""
    r = beads(8, 4, 2, 62)
    beta = 1.7
    Fa, ia = oracle.forces_species(r, [8], beta, 0.0, 1.0, 1.0, 0.5)
    Fb, ib = oracle.forces_species(r, [3, 5], beta, 0.0, 1.0, 1.0, 0.5)
    assert np.abs(Fa - Fb).max() < 1e-12 * np.abs(Fa).max()
    const = (math.lgamma(9) - math.lgamma(4) - math.lgamma(6)) / beta
    assert abs((ia["V_xi"] - ib["V_xi"]) - const) < 1e-10 * abs(ia["V_xi"])


def test_two_species_partition_function_is_the_product_group_sum():
    """Z of two trapped ideal species (N_A = 2, N_B = 3) as the sum over the
    permutations of S_A x S_B with xi^{N_p} and closed-form ring factors
    z_P(k) (Sec. II), against the product of the one-species recursions that
    oracle.exact uses; the energies add."""
    P, beta, d, xi = 8, 1.2, 2, 0.7
    th = P * math.asinh(beta / (2 * P))

    def z(k):
        return (2 * math.sinh(k * th)) ** (-d)

    def perm_sum(n):
        tot = 0.0
        for perm in itertools.permutations(range(n)):
            seen, cyc, swaps = [False] * n, [], 0
            for i in range(n):
                if not seen[i]:
                    L, j = 0, i
                    while not seen[j]:
                        seen[j] = True
                        j = perm[j]
                        L += 1
                    cyc.append(L)
                    swaps += L - 1
            tot += xi ** swaps * math.prod(z(L) for L in cyc)
        return tot / math.factorial(n)

    def rec(n):
        Z = [1.0]
        for m in range(1, n + 1):
            Z.append(sum(xi ** (k - 1) * z(k) * Z[m - k] for k in range(1, m + 1)) / m)
        return Z[n]

    both = 0.0
    for pa in itertools.permutations(range(2)):
        for pb in itertools.permutations(range(3)):
            perm = list(pa) + [2 + q for q in pb]
            seen, cyc, swaps = [False] * 5, [], 0
            for i in range(5):
                if not seen[i]:
                    L, j = 0, i
                    while not seen[j]:
                        seen[j] = True
                        j = perm[j]
                        L += 1
                    cyc.append(L)
                    swaps += L - 1
            both += xi ** swaps * math.prod(z(L) for L in cyc)
    both /= math.factorial(2) * math.factorial(3)
    assert abs(both - perm_sum(2) * perm_sum(3)) < 1e-12 * both
    assert abs(both - rec(2) * rec(3)) < 1e-12 * both
    E_sum = exact.energy(2, beta, P=P, d=d, xi=xi) + exact.energy(3, beta, P=P, d=d, xi=xi)
    h = 1e-6
    # the energy of the product is the sum of the energies: check by differencing ln Z in beta
    def lnZ(b):
        t = P * math.asinh(b / (2 * P))
        zz = lambda k: (2 * math.sinh(k * t)) ** (-d)
        def r_(n):
            Z = [1.0]
            for m in range(1, n + 1):
                Z.append(sum(xi ** (k - 1) * zz(k) * Z[m - k] for k in range(1, m + 1)) / m)
            return Z[n]
        return math.log(r_(2) * r_(3))
    E_fd = -(lnZ(beta + h) - lnZ(beta - h)) / (2 * h)
    assert abs(E_fd - E_sum) < 1e-6 * E_sum
