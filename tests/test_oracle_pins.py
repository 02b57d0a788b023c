"""Pins of the FP64 oracle against things other than itself (no GPU).

Each test fixes one part of the oracle with an independent route: the cycle
energies straight from their definition, brute-force sums over every ring
topology the recursion counts, the N! permutation sum, closed forms of the
trapped ideal gas, finite differences, exact invariants and special cases.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import exact
from workloads import beads

# --------------------------------------------------------------------------
# independent helpers (written from the definitions, not from the oracle)


def E_def(r, beta, u, v):
    """E^[u,v] from its definition (Sec. III): all springs of the ring formed by
    particles u..v, bead P of l joined to bead 1 of l+1, bead P of v to bead 1 of u."""
    N, P, d = r.shape
    k = P / beta**2
    s = 0.0
    for l in range(u, v + 1):
        for j in range(1, P + 1):
            a = r[l - 1, j - 1]
            if j < P:
                b = r[l - 1, j]
            else:
                b = r[l, 0] if l < v else r[u - 1, 0]
            s += float(np.sum((b - a) ** 2))
    return 0.5 * k * s


def compositions(lo, hi):
    """All ways to cut lo..hi into consecutive blocks [(a,b), ...]."""
    n = hi - lo + 1
    if n <= 0:
        yield []
        return
    for cuts in itertools.product([0, 1], repeat=n - 1):
        blocks, start = [], lo
        for i, c in enumerate(cuts):
            if c:
                blocks.append((start, lo + i))
                start = lo + i + 1
        blocks.append((start, hi))
        yield blocks


def xi_pow(xi, n):
    return 1.0 if n == 0 else xi**n


def log_weight(r, beta, xi, blocks):
    """ln of prod_blocks xi^{len-1} (1/end) e^{-beta E^[start,end]} (None if zero)."""
    lw = 0.0
    for a, b in blocks:
        w = xi_pow(xi, b - a)
        if w == 0.0:
            return None
        lw += math.log(w) - math.log(b) - beta * E_def(r, beta, a, b)
    return lw


def lse(vals):
    vals = [v for v in vals if v is not None]
    m = max(vals)
    return m + math.log(math.fsum(math.exp(v - m) for v in vals))


CASES = [(4, 3, 2, 1.0, 1.0, 11), (5, 4, 2, 1.3, 0.3, 12), (6, 2, 3, 0.7, 1.0, 13),
         (3, 5, 1, 2.0, 0.0, 14), (7, 3, 2, 1.0, 0.6, 15)]


# --------------------------------------------------------------------------
# cycle energies

@pytest.mark.parametrize("N,P,d,beta,xi,seed", CASES)
def test_cycle_energies_match_definition(N, P, d, beta, xi, seed):
    r = beads(N, P, d, seed)
    E = oracle.cycle_energies(r, beta)
    for u in range(1, N + 1):
        for v in range(u, N + 1):
            ref = E_def(r, beta, u, v)
            assert abs(E[u - 1, v - 1] - ref) <= 1e-12 * max(1.0, abs(ref))


def test_E_int_definition():
    r = beads(3, 6, 2, 7)
    beta = 1.7
    k = 6 / beta**2
    for v in (1, 2, 3):
        ref = 0.5 * k * sum(float(np.sum((r[v - 1, j + 1] - r[v - 1, j]) ** 2)) for j in range(5))
        assert abs(oracle.E_int(r, beta, v) - ref) <= 1e-13 * ref


# --------------------------------------------------------------------------
# recursions: every ring topology the recursion counts, summed one by one

@pytest.mark.parametrize("N,P,d,beta,xi,seed", CASES)
def test_forward_recursion_is_sum_over_compositions(N, P, d, beta, xi, seed):
    r = beads(N, P, d, seed)
    E = oracle.cycle_energies(r, beta)
    Vf = oracle.V_forward(E, beta, xi)
    assert Vf[0] == 0.0
    for l in range(1, N + 1):
        ref = -lse([log_weight(r, beta, xi, c) for c in compositions(1, l)]) / beta
        assert abs(Vf[l] - ref) <= 1e-12 * max(1.0, abs(ref)), (l, Vf[l], ref)


@pytest.mark.parametrize("N,P,d,beta,xi,seed", CASES)
def test_backward_recursion_is_sum_over_compositions(N, P, d, beta, xi, seed):
    r = beads(N, P, d, seed)
    E = oracle.cycle_energies(r, beta)
    Vb = oracle.V_backward(E, beta, xi)
    assert Vb[N] == 0.0
    for u in range(1, N + 1):
        ref = -lse([log_weight(r, beta, xi, c) for c in compositions(u, N)]) / beta
        assert abs(Vb[u - 1] - ref) <= 1e-12 * max(1.0, abs(ref)), (u, Vb[u - 1], ref)


@pytest.mark.parametrize("N,P,d,beta,xi,seed", CASES)
def test_connection_probabilities_are_marginals(N, P, d, beta, xi, seed):
    """Pr[G(l)=l'] equals the brute-force marginal of 'bead P of l joins bead 1 of l''."""
    r = beads(N, P, d, seed)
    E = oracle.cycle_energies(r, beta)
    Vf = oracle.V_forward(E, beta, xi)
    Vb = oracle.V_backward(E, beta, xi)
    Pr = oracle.connection_probabilities(E, Vf, Vb, beta, xi)
    comps = list(compositions(1, N))
    lws = [log_weight(r, beta, xi, c) for c in comps]
    m = max(w for w in lws if w is not None)
    ref = np.zeros((N, N + 1))
    for c, lw in zip(comps, lws):
        if lw is None:
            continue
        w = math.exp(lw - m)
        for a, b in c:
            ref[b - 1, a - 1] += w
            for l in range(a, b):
                ref[l - 1, l] += w
    ref /= ref.sum(axis=1, keepdims=True)
    np.testing.assert_allclose(Pr, ref, atol=1e-12, rtol=0)


# --------------------------------------------------------------------------
# the recursion's weights against the N! permutation sum (integrated level)

def cycle_lengths(perm):
    n, seen, out = len(perm), [False] * len(perm), []
    for i in range(n):
        if not seen[i]:
            k, j = 0, i
            while not seen[j]:
                seen[j] = True
                j = perm[j]
                k += 1
            out.append(k)
    return out


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("xi", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("P", [None, 4, 32])
def test_partition_function_equals_permutation_sum(N, xi, P):
    beta = 1.3
    z = {k: exact.ring_partition(k, beta, P) for k in range(1, N + 1)}
    tot = 0.0
    for perm in itertools.permutations(range(N)):
        cl = cycle_lengths(perm)
        Np = N - len(cl)  # transpositions needed (Sec. II)
        tot += xi_pow(xi, Np) * math.prod(z[k] for k in cl)
    Zperm = tot / math.factorial(N)
    _, Z = exact.energy_mp(N, beta, P, xi=xi)
    assert abs(float(Z[N]) - Zperm) <= 1e-13 * Zperm


# --------------------------------------------------------------------------
# exact energies: closed forms and limits

def test_single_ring_polymer_energy_normal_modes():
    """N=1: the P-bead ring in a trap, by its normal-mode product, differentiated numerically."""
    P, d = 16, 2
    for beta in (0.5, 2.0, 6.0):
        def lnZ(b):
            x = b / P
            return -0.5 * d * sum(math.log(4 * math.sin(math.pi * j / P) ** 2 + x * x)
                                  for j in range(P))
        h = 1e-5
        E_fd = -(lnZ(beta + h) - lnZ(beta - h)) / (2 * h)
        assert abs(exact.energy(1, beta, P) - E_fd) <= 1e-7 * E_fd


def test_distinguishable_energy_closed_form():
    for beta in (0.5, 3.0):
        for P in (None, 8):
            th, dth = exact.theta(beta, P)
            ref = 7 * 2 * dth / math.tanh(th)
            assert abs(exact.energy(7, beta, P, xi=0.0) - ref) <= 1e-12 * ref


def test_ground_state_energy_is_N():
    """Sec. IV A: at low temperature the ideal trapped Bose gas has E = N (d = 2)."""
    for N in (5, 100, 1600):
        assert abs(exact.energy(N, 40.0) - N) <= 1e-6 * N


def test_rescaled_and_mp_energies_agree():
    for N, beta, P, xi in [(8, 2.0, 32, 1.0), (8, 2.0, None, 0.4), (30, 0.7, 12, 1.0)]:
        e_mp, _ = exact.energy_mp(N, beta, P, xi=xi)
        assert abs(exact.energy(N, beta, P, xi=xi) - e_mp) <= 1e-11 * e_mp


# --------------------------------------------------------------------------
# special cases

def test_single_particle_is_ring_polymer():
    r = beads(1, 7, 2, 3)
    beta = 1.1
    E = oracle.cycle_energies(r, beta)
    for xi in (0.0, 1.0):
        Vf = oracle.V_forward(E, beta, xi)
        assert abs(Vf[1] - E_def(r, beta, 1, 1)) <= 1e-13 * Vf[1]


def test_distinguishable_limit():
    N, P, d, beta = 6, 4, 2, 0.9
    r = beads(N, P, d, 4)
    F, info, Pr = oracle.forces(r, beta, 0.0, want_pr=True)
    ref = sum(E_def(r, beta, l, l) for l in range(1, N + 1)) + math.log(math.factorial(N)) / beta
    assert abs(info["V_xi"] - ref) <= 1e-12 * abs(ref)
    np.testing.assert_allclose(Pr[:, :N + 1], np.eye(N, N + 1), rtol=0, atol=1e-12)


def test_two_particles_closed_form():
    r = beads(2, 5, 2, 5)
    beta, xi = 1.2, 0.7
    E11, E22, E12 = E_def(r, beta, 1, 1), E_def(r, beta, 2, 2), E_def(r, beta, 1, 2)
    ref = -math.log(0.5 * (math.exp(-beta * (E11 + E22)) + xi * math.exp(-beta * E12))) / beta
    _, info = oracle.forces(r, beta, xi)
    assert abs(info["V_xi"] - ref) <= 1e-12 * abs(ref)


# --------------------------------------------------------------------------
# invariants on arbitrary configurations

@pytest.mark.parametrize("N,P,d,beta,xi,seed", CASES + [(40, 8, 2, 2.0, 1.0, 21)])
def test_invariants(N, P, d, beta, xi, seed):
    r = beads(N, P, d, seed)
    F, info, Pr = oracle.forces(r, beta, xi, omega=0.0, A=0.0, want_pr=True)
    assert abs(info["V_xi"] - info["V_xi_bwd"]) <= 1e-12 * max(1.0, abs(info["V_xi"]))
    np.testing.assert_allclose(Pr.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(Pr[:, :N].sum(axis=0), 1.0, atol=1e-12)
    assert Pr[N - 1, N] == 0.0 or abs(Pr[N - 1, N]) < 1e-12
    scale = np.abs(F).max()
    # translation invariance of V_xi: total exchange force vanishes
    np.testing.assert_allclose(F.sum(axis=(0, 1)), 0.0, atol=1e-11 * scale * N * P)
    if d == 2:  # rotation invariance: total torque vanishes
        tau = np.sum(r[..., 0] * F[..., 1] - r[..., 1] * F[..., 0])
        assert abs(tau) <= 1e-10 * scale * N * P


def test_pair_forces_newton_third_law():
    r = beads(30, 4, 2, 8)
    U, F, vir = oracle.interaction(r, 0.0, 3.0 / (math.pi * 0.25), 0.5)
    np.testing.assert_allclose(F.sum(axis=0), 0.0, atol=1e-12)


def test_interaction_two_particles_by_hand():
    P, s, A, om = 3, 0.5, 1.7, 1.3
    r = beads(2, P, 2, 9)
    U_ref, vir_ref = 0.0, 0.0
    F_ref = np.zeros_like(r)
    for j in range(P):
        x1, x2 = r[0, j], r[1, j]
        q = x1 - x2
        e = A * math.exp(-float(q @ q) / s**2)
        U_ref += 0.5 * om**2 * (x1 @ x1 + x2 @ x2) + e
        g1 = om**2 * x1 - 2 * e / s**2 * q
        g2 = om**2 * x2 + 2 * e / s**2 * q
        F_ref[0, j], F_ref[1, j] = -g1 / P, -g2 / P
        vir_ref += x1 @ g1 + x2 @ g2
    U, F, vir = oracle.interaction(r, om, A, s)
    assert abs(U - U_ref) <= 1e-13 * U_ref
    assert abs(vir - vir_ref) <= 1e-12 * abs(vir_ref)
    np.testing.assert_allclose(F, F_ref, rtol=0, atol=1e-13)


# --------------------------------------------------------------------------
# forces against finite differences of the oracle's own potential

def _total_V(r, beta, xi, om, A, s):
    _, info = oracle.forces(r, beta, xi, om, A, s)
    return info["V_xi"] + info["U_over_P"]


@pytest.mark.parametrize("xi,A", [(1.0, 3.0 / (math.pi * 0.25)), (0.35, 0.0), (0.0, 1.0)])
def test_forces_match_finite_differences(xi, A):
    N, P, d, beta, om, s = 4, 5, 2, 1.4, 1.0, 0.5
    r = beads(N, P, d, 31)
    F, _ = oracle.forces(r, beta, xi, om, A, s)
    h = 1e-3
    Ffd = np.zeros_like(r)
    for idx in np.ndindex(r.shape):
        def Vat(dx):
            q = r.copy()
            q[idx] += dx
            return _total_V(q, beta, xi, om, A, s)
        d1 = (Vat(h) - Vat(-h)) / (2 * h)
        d2 = (Vat(h / 2) - Vat(-h / 2)) / h
        Ffd[idx] = -(4 * d2 - d1) / 3  # Richardson
    np.testing.assert_allclose(F, Ffd, rtol=0, atol=1e-7 * np.abs(F).max())


def test_spring_expectation_is_beta_derivative():
    """<spring> = -d(beta V_xi)/d beta at fixed beads (primitive estimator)."""
    N, P, d, xi = 5, 6, 2, 0.8
    r = beads(N, P, d, 41)
    beta = 1.5

    def bV(b):
        _, info = oracle.forces(r, b, xi)
        return b * info["V_xi"]

    _, info = oracle.forces(r, beta, xi)
    h = 1e-4
    d1 = (bV(beta + h) - bV(beta - h)) / (2 * h)
    d2 = (bV(beta + h / 2) - bV(beta - h / 2)) / h
    deriv = (4 * d2 - d1) / 3
    assert abs(info["spring"] + deriv) <= 1e-8 * abs(deriv)


# --------------------------------------------------------------------------
# molecular dynamics

def _state(N, P, d, beta, M, seed):
    from workloads import momenta
    return oracle.MDState(0.5 * beads(N, P, d, seed), momenta(N, P, d, beta, seed), M)


def test_nve_energy_conservation_scales_as_dt_squared():
    N, P, d, beta, xi = 3, 4, 2, 1.0, 1.0
    drifts = []
    for dt in (0.004, 0.002):
        st = _state(N, P, d, beta, 4, 51)
        est = oracle.md_run(st, beta, xi, 1.0, 1.0, 0.5, dt, 0.1, int(2.0 / dt), thermostat=False)
        H = est[:, oracle.ESTIMATE_FIELDS.index("H_conserved")]
        drifts.append(np.abs(H - H[0]).max())
    ratio = drifts[0] / drifts[1]
    assert 3.0 < ratio < 5.0, drifts


def test_nve_time_reversible():
    N, P, d, beta = 3, 4, 2, 1.0
    st = _state(N, P, d, beta, 4, 52)
    r0 = st.r.copy()
    oracle.md_run(st, beta, 1.0, 1.0, 1.0, 0.5, 0.005, 0.1, 200, thermostat=False)
    st.p *= -1
    oracle.md_run(st, beta, 1.0, 1.0, 1.0, 0.5, 0.005, 0.1, 200, thermostat=False)
    np.testing.assert_allclose(st.r, r0, atol=1e-9)


def test_nhc_extended_energy_conserved():
    N, P, d, beta = 3, 4, 2, 1.0
    st = _state(N, P, d, beta, 4, 53)
    est = oracle.md_run(st, beta, 1.0, 1.0, 1.0, 0.5, 0.002, beta / P, 2000, thermostat=True)
    H = est[:, oracle.ESTIMATE_FIELDS.index("H_conserved")]
    assert np.abs(H - H[0]).max() < 2e-4 * abs(H[0])


def blocked_error(x, nblocks=20):
    n = len(x) // nblocks
    means = np.array([x[i * n:(i + 1) * n].mean() for i in range(nblocks)])
    return means.mean(), means.std(ddof=1) / math.sqrt(nblocks)


@pytest.mark.parametrize("xi", [1.0, 0.0])
def test_long_run_energy_matches_exact(xi):
    """Thermostatted MD of 2 ideal trapped particles: <E_prim> and <E_vir> agree
    with the exact finite-P canonical energy within the blocking error."""
    N, P, d, beta, dt = 2, 6, 2, 1.0, 0.02
    st = _state(N, P, d, beta, 4, 60)
    oracle.md_run(st, beta, xi, 1.0, 0.0, 0.5, dt, beta / P, 10000)
    est = oracle.md_run(st, beta, xi, 1.0, 0.0, 0.5, dt, beta / P, 2000000)
    Eex = exact.energy(N, beta, P, xi=xi)
    for name in ("E_prim", "E_vir"):
        x = est[:, oracle.ESTIMATE_FIELDS.index(name)]
        m, err = blocked_error(x)
        assert err < 0.01 * Eex
        assert abs(m - Eex) < 4.0 * err, (name, m, err, Eex)


def test_ground_state_energy_printed_in_paper():
    """Sec. IV A prints E = N for the ideal trapped gas at beta = 6 (ground
    state) and simulated energies within about 0.3 % of it at P = 72; the
    oracle's exact finite-P energy must lie inside that band."""
    import os
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "paper_ground_state.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(v)
    for N in (100, 1600):
        E = exact.energy(N, vals["beta"], P=int(vals["P"]))
        assert abs(E / (N * vals["energy_per_particle"]) - 1.0) < vals["agreement_rel"], (N, E)


# --------------------------------------------------------------------------
# radial density (Sec. IV B density profiles)

def test_bead_variance_limits_and_matrix_inverse():
    """Spectral sum of the distinguishable ring polymer against (i) the
    inverse of its Gaussian weight matrix, (ii) the classical limit P = 1,
    (iii) the quantum oscillator coth(beta omega / 2) / (2 m omega) as P grows,
    and (iv) the ground state (variance 1/2: density exp(-r^2)/pi in d = 2)."""
    beta, om, m, P = 1.7, 1.3, 0.8, 7
    ks = m * P / beta**2
    A = np.zeros((P, P))
    for j in range(P):
        A[j, j] += 2 * ks + m * om**2 / P
        A[j, (j + 1) % P] -= ks
        A[j, (j - 1) % P] -= ks
    cov = np.linalg.inv(beta * A)
    assert abs(exact.bead_variance(beta, P, om, m) - cov[3, 3]) < 1e-13 * cov[3, 3]
    assert abs(exact.bead_variance(beta, 1, om, m) - 1.0 / (beta * m * om**2)) < 1e-14
    q = 1.0 / (2 * m * om * math.tanh(beta * om / 2))
    assert abs(exact.bead_variance(beta, 4000, om, m) - q) < 1e-6 * q
    assert abs(exact.bead_variance(40.0, 4000) - 0.5) < 1e-3


@pytest.mark.parametrize("d", [1, 2, 3])
def test_radial_density_of_gaussian_samples(d):
    """The oracle's binned density of isotropic Gaussian points matches the
    exact shell probabilities within binomial error bars, and sums to the
    fraction inside r_max."""
    rng = np.random.default_rng(40 + d)
    var, n, nbins, r_max = 0.7, 400000, 40, 4.0
    r = rng.normal(0.0, math.sqrt(var), size=(n, 1, d))
    rho, counts = oracle.radial_density(r, nbins, r_max)
    dr = r_max / nbins
    for b in range(nbins):
        p = exact.shell_probability(b * dr, (b + 1) * dr, var, d)
        se = math.sqrt(max(p * (1 - p), 1e-12) / n)
        assert abs(counts[b] / n - p) < 5 * se + 1e-12, (b, counts[b] / n, p)
    edges = np.arange(nbins + 1) * dr
    vol = {1: 2 * np.diff(edges), 2: np.pi * np.diff(edges**2), 3: 4 / 3 * np.pi * np.diff(edges**3)}[d]
    assert abs(float(np.sum(rho * vol)) - counts.sum() / n) < 1e-12


@pytest.mark.parametrize("d", [1, 3])
def test_exact_energy_other_dimensions(d):
    """The trapped ideal gas factorises over Cartesian directions: the d-dimensional
    distinguishable energy is d times the one-dimensional one, the N = 1 energy
    is d/2 coth(beta omega / 2) in the continuum, and the permutation sum of
    the partition function matches the recursion in d dimensions as well."""
    beta, P = 1.7, 9
    th, dth = exact.theta(beta, P)
    ref = 5 * d * dth / math.tanh(th)
    assert abs(exact.energy(5, beta, P, d=d, xi=0.0) - ref) <= 1e-12 * ref
    assert abs(exact.energy(5, beta, P, d=d, xi=0.0) - d * exact.energy(5, beta, P, d=1, xi=0.0)) <= 1e-12 * ref
    e1 = exact.energy(1, beta, None, d=d)
    assert abs(e1 - 0.5 * d / math.tanh(beta / 2)) <= 1e-12 * e1
    N, xi = 4, 0.6
    z = {k: exact.ring_partition(k, beta, P, d=d) for k in range(1, N + 1)}
    tot = 0.0
    for perm in itertools.permutations(range(N)):
        cl = cycle_lengths(perm)
        tot += xi_pow(xi, N - len(cl)) * math.prod(z[k] for k in cl)
    _, Z = exact.energy_mp(N, beta, P, d=d, xi=xi)
    assert abs(float(Z[N]) - tot / math.factorial(N)) <= 1e-13 * tot / math.factorial(N)


@pytest.mark.parametrize("d", [1, 3])
def test_forces_match_finite_differences_other_dimensions(d):
    """Exchange + trap + Gaussian-pair forces against Richardson-extrapolated
    central differences of V_xi + U/P in one and three dimensions."""
    N, P, beta, xi, om, A, s = 3, 4, 1.2, 0.7, 1.1, 2.0, 0.6
    r = beads(N, P, d, 41 + d)
    F, _ = oracle.forces(r, beta, xi, om, A, s)
    h = 1e-3
    Ffd = np.zeros_like(r)
    for idx in np.ndindex(r.shape):
        def Vat(dx):
            q = r.copy()
            q[idx] += dx
            return _total_V(q, beta, xi, om, A, s)
        d1 = (Vat(h) - Vat(-h)) / (2 * h)
        d2 = (Vat(h / 2) - Vat(-h / 2)) / h
        Ffd[idx] = -(4 * d2 - d1) / 3
    np.testing.assert_allclose(F, Ffd, rtol=0, atol=1e-7 * np.abs(F).max())
