"""The factorised form of the exchange recursion that the CUDA path solves,
checked on CPU against the oracle's literal recursions (no GPU, no CUDA code).

Sec. III's forward recursion over cycle energies E^[u,v] becomes, with
a_i = r_i^P, b_k = r_k^1, g(i,k) = kappa |a_i - b_k|^2 (kappa = P / (2 beta)),
row constants c_n = g(n-1,n) - ln n - ln xi (c_N = -ln N - ln xi) and
M[n][k] = exp(c_n - g(n-1,k)) for 0 <= k < n <= N, the unit lower-triangular
system y = e_0 + M y, and the backward recursion its transpose
c = e_N + M^T c; then W_N = xi^N y[N], y[N] = c[0], and

    V_xi = sum_l E_int(l) + sum_{i<N-1} g(i,i+1)/beta - (N ln xi + ln y[N]) / beta,
    Pr[G(l) = k]   = M[l+1][k] y[k] c[l+1] / y[N]     (k <= l),
    Pr[G(l) = l+1] = 1 - y[l+1] c[l+1] / y[N].

Here both sides are plain FP64 (substitution on one side, the oracle's
log-sum-exp recursions on the other), so a wrong sign, index or constant in
the factorisation fails at the 1e-12 level.
"""
import math

import numpy as np
import pytest

import oracle
from workloads import beads


def _factorised(r, beta, xi):
    N, P, d = r.shape
    kappa = P / (2.0 * beta)
    a, b = r[:, P - 1, :], r[:, 0, :]

    def g(i, k):
        return kappa * float(np.sum((a[i] - b[k]) ** 2))

    c = np.zeros(N + 1)
    for n in range(1, N + 1):
        c[n] = (g(n - 1, n) if n < N else 0.0) - math.log(n) - math.log(xi)
    M = np.zeros((N + 1, N + 1))
    for n in range(1, N + 1):
        for k in range(n):
            M[n, k] = math.exp(c[n] - g(n - 1, k))
    # forward and back substitution (every term is non-negative, so nothing cancels)
    y = np.zeros(N + 1)
    y[0] = 1.0
    for n in range(1, N + 1):
        y[n] = math.fsum(M[n, k] * y[k] for k in range(n))
    cb = np.zeros(N + 1)
    cb[N] = 1.0
    for k in range(N - 1, -1, -1):
        cb[k] = math.fsum(M[n, k] * cb[n] for n in range(k + 1, N + 1))
    return M, y, cb, g


@pytest.mark.parametrize("N,P,d,beta,xi,seed", [(1, 4, 2, 1.0, 1.0, 3), (5, 6, 2, 1.3, 0.4, 4),
                                                (17, 8, 3, 0.8, 1.0, 5), (40, 5, 1, 2.0, 0.7, 6)])
def test_factorised_system_reproduces_the_recursions(N, P, d, beta, xi, seed):
    r = beads(N, P, d, seed) * 0.6  # keeps the plain (unscaled) FP64 factors in range
    M, y, cb, g = _factorised(r, beta, xi)
    Z = y[N]
    assert abs(Z - cb[0]) <= 1e-12 * Z                      # forward and backward agree
    E_int = sum(0.5 * P / beta**2 * float(np.sum(np.diff(r[l], axis=0) ** 2)) for l in range(N))
    link = sum(g(i, i + 1) for i in range(N - 1)) / beta
    V = E_int + link - (N * math.log(xi) + math.log(Z)) / beta
    F, info, Pr = oracle.forces(r, beta, xi, want_pr=True)
    assert abs(V - info["V_xi"]) <= 1e-12 * max(1.0, abs(info["V_xi"]))
    Pf = np.zeros((N, N + 1))
    for l in range(N):
        for k in range(l + 1):
            Pf[l, k] = M[l + 1, k] * y[k] * cb[l + 1] / Z
        if l + 1 < N:
            Pf[l, l + 1] = 1.0 - y[l + 1] * cb[l + 1] / Z
    np.testing.assert_allclose(Pf, Pr, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N,B", [(23, 4), (40, 8), (9, 32)])
def test_blocked_look_ahead_solve(N, B):
    """The blocked form of the solve: with G_J = (I - M_JJ)^{-1},
    Q_J = G_J M_{J,J-1}, P_J = M_{J+1,J} G_J and the off-band sums
    h_J = sum_{I<=J-2} M_JI y_I, hb_J = sum_{I>=J+2} M_IJ^T c_I,
        y_J = G_J h_J + Q_J y_{J-1},   c_J = G_J^T hb_J + P_J^T c_{J+1},
    block by block (blocks of B indices, the last one ragged), equals the
    plain substitution."""
    r = beads(N, 5, 2, 70 + N) * 0.6
    M, y, cb, _ = _factorised(r, 1.1, 0.8)
    n = N + 1
    nb = (n + B - 1) // B
    sl = [slice(J * B, min(n, J * B + B)) for J in range(nb)]
    e0 = np.zeros(n)
    e0[0] = 1.0
    eN = np.zeros(n)
    eN[N] = 1.0
    la = pytest.importorskip("scipy.linalg")
    # G_J by unit lower-triangular substitution (all terms non-negative: no cancellation)
    G = [la.solve_triangular(np.eye(sl[J].stop - sl[J].start) - M[sl[J], sl[J]], np.eye(sl[J].stop - sl[J].start),
                             lower=True, unit_diagonal=True) for J in range(nb)]
    yb = np.zeros(n)
    for J in range(nb):
        h = e0[sl[J]] + sum((M[sl[J], sl[I]] @ yb[sl[I]] for I in range(J - 1)), np.zeros(sl[J].stop - sl[J].start))
        q = G[J] @ M[sl[J], sl[J - 1]] @ yb[sl[J - 1]] if J >= 1 else 0.0
        yb[sl[J]] = G[J] @ h + q
    np.testing.assert_allclose(yb, y, rtol=1e-11, atol=0)
    cbb = np.zeros(n)
    for J in range(nb - 1, -1, -1):
        hb = eN[sl[J]] + sum((M[sl[I], sl[J]].T @ cbb[sl[I]] for I in range(J + 2, nb)),
                             np.zeros(sl[J].stop - sl[J].start))
        p = (M[sl[J + 1], sl[J]] @ G[J]).T @ cbb[sl[J + 1]] if J + 1 < nb else 0.0
        cbb[sl[J]] = G[J].T @ hb + p
    np.testing.assert_allclose(cbb, cb, rtol=1e-11, atol=0)


@pytest.mark.parametrize("N,P,d,beta,xi", [(7, 5, 2, 1.2, 1.0), (30, 4, 3, 0.9, 0.6), (12, 6, 1, 2.0, 0.3)])
def test_endpoint_forces_from_connection_probabilities(N, P, d, beta, xi):
    """Exterior-bead forces (Sec. III) in the form the finalize step uses:
    bead P of l is pulled towards bead 1 of every l' it may connect to,
    bead 1 of l towards bead P of every l'' that may connect to it, each
    weighted by Pr; plus the internal springs.  Against the oracle's forces."""
    r = beads(N, P, d, 90 + N) * 0.6
    M, y, cb, _ = _factorised(r, beta, xi)
    Z = y[N]
    Pf = np.zeros((N, N + 1))
    for l in range(N):
        for k in range(l + 1):
            Pf[l, k] = M[l + 1, k] * y[k] * cb[l + 1] / Z
        if l + 1 < N:
            Pf[l, l + 1] = 1.0 - y[l + 1] * cb[l + 1] / Z
    ks = P / beta**2
    a, b = r[:, P - 1, :], r[:, 0, :]
    F, _ = oracle.forces(r, beta, xi, omega=0.0, A=0.0)  # exchange and springs only
    for l in range(N):
        fp = -ks * (a[l] - r[l, P - 2])
        fp -= ks * sum(Pf[l, k] * (a[l] - b[k]) for k in range(l + 1))
        if l + 1 < N:
            fp -= ks * Pf[l, l + 1] * (a[l] - b[l + 1])
        f1 = -ks * (b[l] - r[l, 1])
        f1 -= ks * sum(Pf[m, l] * (b[l] - a[m]) for m in range(l, N))
        if l >= 1:
            f1 -= ks * Pf[l - 1, l] * (b[l] - a[l - 1])
        scale = np.abs(F).max()
        assert np.abs(fp - F[l, P - 1]).max() <= 1e-11 * scale, l
        assert np.abs(f1 - F[l, 0]).max() <= 1e-11 * scale, l
