"""Exact canonical energies of N non-interacting fictitious particles in an
isotropic harmonic trap (hbar = m = omega = k_B = 1 unless omega is given).

TEST INFRASTRUCTURE ONLY (part of the oracle).

The partition function obeys the cycle recursion behind the exchange
potential of Sec. III,

    Z_N = (1/N) sum_{k=1}^{N} xi^{k-1} z(k) Z_{N-k},   Z_0 = 1,

where z(k) is the partition function of one ring of k particles: a single
particle at inverse temperature k*beta.  With P beads per particle the ring has
k*P beads at the same imaginary-time step beta/P, and its Gaussian integral
(with the normalisation of the discretised partition function of Sec. II) is

    z_P(k) = [2 sinh(k theta_P)]^{-d},  theta_P = P asinh(beta omega / (2P)),

which tends to the continuum value [2 sinh(k beta omega / 2)]^{-d} as P grows.
E = -d ln Z_N / d beta; the derivative is carried through the recursion
exactly.  Large N uses the rescaled form z(k) e^{d k theta} = (1-e^{-2k theta})^{-d}
so that FP64 never overflows.
"""
from __future__ import annotations

import math

import numpy as np


def theta(beta, P=None, omega=1.0):
    """theta_P and d theta_P / d beta (P=None: continuum theta = beta omega / 2)."""
    if P is None:
        return 0.5 * beta * omega, 0.5 * omega
    x = beta * omega / (2.0 * P)
    return P * math.asinh(x), 0.5 * omega / math.sqrt(1.0 + x * x)


def energy(N, beta, P=None, d=2, xi=1.0, omega=1.0):
    """Exact E = -d ln Z_N / d beta (finite P, or continuum when P is None)."""
    th, dth = theta(beta, P, omega)
    k = np.arange(1, N + 1, dtype=np.float64)
    q = np.exp(-2.0 * k * th)
    zt = (1.0 - q) ** (-d)                          # z(k) e^{d k theta}
    dzt = zt * (-d) * (2.0 * k * dth * q) / (1.0 - q)  # d/d beta of zt
    w = np.array([xi ** (kk - 1) if kk > 1 else 1.0 for kk in range(1, N + 1)])
    Z = np.zeros(N + 1)
    D = np.zeros(N + 1)
    Z[0] = 1.0
    for n in range(1, N + 1):
        a = w[:n] * zt[:n]
        b = w[:n] * dzt[:n]
        Zrev = Z[n - 1::-1]
        Drev = D[n - 1::-1]
        Z[n] = float(np.dot(a, Zrev)) / n
        D[n] = (float(np.dot(b, Zrev)) + float(np.dot(a, Drev))) / n
    return d * N * dth - D[N] / Z[N]


def energy_mp(N, beta, P=None, d=2, xi=1.0, omega=1.0, dps=60):
    """Same quantity in mpmath arithmetic (small N), without the rescaling."""
    import mpmath as mp

    with mp.workdps(dps):
        beta = mp.mpf(beta)
        omega = mp.mpf(omega)
        xi = mp.mpf(xi)
        if P is None:
            th = beta * omega / 2
            dth = omega / 2
        else:
            x = beta * omega / (2 * P)
            th = P * mp.asinh(x)
            dth = (omega / 2) / mp.sqrt(1 + x * x)
        z = [None] + [(2 * mp.sinh(k * th)) ** (-d) for k in range(1, N + 1)]
        dz = [None] + [-d * k * mp.coth(k * th) * dth * z[k] for k in range(1, N + 1)]
        Z = [mp.mpf(1)] + [mp.mpf(0)] * N
        D = [mp.mpf(0)] * (N + 1)
        for n in range(1, N + 1):
            sZ = mp.mpf(0)
            sD = mp.mpf(0)
            for k in range(1, n + 1):
                w = mp.mpf(1) if k == 1 else xi ** (k - 1)
                sZ += w * z[k] * Z[n - k]
                sD += w * (dz[k] * Z[n - k] + z[k] * D[n - k])
            Z[n] = sZ / n
            D[n] = sD / n
        return float(-D[N] / Z[N]), Z


def ring_partition(k, beta, P=None, d=2, omega=1.0):
    """z(k): partition function of one exchange ring of k particles."""
    th, _ = theta(beta, P, omega)
    return (2.0 * math.sinh(k * th)) ** (-d)


def bead_variance(beta, P, omega=1.0, m=1.0):
    """Variance of one Cartesian coordinate of any bead of a distinguishable
    trapped ring polymer (xi = 0, Sec. III springs k_s = m P / beta^2, trap
    weighted 1/P): the Gaussian weight exp(-beta x^T A x / 2) with
    A = k_s L + (m omega^2 / P) I, L the ring Laplacian (eigenvalues
    4 sin^2(pi k / P)), gives (1/P) sum_k 1 / (beta A_k)."""
    ks = m * P / beta**2
    return sum(1.0 / (beta * (ks * 4.0 * math.sin(math.pi * k / P) ** 2 + m * omega**2 / P))
               for k in range(P)) / P


def shell_probability(r1, r2, var, d):
    """Probability that an isotropic Gaussian point (variance var per
    coordinate) in d dimensions lies at radius in [r1, r2)."""
    if d == 1:
        return math.erf(r2 / math.sqrt(2 * var)) - math.erf(r1 / math.sqrt(2 * var))
    if d == 2:
        return math.exp(-r1 * r1 / (2 * var)) - math.exp(-r2 * r2 / (2 * var))
    def cdf(x):  # chi distribution with 3 degrees of freedom
        z = x / math.sqrt(2 * var)
        return math.erf(z) - 2 * z * math.exp(-z * z) / math.sqrt(math.pi)
    return cdf(r2) - cdf(r1)
