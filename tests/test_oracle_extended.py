"""The oracle's extended-precision twin (same C source, every quantity long
double) against mpmath brute force, and against the FP64 oracle where FP64 is
well conditioned (no GPU)."""
import math

import numpy as np
import pytest

import oracle
from workloads import beads

from test_oracle_pins import E_def, compositions


def test_twin_has_a_wider_significand():
    assert oracle.extended_significand_bits() >= 64


def test_twin_matches_fp64_oracle_where_fp64_is_accurate():
    for N, P, d, beta, xi, seed in [(40, 6, 2, 1.0, 1.0, 3), (25, 4, 3, 1.5, 0.3, 4), (30, 5, 1, 2.0, 0.0, 5)]:
        r = beads(N, P, d, seed)
        Fx, ix = oracle.exchange_extended(r, beta, xi)
        F, i64 = oracle.forces(r, beta, xi, 0.0, 0.0, 0.5)
        assert float(np.abs(Fx.astype(np.float64) - F).max()) <= 1e-12 * float(np.abs(F).max())
        assert abs(float(ix["V_xi"]) - i64["V_xi"]) <= 1e-13 * abs(i64["V_xi"])
        assert abs(float(ix["spring"]) - i64["spring"]) <= 1e-12 * abs(i64["spring"])


def test_twin_forward_value_matches_mpmath_brute_force():
    """V_xi^[1,N] as the sum over every ring topology the forward recursion
    counts (Sec. III), in 50-digit arithmetic: the twin agrees far below FP64
    rounding."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    N, P, d, beta, xi = 7, 3, 2, 1.3, 0.6
    r = beads(N, P, d, 21)
    terms = []
    for blocks in compositions(1, N):
        t = mp.mpf(1)
        for a, b in blocks:
            t *= mp.mpf(xi) ** (b - a) / b * mp.exp(-mp.mpf(beta) * mp.mpf(E_def(r, beta, a, b)))
        terms.append(t)
    V_ref = -mp.log(mp.fsum(terms)) / beta
    _, ix = oracle.exchange_extended(r, beta, xi)
    # E_def evaluates the cycle energies in FP64 (relative 1e-16 each), which
    # bounds the agreement; the twin's own arithmetic is tighter
    assert abs(mp.mpf(float(ix["V_xi"])) - V_ref) < 1e-15 * abs(V_ref)
    eps_ld = float(np.finfo(np.longdouble).eps)
    assert abs(float(ix["V_xi"] - ix["V_xi_bwd"])) <= 64 * eps_ld * abs(float(ix["V_xi"]))


def test_fp64_oracle_distance_at_the_benchmarked_size():
    """Reading of Sec. III's probabilities at N = 1600, P = 32: the FP64 oracle's
    endpoint forces sit 1e-10..1e-8 from the extended result, because each
    probability's exponent is a difference of terms of size beta*|V_xi|
    (about 1e6 here); V_xi itself stays FP64-accurate."""
    r = beads(1600, 32, 2, 3)
    Fx, ix = oracle.exchange_extended(r, 3.0, 1.0)
    F, i64 = oracle.forces(r, 3.0, 1.0, 0.0, 0.0, 0.5)
    Fx = Fx.astype(np.float64)
    err = float(np.abs(F - Fx).max() / np.abs(Fx).max())
    assert 1e-11 < err < 1e-8, err
    assert abs(i64["V_xi"] - float(ix["V_xi"])) < 1e-14 * abs(float(ix["V_xi"]))
    assert 3.0 * abs(float(ix["V_xi"])) > 1e6
