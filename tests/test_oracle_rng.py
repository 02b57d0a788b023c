"""Pins of the oracle's seeded initial state (oracle/rng.py), no GPU.

The generator is splitmix64 used counter-wise; its outputs for seed 0 are
pinned to the published reference sequence (tests/golden), the uniform and
normal deviates to their distributions (Kolmogorov-Smirnov tests against the
exact CDFs), and the state to the variances Sec. IV fixes: beads N(0, 1),
momenta N(0, m/beta).
"""
import os

import numpy as np
import pytest

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            rows.append(line.split())
    return rows


def test_splitmix64_reference_outputs():
    for i, hexval in _golden("splitmix64_seed0.txt"):
        assert int(rng.splitmix64(0, int(i))) == int(hexval, 16)


def test_uniforms_are_uniform_on_half_open_unit_interval():
    stats = pytest.importorskip("scipy.stats")
    u = rng.uniform(12345, np.arange(200000, dtype=np.uint64))
    assert u.min() > 0.0 and u.max() <= 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    # no correlation between neighbouring counters (1 / sqrt(n) ~ 2.2e-3)
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.015


def test_box_muller_normals():
    stats = pytest.importorskip("scipy.stats")
    z = rng.normal(7, np.arange(200000, dtype=np.uint64))
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)


@pytest.mark.parametrize("N,P,d,beta,mass", [(300, 16, 2, 3.0, 1.0), (101, 7, 3, 0.5, 2.0)])
def test_initial_state_variances(N, P, d, beta, mass):
    r, p = rng.init_state(N, P, d, beta, 99, mass=mass)
    assert r.shape == p.shape == (N, P, d)
    n = r.size
    assert abs(r.var() - 1.0) < 6 * np.sqrt(2.0 / n)
    assert abs(p.var() / (mass / beta) - 1.0) < 6 * np.sqrt(2.0 / n)
    # beads and momenta come from disjoint counters: uncorrelated
    assert abs(np.corrcoef(r.ravel(), p.ravel())[0, 1]) < 6 / np.sqrt(n)


def test_counter_layout_and_seeds():
    N, P, d = 5, 3, 2
    r, p = rng.init_state(N, P, d, 1.0, 42)
    # coordinate (q=0, j, c, l) uses counter (j d + c) N + l
    j, c, l = 2, 1, 4
    assert r[l, j, c] == rng.normal(42, (j * d + c) * N + l)
    assert p[l, j, c] == rng.normal(42, ((P + j) * d + c) * N + l)
    r2, _ = rng.init_state(N, P, d, 1.0, 43)
    assert not np.array_equal(r, r2)
    assert rng.replica_seed(0, 0) == 0xe220a8397b1dcdaf
