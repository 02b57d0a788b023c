"""Seeded initial state, oracle side (TEST INFRASTRUCTURE ONLY).

Sec. IV draws the beads from a standard normal per coordinate and the momenta
from the Maxwell-Boltzmann distribution at kT = 1/beta.  The draws come from
splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used as a counter-based generator, written here
from its published definition, independently of the CUDA path:

    output i of stream s = mix(s + (i + 1) * 0x9E3779B97F4A7C15)
    mix(z): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
            z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31  (mod 2^64)

Coordinate (q, j, c, l) -- q = 0 beads, 1 momenta -- has counter
k = ((q P + j) d + c) N + l and uses outputs 2k, 2k + 1 as uniforms
u = ((x >> 11) + 1) 2^-53 in (0, 1]; the normal deviate is the cosine branch
of Box-Muller, z = sqrt(-2 ln u1) cos(2 pi u2).  Replica r of a batch uses
the stream whose seed is output r of stream `seed`.

Layout here is particle-major, like the rest of the oracle: r[l, j, c].
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64(seed: int, i) -> np.ndarray:
    """Outputs i (int or integer array) of the splitmix64 stream `seed`, as uint64."""
    i = np.asarray(i, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + (i + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, i) -> np.ndarray:
    """Uniforms in (0, 1]: the top 53 bits of output i, plus one unit of 2^-53."""
    x = splitmix64(seed, i)
    return ((x >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0**-53


def normal(seed: int, k) -> np.ndarray:
    """Standard normal deviate for counter k (uniforms 2k and 2k + 1)."""
    k = np.asarray(k, dtype=np.uint64)
    u1 = uniform(seed, 2 * k)
    u2 = uniform(seed, 2 * k + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def init_state(N: int, P: int, d: int, beta: float, seed: int, mass: float = 1.0):
    """(r, p), each of shape (N, P, d): beads ~ N(0, 1), momenta ~ N(0, m/beta)."""
    j, c, l = np.meshgrid(np.arange(P), np.arange(d), np.arange(N), indexing="ij")  # [P][d][N]
    out = []
    for q in (0, 1):
        k = ((q * P + j) * d + c) * N + l
        z = normal(seed, k.astype(np.uint64))
        out.append(np.ascontiguousarray(z.transpose(2, 0, 1)))
    r, p = out
    return r, np.sqrt(mass / beta) * p


def replica_seed(seed: int, r: int) -> int:
    """Seed of replica r in a batch: output r of the stream `seed`."""
    return int(splitmix64(seed, r))
