"""Seeded synthetic inputs shared by the tests, bench.py and smoke().

This module only draws random numbers and reorders arrays; it holds none of
the method's arithmetic.  Both the oracle (``oracle/``) and the CUDA path
(``paper_2404_02628_gb300``) receive what it produces.

Workloads (trapped bosons in d = 2, hbar = m = omega = 1, the systems of
arXiv 2404.02628 Sec. IV with P = 32 / 64 instead of 72):

  ideal16      N=16,    P=32, beta=2, xi=1, g=0        FP64, 20000 steps
  gauss100     N=100,   P=64, beta=3, xi=1, g=3, s=0.5 FP64
  gauss1600    N=1600,  P=32, beta=3, xi=1, g=1, s=0.5 mixed precision
               (FP32 springs, pairs and thermostat-chain arithmetic)
  batch64      64 replicas, N ~ U{32..512}, P=32, beta in {1,2,3,4},
               xi in {0,0.2,...,1}, g=3, s=0.5        mixed precision
  ideal10000   N=10000, P=32, beta=3, xi=1, g=0        FP64 exchange + FP32 springs

Beads are i.i.d. N(0,1) per coordinate; momenta N(0, m'/beta); Nose-Hoover
chain length 4; dt = 0.01.
"""
from __future__ import annotations

import numpy as np

WORKLOADS = {
    "ideal16": dict(N=16, P=32, d=2, beta=2.0, xi=1.0, g=0.0, s=0.5, omega=1.0,
                    precision="fp64", M=4, dt=0.01, seed=1),
    "gauss100": dict(N=100, P=64, d=2, beta=3.0, xi=1.0, g=3.0, s=0.5, omega=1.0,
                     precision="fp64", M=4, dt=0.01, seed=2),
    "gauss1600": dict(N=1600, P=32, d=2, beta=3.0, xi=1.0, g=1.0, s=0.5, omega=1.0,
                      precision="mixed", nhc_fp32=1, M=4, dt=0.01, seed=3),
    "ideal10000": dict(N=10000, P=32, d=2, beta=3.0, xi=1.0, g=0.0, s=0.5, omega=1.0,
                       precision="mixed", nhc_fp32=1, M=4, dt=0.01, seed=5),
    # the paper's own timing runs (Sec. IV A: ideal trapped bosons at beta = 6, P = 72)
    "paper1600": dict(N=1600, P=72, d=2, beta=6.0, xi=1.0, g=0.0, s=0.5, omega=1.0,
                      precision="mixed", nhc_fp32=1, M=4, dt=0.01, seed=6),
    "paper10000": dict(N=10000, P=72, d=2, beta=6.0, xi=1.0, g=0.0, s=0.5, omega=1.0,
                       precision="mixed", nhc_fp32=1, M=4, dt=0.01, seed=7),
}

BATCH64 = dict(R=64, N_lo=32, N_hi=512, P=32, d=2, betas=(1.0, 2.0, 3.0, 4.0),
               xis=(0.0, 0.2, 0.4, 0.6, 0.8, 1.0), g=3.0, s=0.5, omega=1.0,
               precision="mixed", M=4, dt=0.01, seed=4)


def beads(N, P, d, seed):
    """Bead configuration r[l, j, c] ~ N(0, 1), shape (N, P, d), float64."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, P, d))


def momenta(N, P, d, beta, seed, mass=1.0):
    """Momenta p[l, j, c] ~ N(0, mass/beta), shape (N, P, d), float64."""
    rng = np.random.default_rng(seed + 1_000_003)
    return rng.standard_normal((N, P, d)) * np.sqrt(mass / beta)


def to_slice_major(x, n_pad=None):
    """(N, P, d[, M]) particle-major -> (P, d, N_pad) or (M, P, d, N_pad), zero padded."""
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[0]
    n_pad = N if n_pad is None else n_pad
    if x.ndim == 3:
        out = np.zeros((x.shape[1], x.shape[2], n_pad))
        out[:, :, :N] = np.transpose(x, (1, 2, 0))
    else:
        out = np.zeros((x.shape[3], x.shape[1], x.shape[2], n_pad))
        out[:, :, :, :N] = np.transpose(x, (3, 1, 2, 0))
    return out


def from_slice_major(x, N):
    """Inverse of to_slice_major."""
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 3:
        return np.ascontiguousarray(np.transpose(x[:, :, :N], (2, 0, 1)))
    return np.ascontiguousarray(np.transpose(x[:, :, :, :N], (3, 1, 2, 0)))


def batch_replicas(cfg=BATCH64):
    """Replica list for the batched workload: dicts with N, beta, xi and a seed."""
    rng = np.random.default_rng(cfg["seed"])
    Ns = rng.integers(cfg["N_lo"], cfg["N_hi"] + 1, size=cfg["R"])
    out = []
    for r in range(cfg["R"]):
        out.append(dict(N=int(Ns[r]), P=cfg["P"], d=cfg["d"],
                        beta=cfg["betas"][r % len(cfg["betas"])],
                        xi=cfg["xis"][(r // len(cfg["betas"])) % len(cfg["xis"])],
                        g=cfg["g"], s=cfg["s"], omega=cfg["omega"], M=cfg["M"],
                        dt=cfg["dt"], seed=cfg["seed"] * 1000 + r))
    return out
