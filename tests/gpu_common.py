"""Helpers shared by the GPU parity tests (marshalling only)."""
import math

import numpy as np

import paper_2404_02628_gb300 as pkg


def amplitude(g, s):
    """A = g/(pi s^2): the Gaussian prefactor printed in the Hamiltonian of Sec. IV B."""
    return g / (math.pi * s * s)


def make_system(N, P, d, beta, omega, g, s, xi, r, p=None, **cfg):
    return pkg.System(N, P, d, beta, omega, g, s, xi, r=r, p=p, **cfg)


def rel_inf(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))
