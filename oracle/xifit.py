"""Reference of the xi extrapolation (TEST INFRASTRUCTURE ONLY, part of the oracle).

Fictitious identical particles (arXiv 2404.02628, Sec. I and Sec. IV D) are
simulated at xi in [0, 1] and an observable is carried to xi = -1 by a fit in
xi.  The paper does not print the fitting form; the reading used here (and
by the library's pimd_xi_extrapolate) is a polynomial in xi fitted by weighted
least squares with weights 1/sigma^2, quadratic by default.  Written from the
definition: minimise sum_i ((E_i - sum_k c_k xi_i^k) / sigma_i)^2, whose
parameter covariance is (A^T W A)^{-1} with A the Vandermonde matrix.
"""
from __future__ import annotations

import numpy as np


def extrapolate(xi, E, sigma, degree=2, xi_target=-1.0):
    """Returns (value, value_sigma, chi2, coef[constant first])."""
    xi = np.asarray(xi, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    A = np.vander(xi, degree + 1, increasing=True)
    Aw = A / sigma[:, None]
    coef, *_ = np.linalg.lstsq(Aw, E / sigma, rcond=None)
    cov = np.linalg.inv(Aw.T @ Aw)
    p = xi_target ** np.arange(degree + 1)
    value = float(p @ coef)
    value_sigma = float(np.sqrt(max(p @ cov @ p, 0.0)))
    chi2 = float(np.sum(((E - A @ coef) / sigma) ** 2))
    return value, value_sigma, chi2, coef
