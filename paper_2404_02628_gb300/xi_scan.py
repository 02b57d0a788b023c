"""xi scan and extrapolation to fermions (arXiv 2404.02628, Sec. I and Sec. IV D).

Fictitious identical particles with xi in [0, 1] have a non-negative path
weight exp(-beta (V_xi + U/P)), so they can be sampled; fermions (xi = -1)
cannot.  This workflow runs every xi of a scan as replicas of one batch (one
set of launches per step for all of them, pimd_batch_*), collects the energy
estimators, and extrapolates to xi = -1 with pimd_xi_extrapolate.  The MD and
estimators run in the library's kernels; this module only schedules the runs
and averages the sampled scalars (block averages for the error bars).
"""
from __future__ import annotations

import numpy as np

from . import Batch, pimd_xi_extrapolate


def block_mean(series, nblocks=20):
    """Mean and standard error of a sampled series from `nblocks` consecutive
    block averages (blocks long against the correlation time)."""
    x = np.asarray(series, dtype=np.float64)
    n = (len(x) // nblocks) * nblocks
    b = x[:n].reshape(nblocks, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / np.sqrt(nblocks))


def xi_scan(N, P, d, beta, xis, omega=1.0, g=0.0, s=0.5, replicas=4, equil_steps=10000, samples=10000,
            stride=10, seed=0, estimators=("E_prim", "E_vir"), nblocks=20, device="cuda", **cfg):
    """Runs len(xis) * replicas independent systems of N particles (one batch),
    equilibrates, then samples the estimators every `stride` steps.

    Returns {"xi": [...], name: {"E": [...], "sigma": [...]} for each
    estimator name}, one block-averaged mean per xi (replicas of the same xi
    averaged, their standard errors combined).  Initial beads and momenta
    come from pimd_batch_init_state with `seed`."""
    xis = [float(x) for x in xis]
    R = len(xis) * replicas
    B = Batch([N] * R, P, d, [beta] * R, [x for x in xis for _ in range(replicas)], omega, g, s,
              device=device, **cfg)
    try:
        B.init_state(seed)
        B.step(equil_steps)
        series = {name: np.empty((samples, R)) for name in estimators}
        for i in range(samples):
            B.step(stride)
            est = B.estimators()
            for name in estimators:
                series[name][i] = [e[name] for e in est]
    finally:
        B.close()
    out = {"xi": xis, "samples": samples, "stride": stride, "replicas": replicas, "equil_steps": equil_steps}
    for name in estimators:
        E, sig = [], []
        for k in range(len(xis)):
            ms = [block_mean(series[name][:, k * replicas + q], nblocks) for q in range(replicas)]
            E.append(float(np.mean([m for m, _ in ms])))
            sig.append(float(np.sqrt(np.sum([e * e for _, e in ms])) / replicas))
        out[name] = {"E": E, "sigma": sig}
    return out


def extrapolate(scan, estimator="E_prim", degree=2, xi_target=-1.0):
    """Fit of one estimator of a xi_scan result, evaluated at xi_target (fermions: -1)."""
    e = scan[estimator]
    v, vs, chi2, coef = pimd_xi_extrapolate(scan["xi"], e["E"], e["sigma"], degree, xi_target)
    return {"value": v, "sigma": vs, "chi2": chi2, "dof": len(scan["xi"]) - degree - 1, "coef": coef,
            "degree": degree, "xi_target": xi_target, "estimator": estimator}
