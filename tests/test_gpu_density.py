"""Radial bead density (pimd_density_accumulate) against the oracle.

The bin of each bead is decided in FP64 with every operation rounded (sum of
squares in component order, correctly rounded sqrt and divide) on both
sides, so the counts agree exactly; the densities then agree to the rounding
of the weighted atomic additions (1e-13 relative).
"""
import math

import numpy as np
import pytest

import oracle
from workloads import beads

pytestmark = pytest.mark.gpu


def _vol(d, nbins, r_max):
    e = np.arange(nbins + 1) * (r_max / nbins)
    return {1: 2 * np.diff(e), 2: np.pi * np.diff(e**2), 3: 4 / 3 * np.pi * np.diff(e**3)}[d]


@pytest.mark.parametrize("N,P,d,nbins,r_max", [(1, 4, 2, 8, 3.0), (100, 8, 2, 64, 4.0), (257, 6, 3, 33, 3.5),
                                               (300, 4, 1, 100, 2.0), (1600, 32, 2, 256, 5.0)])
def test_density_matches_oracle(N, P, d, nbins, r_max):
    import paper_2404_02628_gb300 as pkg
    r = beads(N, P, d, 1800 + N)
    S = pkg.System(N, P, d, 2.0, 1.0, 0.0, 0.5, 1.0, r=r)
    h = S.density(nbins, r_max)
    h = S.density(nbins, r_max, h)  # accumulates: twice the single density
    rho = h.cpu().numpy() / 2
    rho_o, counts_o = oracle.radial_density(r, nbins, r_max)
    counts = np.rint(rho * N * P * _vol(d, nbins, r_max)).astype(np.int64)
    assert np.array_equal(counts, counts_o)
    assert np.abs(rho - rho_o).max() <= 1e-13 * max(np.abs(rho_o).max(), 1e-300)
    S.close()


def test_density_rejects_bad_arguments():
    import paper_2404_02628_gb300 as pkg
    S = pkg.System(10, 4, 2, 1.0, r=beads(10, 4, 2, 1))
    buf = S.torch.zeros(9000, dtype=S.torch.float64, device="cuda")
    for nb, rm in ((0, 1.0), (9000, 1.0), (10, 0.0), (10, float("nan")), (10, float("inf"))):
        with pytest.raises(pkg.PimdError):
            pkg.pimd_density_accumulate(S.h, nb, rm, buf.data_ptr())
    assert float(buf.abs().max()) == 0.0
    S.close()
