"""Device-side failures of the exchange-potential calls are visible to the caller.

A bounded cross-block wait that gives up inside pimd_vb_forward leaves NaN in
V (and in the gradients of a pimd_vb_backward that follows), and
pimd_vb_sync reports PIMD_ETIMEOUT; afterwards a fresh call on the same
workspace is correct again.  The give-up is forced with a one-poll wait limit
(PIMD_SPIN_LIMIT=1), so nothing faults or hangs.
"""
import math

import numpy as np
import pytest

import oracle
from workloads import beads

pytestmark = pytest.mark.gpu


def _ends(torch, r):
    P = r.shape[1]
    r1 = torch.tensor(np.ascontiguousarray(r[:, 0, :].T), dtype=torch.float64, device="cuda")
    rP = torch.tensor(np.ascontiguousarray(r[:, P - 1, :].T), dtype=torch.float64, device="cuda")
    return r1, rP


def _e_int_sum(r, beta):
    """sum_l E_int^(l) = 1/2 k sum_{l, j<P} |r_l^{j+1} - r_l^j|^2 with k = P/beta^2 (Sec. III)."""
    P = r.shape[1]
    return 0.5 * P / beta ** 2 * float(np.sum(np.diff(r, axis=1) ** 2))


def test_vb_timeout_gives_nan_and_status_then_recovers(monkeypatch):
    torch = pytest.importorskip("torch")
    import paper_2404_02628_gb300 as pkg
    pkg.load()
    N, P, d, beta, xi = 2000, 4, 2, 2.0, 1.0
    r = beads(N, P, d, 1901)
    r1, rP = _ends(torch, r)
    h = pkg.pimd_vb_create(N, P, d, beta, xi)
    nb = pkg.pimd_vb_workspace_bytes(h)
    work = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    base = (work.data_ptr() + 255) // 256 * 256
    st = torch.cuda.current_stream().cuda_stream
    V = torch.zeros(1, dtype=torch.float64, device="cuda")
    gV = torch.ones(1, dtype=torch.float64, device="cuda")
    g1 = torch.zeros_like(r1)
    gP = torch.zeros_like(rP)
    monkeypatch.setenv("PIMD_SPIN_LIMIT", "1")
    pkg.pimd_vb_forward(h, r1.data_ptr(), rP.data_ptr(), N, base, nb, V.data_ptr(), st)
    pkg.pimd_vb_backward(h, r1.data_ptr(), rP.data_ptr(), N, base, nb, gV.data_ptr(), g1.data_ptr(),
                         gP.data_ptr(), st)
    torch.cuda.synchronize()
    assert math.isnan(float(V.item()))
    assert bool(torch.isnan(g1).all()) and bool(torch.isnan(gP).all())
    with pytest.raises(pkg.PimdError) as ei:
        pkg.pimd_vb_sync(h, base, nb, st)
    assert ei.value.status == pkg.PIMD_ETIMEOUT
    monkeypatch.delenv("PIMD_SPIN_LIMIT")
    pkg.pimd_vb_forward(h, r1.data_ptr(), rP.data_ptr(), N, base, nb, V.data_ptr(), st)
    pkg.pimd_vb_sync(h, base, nb, st)
    _, info = oracle.forces(r, beta, xi, 0.0, 0.0, 0.5)
    ref = info["V_xi"] - _e_int_sum(r, beta)
    assert abs(float(V.item()) - ref) <= 1e-10 * abs(info["V_xi"])
    pkg.pimd_vb_destroy(h)


def test_vbfunction_raises_on_timeout(monkeypatch):
    torch = pytest.importorskip("torch")
    import paper_2404_02628_gb300 as pkg
    from paper_2404_02628_gb300.autograd import VB, vb_ends
    N, P, d, beta = 2000, 4, 2, 2.0
    r = beads(N, P, d, 1902)
    r1 = torch.tensor(r[:, 0, :], dtype=torch.float64, device="cuda")
    rP = torch.tensor(r[:, P - 1, :], dtype=torch.float64, device="cuda")
    vb = VB(N, P, d, beta, 1.0)
    monkeypatch.setenv("PIMD_SPIN_LIMIT", "1")
    with pytest.raises(pkg.PimdError) as ei:
        vb_ends(r1, rP, vb)
    assert ei.value.status == pkg.PIMD_ETIMEOUT
    monkeypatch.delenv("PIMD_SPIN_LIMIT")
    V = vb_ends(r1, rP, vb)
    assert math.isfinite(float(V))
    vb.close()
