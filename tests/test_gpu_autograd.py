"""VBFunction (autograd of V_ends = V_xi - sum E_int) against the oracle and finite differences.

The gradient comes from the library's adjoint kernel (connection
probabilities, Sec. III); it is checked against (i) the oracle's forces with
the internal-spring part written out, (ii) central finite differences of the
forward value, (iii) torch.autograd.gradcheck, and the table-recompute mode
against the table-store mode.
"""
import numpy as np
import pytest

import oracle
from workloads import beads

pytestmark = pytest.mark.gpu


def _torch():
    return pytest.importorskip("torch")


def _ends(torch, r):
    P = r.shape[1]
    r1 = torch.tensor(np.ascontiguousarray(r[:, 0, :]), dtype=torch.float64, device="cuda")
    rP = torch.tensor(np.ascontiguousarray(r[:, P - 1, :]), dtype=torch.float64, device="cuda")
    return r1, rP


def _e_int_sum(r, beta):
    """sum_l E_int^(l) = 1/2 k sum_{l, j<P} |r_l^{j+1} - r_l^j|^2, k = P/beta^2 (Sec. III)."""
    P = r.shape[1]
    return 0.5 * P / beta ** 2 * float(np.sum(np.diff(r, axis=1) ** 2))


@pytest.mark.parametrize("N,P,d,beta,xi", [(1, 4, 2, 1.0, 1.0), (40, 8, 2, 2.0, 1.0), (257, 6, 3, 1.5, 0.5),
                                         (130, 4, 2, 2.0, 0.0), (600, 4, 1, 3.0, 1.0)])
def test_vb_value_and_gradient_match_oracle(N, P, d, beta, xi):
    torch = _torch()
    from paper_2404_02628_gb300.autograd import VB, vb_ends
    r = beads(N, P, d, 1200 + N)
    r1, rP = _ends(torch, r)
    r1.requires_grad_(True)
    rP.requires_grad_(True)
    vb = VB(N, P, d, beta, xi)
    V = vb_ends(r1, rP, vb)
    V.backward()
    F, info = oracle.forces(r, beta, xi, 0.0, 0.0, 0.5)
    V_ends = info["V_xi"] - _e_int_sum(r, beta)
    assert abs(float(V.detach()) - V_ends) < 1e-10 * max(1.0, abs(info["V_xi"]))
    k = P / beta ** 2
    # dV_ends/dr^1 = -F^1 - d(E_int)/dr^1 and dV_ends/dr^P = -F^P - d(E_int)/dr^P
    g1 = -F[:, 0, :] + k * (r[:, 1, :] - r[:, 0, :])
    gP = -F[:, P - 1, :] - k * (r[:, P - 1, :] - r[:, P - 2, :])
    scale = max(np.abs(g1).max(), np.abs(gP).max())
    assert np.abs(r1.grad.cpu().numpy() - g1).max() < 1e-10 * scale
    assert np.abs(rP.grad.cpu().numpy() - gP).max() < 1e-10 * scale
    vb.close()


@pytest.mark.parametrize("N,xi", [(200, 1.0), (10000, 1.0)])
def test_vb_gradient_finite_differences(N, xi):
    """Adjoint gradient against central differences on 64 random coordinates."""
    torch = _torch()
    from paper_2404_02628_gb300.autograd import VB, vb_ends
    P, d, beta = 32, 2, 3.0
    r = beads(N, P, d, 1300 + N)
    r1, rP = _ends(torch, r)
    r1.requires_grad_(True)
    rP.requires_grad_(True)
    vb = VB(N, P, d, beta, xi)
    V = vb_ends(r1, rP, vb)
    V.backward()
    g = [r1.grad.clone(), rP.grad.clone()]
    rng = np.random.default_rng(7)
    h = 1e-5
    errs = []
    with torch.no_grad():
        for _ in range(64):
            which, l, c = int(rng.integers(2)), int(rng.integers(N)), int(rng.integers(d))
            x = (r1 if which == 0 else rP)
            x0 = float(x[l, c])
            x[l, c] = x0 + h
            Vp = float(vb_ends(r1, rP, vb))
            x[l, c] = x0 - h
            Vm = float(vb_ends(r1, rP, vb))
            x[l, c] = x0
            fd = (Vp - Vm) / (2 * h)
            errs.append(abs(fd - float(g[which][l, c])))
    scale = max(float(g[0].abs().max()), float(g[1].abs().max()))
    assert max(errs) < 1e-6 * scale
    vb.close()


def test_vb_gradcheck_small():
    torch = _torch()
    from paper_2404_02628_gb300.autograd import VB, VBFunction
    N, P, d, beta, xi = 12, 4, 2, 1.0, 0.7
    r = beads(N, P, d, 1400)
    r1, rP = _ends(torch, r)
    r1.requires_grad_(True)
    rP.requires_grad_(True)
    vb = VB(N, P, d, beta, xi)
    assert torch.autograd.gradcheck(lambda a, b: VBFunction.apply(a, b, vb), (r1, rP), eps=1e-6, atol=1e-6,
                                    rtol=1e-5)
    vb.close()


def test_vb_recompute_equals_store():
    torch = _torch()
    import paper_2404_02628_gb300 as pkg
    from paper_2404_02628_gb300.autograd import VB, vb_ends
    N, P, d, beta, xi = 3000, 8, 2, 2.0, 0.8
    r = beads(N, P, d, 1500)
    out = []
    for mode in (pkg.TABLE_STORE, pkg.TABLE_RECOMPUTE):
        r1, rP = _ends(torch, r)
        r1.requires_grad_(True)
        rP.requires_grad_(True)
        vb = VB(N, P, d, beta, xi, table_mode=mode)
        V = vb_ends(r1, rP, vb)
        V.backward()
        out.append((float(V.detach()), r1.grad.cpu().numpy(), rP.grad.cpu().numpy(), vb.work_bytes))
        vb.close()
    (Vs, g1s, gPs, bs), (Vr, g1r, gPr, br) = out
    assert abs(Vs - Vr) < 1e-12 * abs(Vs)
    assert np.abs(g1s - g1r).max() < 1e-12 * np.abs(g1s).max()
    assert np.abs(gPs - gPr).max() < 1e-12 * np.abs(gPs).max()
    assert br < bs / 4


def test_vb_n40000_recompute():
    """N = 40000: the automatic mode recomputes the O(N^2) factors; the
    workspace stays O(N) and the gradient still matches central differences."""
    torch = _torch()
    from paper_2404_02628_gb300.autograd import VB, vb_ends
    N, P, d, beta, xi = 40000, 32, 2, 3.0, 1.0
    r = beads(N, P, d, 1600)
    r1, rP = _ends(torch, r)
    r1.requires_grad_(True)
    rP.requires_grad_(True)
    vb = VB(N, P, d, beta, xi)
    assert vb.work_bytes < 12 * N * (N + 1) // 2 // 50  # under 2% of the stored table
    V = vb_ends(r1, rP, vb)
    V.backward()
    assert np.isfinite(float(V.detach()))
    rng = np.random.default_rng(9)
    h = 1e-4
    scale = max(float(r1.grad.abs().max()), float(rP.grad.abs().max()))
    with torch.no_grad():
        for _ in range(6):
            which, l, c = int(rng.integers(2)), int(rng.integers(N)), int(rng.integers(d))
            x = (r1 if which == 0 else rP)
            gx = float((r1.grad if which == 0 else rP.grad)[l, c])
            x0 = float(x[l, c])
            x[l, c] = x0 + h
            Vp = float(vb_ends(r1, rP, vb))
            x[l, c] = x0 - h
            Vm = float(vb_ends(r1, rP, vb))
            x[l, c] = x0
            assert abs((Vp - Vm) / (2 * h) - gx) < 1e-5 * scale
    vb.close()
