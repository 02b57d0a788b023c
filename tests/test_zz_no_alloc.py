"""The allocation-free exchange-potential entry point against the workspace one.

pimd_vb_forward_noalloc serves callers that hand the library only their input
and output arrays and cannot allocate device memory for a workspace.  It must
give the same V_ends as pimd_vb_forward, on consecutive calls that reuse its
fixed scratch.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import paper_2404_02628_gb300 as pkg
from workloads import beads

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _endpoints(torch, N, P, d, seed):
    r = beads(N, P, d, seed)
    r1 = torch.tensor(np.ascontiguousarray(r[:, 0, :].T), dtype=torch.float64, device="cuda")
    rP = torch.tensor(np.ascontiguousarray(r[:, P - 1, :].T), dtype=torch.float64, device="cuda")
    return r1, rP


def _with_workspace(torch, N, P, d, beta, xi, r1, rP, stream):
    h = pkg.pimd_vb_create(N, P, d, beta, xi)
    try:
        nb = pkg.pimd_vb_workspace_bytes(h)
        work = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        base = (work.data_ptr() + 255) // 256 * 256
        V = torch.zeros(1, dtype=torch.float64, device="cuda")
        pkg.pimd_vb_forward(h, r1.data_ptr(), rP.data_ptr(), N, base, nb, V.data_ptr(), stream)
        torch.cuda.synchronize()
        return float(V.item())
    finally:
        pkg.pimd_vb_destroy(h)


def test_noalloc_matches_workspace_entry_point_twice():
    torch = pytest.importorskip("torch")
    pkg.load()
    stream = torch.cuda.current_stream().cuda_stream
    # the documented limit N = 1024, a ragged N, d = 3 and the xi = 0 branch
    # (V from the diagonal chain only)
    cases = [(300, 8, 2, 2.0, 1.0, 11), (257, 6, 2, 1.5, 0.4, 12), (1024, 8, 2, 2.0, 1.0, 13),
             (333, 6, 3, 1.5, 0.0, 14)]
    for N, P, d, beta, xi, seed in cases:
        r1, rP = _endpoints(torch, N, P, d, seed)
        ref = _with_workspace(torch, N, P, d, beta, xi, r1, rP, stream)
        V = torch.zeros(1, dtype=torch.float64, device="cuda")
        pkg.pimd_vb_forward_noalloc(N, P, d, beta, xi, r1.data_ptr(), rP.data_ptr(), N, V.data_ptr(), stream)
        torch.cuda.synchronize()
        got = float(V.item())
        assert abs(got - ref) <= TOL * abs(ref), (N, got, ref)


def test_noalloc_timeout_writes_nan_then_recovers(monkeypatch):
    """A bounded wait that gives up (one-poll limit via PIMD_SPIN_LIMIT) makes
    the call write NaN, since the call itself does not synchronise; the next
    call with the normal limit gives the right value from the same scratch."""
    torch = pytest.importorskip("torch")
    pkg.load()
    stream = torch.cuda.current_stream().cuda_stream
    N, P, d, beta, xi = 1024, 4, 2, 2.0, 1.0
    r1, rP = _endpoints(torch, N, P, d, 15)
    V = torch.zeros(1, dtype=torch.float64, device="cuda")
    monkeypatch.setenv("PIMD_SPIN_LIMIT", "1")
    pkg.pimd_vb_forward_noalloc(N, P, d, beta, xi, r1.data_ptr(), rP.data_ptr(), N, V.data_ptr(), stream)
    torch.cuda.synchronize()
    assert np.isnan(float(V.item()))
    monkeypatch.delenv("PIMD_SPIN_LIMIT")
    ref = _with_workspace(torch, N, P, d, beta, xi, r1, rP, stream)
    pkg.pimd_vb_forward_noalloc(N, P, d, beta, xi, r1.data_ptr(), rP.data_ptr(), N, V.data_ptr(), stream)
    torch.cuda.synchronize()
    assert abs(float(V.item()) - ref) <= TOL * abs(ref)


def test_noalloc_rejects_oversized_problem():
    pkg.load()
    with pytest.raises(pkg.PimdError) as ei:
        pkg.pimd_vb_forward_noalloc(1025, 8, 2, 2.0, 1.0, 1, 1, 1025, 1, None)
    assert ei.value.status == pkg.PIMD_EINVAL
    assert "1024" in str(ei.value)
