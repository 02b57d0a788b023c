"""torch.autograd wrapper of the exchange potential's endpoint part.

V_ends(r^1, r^P) = V_xi^[1,N] - sum_l E_int^(l) is the part of the exchange
potential (arXiv 2404.02628, Sec. III forward recursion) that depends on the
endpoint beads only.  Its gradient is the adjoint of that recursion: the
connection probabilities Pr[G(l) = l'] weight the spring vectors between
bead P of particle l and bead 1 of particle l' (Sec. III, exterior-bead
forces).  Both directions run in the library's kernels (pimd_vb_forward /
pimd_vb_backward); this module only marshals tensors.
"""
import torch

from . import (pimd_vb_backward, pimd_vb_create, pimd_vb_destroy, pimd_vb_forward, pimd_vb_set_table_mode,
               pimd_vb_sync, pimd_vb_workspace_bytes)


class VB:
    """Handle + workspace for V_ends of N particles, P beads, d dimensions.

    table_mode: None (store up to N = 16383, recompute above), or the
    package's TABLE_STORE / TABLE_RECOMPUTE.
    check: after each forward and backward, synchronise and raise PimdError
    (PIMD_ETIMEOUT) if a bounded device wait gave up (pimd_vb_sync).  With
    check=False the calls stay asynchronous and a failed call shows up as
    NaN in V and the gradients.
    """

    def __init__(self, N, P, d, beta, xi, device="cuda", table_mode=None, check=True):
        self.N, self.P, self.d, self.beta, self.xi = N, P, d, beta, xi
        self.check = check
        self.h = pimd_vb_create(N, P, d, beta, xi)
        if table_mode is not None:
            pimd_vb_set_table_mode(self.h, table_mode)
        self.work_bytes = pimd_vb_workspace_bytes(self.h)
        self.work = torch.empty(self.work_bytes + 256, dtype=torch.uint8, device=device)
        self.work_ptr = (self.work.data_ptr() + 255) // 256 * 256
        self.generation = 0  # forward calls so far; backward needs its own forward's state

    def close(self):
        if self.h:
            pimd_vb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _forward(self, r1c, rPc, V):
        stream = torch.cuda.current_stream(r1c.device).cuda_stream
        pimd_vb_forward(self.h, r1c.data_ptr(), rPc.data_ptr(), self.N, self.work_ptr, self.work_bytes,
                        V.data_ptr(), stream)
        self.generation += 1
        self._check(stream)
        return self.generation

    def _check(self, stream):
        if self.check:
            pimd_vb_sync(self.h, self.work_ptr, self.work_bytes, stream)


def _component_major(x, N, d):
    if x.shape != (N, d) or x.dtype != torch.float64 or not x.is_cuda:
        raise ValueError("expected a float64 CUDA tensor of shape (N, d)")
    return x.detach().t().contiguous()  # [d][N], leading dimension N


class VBFunction(torch.autograd.Function):
    """V = V_ends(r1, rP) for r1, rP of shape (N, d) (beads 1 and P)."""

    @staticmethod
    def forward(ctx, r1, rP, vb):
        r1c = _component_major(r1, vb.N, vb.d)
        rPc = _component_major(rP, vb.N, vb.d)
        V = torch.empty(1, dtype=torch.float64, device=r1.device)
        ctx.gen = vb._forward(r1c, rPc, V)
        ctx.vb = vb
        ctx.save_for_backward(r1c, rPc)
        return V[0]

    @staticmethod
    def backward(ctx, gV):
        vb = ctx.vb
        r1c, rPc = ctx.saved_tensors
        if vb.generation != ctx.gen:  # another forward reused the workspace: redo this one's
            scratch = torch.empty(1, dtype=torch.float64, device=r1c.device)
            vb._forward(r1c, rPc, scratch)
        g = gV.detach().to(torch.float64).reshape(1).contiguous()
        g1 = torch.empty_like(r1c)
        gP = torch.empty_like(rPc)
        stream = torch.cuda.current_stream(r1c.device).cuda_stream
        pimd_vb_backward(vb.h, r1c.data_ptr(), rPc.data_ptr(), vb.N, vb.work_ptr, vb.work_bytes, g.data_ptr(),
                         g1.data_ptr(), gP.data_ptr(), stream)
        vb._check(stream)
        return g1.t(), gP.t(), None


def vb_ends(r1, rP, vb):
    """V_ends(r1, rP) with autograd support."""
    return VBFunction.apply(r1, rP, vb)
