"""GB300-native bosonic / fictitious-particle PIMD hot path (arXiv 2404.02628).

Thin ctypes binding of the C ABI declared in ``include/pimd.h``.  Every step
of the path runs in the sm_103a kernels of ``_build/libpimd.so``; this module
only marshals arguments.  PyTorch provides device memory and streams.  There
is no CPU fallback: if the library is missing or no GPU is present, the calls
raise.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

__all__ = [
    "PIMD_OK", "PimdError", "Config", "Buffers", "BatchBuffers", "Estimates", "lib", "load", "symbols", "Batch",
    "pimd_create", "pimd_default_config", "pimd_configure", "pimd_workspace_bytes", "pimd_bind",
    "pimd_forces", "pimd_exchange_forces", "pimd_interaction_forces", "pimd_step", "pimd_step_eager",
    "pimd_estimators", "pimd_state_bytes", "pimd_get_state", "pimd_set_state", "pimd_sync",
    "pimd_last_error", "pimd_global_error", "pimd_destroy", "pimd_vb_create", "pimd_vb_workspace_bytes",
    "pimd_vb_forward", "pimd_vb_backward", "pimd_vb_destroy", "pimd_vb_sync", "pimd_vb_set_table_mode", "pimd_step_profiled",
    "pimd_profile_slot_name", "pimd_vb_forward_noalloc", "System",
    "pimd_batch_create", "pimd_batch_configure", "pimd_batch_layout", "pimd_batch_workspace_bytes",
    "pimd_batch_bind", "pimd_batch_forces", "pimd_batch_capture_graph", "pimd_batch_step",
    "pimd_batch_step_eager", "pimd_batch_step_profiled", "pimd_batch_profile_slot_name",
    "pimd_batch_estimators", "pimd_batch_sync", "pimd_batch_last_error", "pimd_batch_destroy",
    "pimd_batch_autotune", "pimd_autotune", "pimd_tuning", "pimd_init_state", "pimd_batch_init_state",
    "pimd_density_accumulate", "pimd_batch_tuning", "pimd_batch_schedule", "pimd_cycle_energies_naive",
    "pimd_xi_extrapolate",
    "pimd_set_species", "pimd_probe_rates", "pimd_probe_chain", "probe_chain_latency",
]

PIMD_OK, PIMD_EINVAL, PIMD_ENOMEM, PIMD_ECUDA, PIMD_ETIMEOUT, PIMD_ENONFINITE, PIMD_ESTATE = range(7)
STATUS_NAMES = {0: "PIMD_OK", 1: "PIMD_EINVAL", 2: "PIMD_ENOMEM", 3: "PIMD_ECUDA", 4: "PIMD_ETIMEOUT",
                5: "PIMD_ENONFINITE", 6: "PIMD_ESTATE"}
PREC_FP64, PREC_MIXED = 0, 1
AMP_PAPER, AMP_RAW = 0, 1
TABLE_STORE, TABLE_RECOMPUTE = 0, 1
XARITH_DF, XARITH_FP64 = 0, 1
BATCH_PERSISTENT, BATCH_KERNELS = 0, 1

LIB_PATH = _build.LIB


class PimdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("nhc_len", ctypes.c_int), ("nhc_Q", ctypes.c_double),
                ("mass", ctypes.c_double), ("precision", ctypes.c_int), ("amp_convention", ctypes.c_int),
                ("table_mode", ctypes.c_int), ("thermostat", ctypes.c_int), ("helper_ctas", ctypes.c_int),
                ("spin_limit", ctypes.c_int), ("exchange_arith", ctypes.c_int), ("exch_band", ctypes.c_int),
                ("nhc_fp32", ctypes.c_int), ("batch_schedule", ctypes.c_int)]


class Buffers(ctypes.Structure):
    _fields_ = [("r", ctypes.c_void_p), ("p", ctypes.c_void_p), ("f", ctypes.c_void_p),
                ("eta", ctypes.c_void_p), ("peta", ctypes.c_void_p), ("work", ctypes.c_void_p),
                ("work_bytes", ctypes.c_size_t), ("n_pad", ctypes.c_int)]


class BatchBuffers(ctypes.Structure):
    _fields_ = [("r", ctypes.c_void_p), ("p", ctypes.c_void_p), ("f", ctypes.c_void_p),
                ("eta", ctypes.c_void_p), ("peta", ctypes.c_void_p), ("work", ctypes.c_void_p),
                ("work_bytes", ctypes.c_size_t)]


class Rates(ctypes.Structure):
    _fields_ = [("fp64_tflops", ctypes.c_double), ("fp32_tflops", ctypes.c_double), ("ex2_per_s", ctypes.c_double),
                ("sms", ctypes.c_int)]


class Estimates(ctypes.Structure):
    _fields_ = [("E_prim", ctypes.c_double), ("E_vir", ctypes.c_double), ("V_xi", ctypes.c_double),
                ("U_over_P", ctypes.c_double), ("kinetic", ctypes.c_double), ("spring", ctypes.c_double),
                ("H_conserved", ctypes.c_double), ("virial", ctypes.c_double), ("V_xi_bwd", ctypes.c_double),
                ("step", ctypes.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "pimd_create": ([ctypes.c_int] * 3 + [ctypes.c_double] * 5 + [ctypes.POINTER(_vp)], ctypes.c_int),
    "pimd_default_config": ([ctypes.POINTER(Config)], None),
    "pimd_configure": ([_vp, ctypes.POINTER(Config)], ctypes.c_int),
    "pimd_workspace_bytes": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "pimd_bind": ([_vp, ctypes.POINTER(Buffers), _vp], ctypes.c_int),
    "pimd_forces": ([_vp, _dp], ctypes.c_int),
    "pimd_exchange_forces": ([_vp, _vp, _dp], ctypes.c_int),
    "pimd_interaction_forces": ([_vp, _vp, _dp], ctypes.c_int),
    "pimd_step": ([_vp, ctypes.c_int], ctypes.c_int),
    "pimd_step_eager": ([_vp, ctypes.c_int], ctypes.c_int),
    "pimd_estimators": ([_vp, ctypes.POINTER(Estimates)], ctypes.c_int),
    "pimd_state_bytes": ([_vp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "pimd_get_state": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "pimd_set_state": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "pimd_sync": ([_vp], ctypes.c_int),
    "pimd_last_error": ([_vp], ctypes.c_char_p),
    "pimd_global_error": ([], ctypes.c_char_p),
    "pimd_destroy": ([_vp], None),
    "pimd_vb_create": ([ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [ctypes.POINTER(_vp)], ctypes.c_int),
    "pimd_vb_workspace_bytes": ([_vp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "pimd_vb_set_table_mode": ([_vp, ctypes.c_int], ctypes.c_int),
    "pimd_vb_forward": ([_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_size_t, _vp, _vp], ctypes.c_int),
    "pimd_vb_backward": ([_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_size_t, _vp, _vp, _vp, _vp], ctypes.c_int),
    "pimd_vb_destroy": ([_vp], None),
    "pimd_vb_sync": ([_vp, _vp, ctypes.c_size_t, _vp], ctypes.c_int),
    "pimd_step_profiled": ([_vp, ctypes.c_int, _dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "pimd_profile_slot_name": ([_vp, ctypes.c_int], ctypes.c_char_p),
    "pimd_vb_forward_noalloc": ([ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [_vp, _vp, ctypes.c_int, _vp, _vp],
                                ctypes.c_int),
    "pimd_batch_create": ([ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, _dp, _dp]
                          + [ctypes.c_double] * 3 + [ctypes.POINTER(_vp)], ctypes.c_int),
    "pimd_batch_configure": ([_vp, ctypes.POINTER(Config)], ctypes.c_int),
    "pimd_batch_layout": ([_vp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "pimd_batch_workspace_bytes": ([_vp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "pimd_batch_bind": ([_vp, ctypes.POINTER(BatchBuffers), _vp], ctypes.c_int),
    "pimd_batch_forces": ([_vp], ctypes.c_int),
    "pimd_batch_capture_graph": ([_vp], ctypes.c_int),
    "pimd_batch_step": ([_vp, ctypes.c_int], ctypes.c_int),
    "pimd_batch_step_eager": ([_vp, ctypes.c_int], ctypes.c_int),
    "pimd_batch_step_profiled": ([_vp, ctypes.c_int, _dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "pimd_batch_profile_slot_name": ([_vp, ctypes.c_int], ctypes.c_char_p),
    "pimd_batch_estimators": ([_vp, ctypes.POINTER(Estimates)], ctypes.c_int),
    "pimd_batch_sync": ([_vp], ctypes.c_int),
    "pimd_batch_last_error": ([_vp], ctypes.c_char_p),
    "pimd_batch_destroy": ([_vp], None),
    "pimd_autotune": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "pimd_density_accumulate": ([_vp, ctypes.c_int, ctypes.c_double, _vp], ctypes.c_int),
    "pimd_batch_tuning": ([_vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "pimd_batch_schedule": ([_vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "pimd_init_state": ([_vp, ctypes.c_ulonglong], ctypes.c_int),
    "pimd_batch_init_state": ([_vp, ctypes.c_ulonglong], ctypes.c_int),
    "pimd_tuning": ([_vp] + [ctypes.POINTER(ctypes.c_int)] * 5, ctypes.c_int),
    "pimd_batch_autotune": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "pimd_cycle_energies_naive": ([_vp, _vp, ctypes.c_int], ctypes.c_int),
    "pimd_set_species": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "pimd_probe_rates": ([_vp, ctypes.POINTER(Rates), _vp], ctypes.c_int),
    "pimd_probe_chain": ([ctypes.c_int] * 3 + [_vp] * 7, ctypes.c_int),
    "pimd_xi_extrapolate": ([ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp],
                            ctypes.c_int),
}


def symbols():
    """Names of every entry point declared in include/pimd.h that the binding wraps."""
    return list(_SIGS)


def load(path=None):
    """Load the C-ABI library (no compilation, no GPU needed to load)."""
    global _lib
    if _lib is None:
        path = path or LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError("libpimd.so is not built (run __graft_entry__.build()); no CPU fallback exists")
        L = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def lib():
    return load()


def _check(status, handle=None):
    if status != PIMD_OK:
        L = lib()
        msg = L.pimd_last_error(handle) if handle else L.pimd_global_error()
        raise PimdError(status, (msg or b"").decode())
    return status


def _bcheck(status, handle=None):
    if status != PIMD_OK:
        L = lib()
        msg = L.pimd_batch_last_error(handle) if handle else L.pimd_global_error()
        raise PimdError(status, (msg or b"").decode())
    return status


# ---- one-to-one wrappers (same names as the C ABI) ------------------------

def pimd_create(N, P, d, beta, omega, g, s, xi):
    h = _vp()
    _check(lib().pimd_create(N, P, d, beta, omega, g, s, xi, ctypes.byref(h)))
    return h


def pimd_set_species(h, counts):
    n = len(counts)
    return _check(lib().pimd_set_species(h, n, (ctypes.c_int * n)(*[int(x) for x in counts])), h)


def pimd_probe_rates(sink_ptr, stream):
    """Measured FP64 / FP32 FMA and MUFU ex2 throughput of the current device."""
    out = Rates()
    st = lib().pimd_probe_rates(sink_ptr, ctypes.byref(out), stream)
    if st != PIMD_OK:
        raise PimdError(st, "pimd_probe_rates failed")
    return {f: getattr(out, f) for f, _ in Rates._fields_}


def pimd_probe_chain(nblk, n_iter, split, Q, G, y0, s, y_out, cycles, stream):
    st = lib().pimd_probe_chain(nblk, n_iter, split, Q, G, y0, s, y_out, cycles, stream)
    if st != PIMD_OK:
        raise PimdError(st, "pimd_probe_chain: bad argument or launch failure")
    return st


def pimd_default_config():
    c = Config()
    lib().pimd_default_config(ctypes.byref(c))
    return c


def pimd_configure(h, cfg):
    return _check(lib().pimd_configure(h, ctypes.byref(cfg)), h)


def pimd_workspace_bytes(h, n_pad):
    n = ctypes.c_size_t()
    _check(lib().pimd_workspace_bytes(h, n_pad, ctypes.byref(n)), h)
    return n.value


def pimd_bind(h, bufs, stream):
    return _check(lib().pimd_bind(h, ctypes.byref(bufs), stream), h)


def pimd_forces(h, want_value=True):
    v = ctypes.c_double()
    _check(lib().pimd_forces(h, ctypes.byref(v) if want_value else None), h)
    return v.value if want_value else None


def pimd_exchange_forces(h, f_ptr, want_value=True):
    v = ctypes.c_double()
    _check(lib().pimd_exchange_forces(h, f_ptr, ctypes.byref(v) if want_value else None), h)
    return v.value if want_value else None


def pimd_interaction_forces(h, f_ptr, want_value=True):
    v = ctypes.c_double()
    _check(lib().pimd_interaction_forces(h, f_ptr, ctypes.byref(v) if want_value else None), h)
    return v.value if want_value else None


def pimd_step(h, nsteps):
    return _check(lib().pimd_step(h, nsteps), h)


def pimd_step_eager(h, nsteps):
    return _check(lib().pimd_step_eager(h, nsteps), h)


def pimd_step_profiled(h, nsteps, max_slots=64):
    """Eager steps with per-kernel CUDA-event times; returns [(name, total_ms)]."""
    ms = (ctypes.c_double * max_slots)()
    n = ctypes.c_int()
    _check(lib().pimd_step_profiled(h, nsteps, ms, max_slots, ctypes.byref(n)), h)
    return [((lib().pimd_profile_slot_name(h, i) or b"").decode(), ms[i]) for i in range(n.value)]


def pimd_profile_slot_name(h, slot):
    return (lib().pimd_profile_slot_name(h, slot) or b"").decode()


def pimd_estimators(h):
    e = Estimates()
    _check(lib().pimd_estimators(h, ctypes.byref(e)), h)
    return e.as_dict()


def pimd_state_bytes(h):
    n = ctypes.c_size_t()
    _check(lib().pimd_state_bytes(h, ctypes.byref(n)), h)
    return n.value


def pimd_get_state(h, host_ptr, nbytes):
    return _check(lib().pimd_get_state(h, host_ptr, nbytes), h)


def pimd_set_state(h, host_ptr, nbytes):
    return _check(lib().pimd_set_state(h, host_ptr, nbytes), h)


def pimd_sync(h):
    return _check(lib().pimd_sync(h), h)


def pimd_last_error(h):
    return (lib().pimd_last_error(h) or b"").decode()


def pimd_global_error():
    return (lib().pimd_global_error() or b"").decode()


def pimd_destroy(h):
    lib().pimd_destroy(h)


def pimd_vb_create(N, P, d, beta, xi):
    h = _vp()
    _check(lib().pimd_vb_create(N, P, d, beta, xi, ctypes.byref(h)))
    return h


def pimd_vb_set_table_mode(h, mode):
    return _check(lib().pimd_vb_set_table_mode(h, mode))


def pimd_vb_workspace_bytes(h):
    n = ctypes.c_size_t()
    _check(lib().pimd_vb_workspace_bytes(h, ctypes.byref(n)))
    return n.value


def pimd_vb_forward(h, r1, rP, ld, work, work_bytes, V_out, stream):
    return _check(lib().pimd_vb_forward(h, r1, rP, ld, work, work_bytes, V_out, stream))


def pimd_vb_backward(h, r1, rP, ld, work, work_bytes, gV, g_r1, g_rP, stream):
    return _check(lib().pimd_vb_backward(h, r1, rP, ld, work, work_bytes, gV, g_r1, g_rP, stream))


def pimd_vb_sync(h, work, work_bytes, stream):
    return _check(lib().pimd_vb_sync(h, work, work_bytes, stream))


def pimd_vb_destroy(h):
    lib().pimd_vb_destroy(h)


def pimd_vb_forward_noalloc(N, P, d, beta, xi, r1, rP, ld, V_out, stream):
    """V_ends without a caller workspace (library-owned fixed scratch, N <= 1024)."""
    return _check(lib().pimd_vb_forward_noalloc(N, P, d, beta, xi, r1, rP, ld, V_out, stream))


# ---- batched replicas ---------------------------------------------------------

def pimd_batch_create(Ns, P, d, betas, xis, omega, g, s):
    R = len(Ns)
    h = _vp()
    _bcheck(lib().pimd_batch_create(R, (ctypes.c_int * R)(*Ns), P, d, (ctypes.c_double * R)(*betas),
                                    (ctypes.c_double * R)(*xis), omega, g, s, ctypes.byref(h)))
    return h


def pimd_batch_configure(h, cfg):
    return _bcheck(lib().pimd_batch_configure(h, ctypes.byref(cfg)), h)


def pimd_batch_layout(h, R):
    off = (ctypes.c_size_t * (R + 1))()
    _bcheck(lib().pimd_batch_layout(h, off), h)
    return list(off)


def pimd_batch_workspace_bytes(h):
    n = ctypes.c_size_t()
    _bcheck(lib().pimd_batch_workspace_bytes(h, ctypes.byref(n)), h)
    return n.value


def pimd_batch_bind(h, bufs, stream):
    return _bcheck(lib().pimd_batch_bind(h, ctypes.byref(bufs), stream), h)


def pimd_batch_forces(h):
    return _bcheck(lib().pimd_batch_forces(h), h)


def pimd_batch_capture_graph(h):
    return _bcheck(lib().pimd_batch_capture_graph(h), h)


def pimd_batch_step(h, nsteps):
    return _bcheck(lib().pimd_batch_step(h, nsteps), h)


def pimd_batch_step_eager(h, nsteps):
    return _bcheck(lib().pimd_batch_step_eager(h, nsteps), h)


def pimd_batch_step_profiled(h, nsteps, max_slots=64):
    ms = (ctypes.c_double * max_slots)()
    n = ctypes.c_int()
    _bcheck(lib().pimd_batch_step_profiled(h, nsteps, ms, max_slots, ctypes.byref(n)), h)
    return [(lib().pimd_batch_profile_slot_name(h, i).decode(), ms[i]) for i in range(n.value)]


def pimd_batch_profile_slot_name(h, slot):
    return lib().pimd_batch_profile_slot_name(h, slot).decode()


def pimd_batch_estimators(h, R):
    out = (Estimates * R)()
    _bcheck(lib().pimd_batch_estimators(h, out), h)
    return [e.as_dict() for e in out]


def pimd_batch_sync(h):
    return _bcheck(lib().pimd_batch_sync(h), h)


def pimd_batch_last_error(h):
    return (lib().pimd_batch_last_error(h) or b"").decode()


def pimd_batch_destroy(h):
    lib().pimd_batch_destroy(h)


def pimd_batch_autotune(h, cache_path=None):
    return _bcheck(lib().pimd_batch_autotune(h, cache_path.encode() if cache_path else None), h)


def pimd_density_accumulate(h, nbins, r_max, hist_ptr):
    return _check(lib().pimd_density_accumulate(h, int(nbins), float(r_max), hist_ptr), h)


def pimd_batch_tuning(h):
    T = ctypes.c_int()
    _bcheck(lib().pimd_batch_tuning(h, ctypes.byref(T)), h)
    S = ctypes.c_int()
    _bcheck(lib().pimd_batch_schedule(h, ctypes.byref(S)), h)
    return {"pair_block": T.value, "schedule": "persistent" if S.value == BATCH_PERSISTENT else "kernels"}


def pimd_batch_schedule(h):
    S = ctypes.c_int()
    _bcheck(lib().pimd_batch_schedule(h, ctypes.byref(S)), h)
    return S.value


def pimd_init_state(h, seed):
    return _check(lib().pimd_init_state(h, int(seed) & 0xFFFFFFFFFFFFFFFF), h)


def pimd_batch_init_state(h, seed):
    return _bcheck(lib().pimd_batch_init_state(h, int(seed) & 0xFFFFFFFFFFFFFFFF), h)


def pimd_cycle_energies_naive(h, E_ptr, ldE):
    return _check(lib().pimd_cycle_energies_naive(h, E_ptr, int(ldE)), h)


def pimd_xi_extrapolate(xi, E, sigma, degree=2, xi_target=-1.0):
    """Weighted least-squares polynomial in xi evaluated at xi_target (host
    call): returns (value, value_sigma, chi2, coef[constant first])."""
    n = len(xi)
    arr = ctypes.c_double * n
    v, vs, c2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    coef = (ctypes.c_double * (degree + 1))()
    st = lib().pimd_xi_extrapolate(n, arr(*map(float, xi)), arr(*map(float, E)), arr(*map(float, sigma)),
                                   int(degree), float(xi_target), ctypes.byref(v), ctypes.byref(vs),
                                   ctypes.byref(c2), coef)
    if st != PIMD_OK:
        raise PimdError(st, "pimd_xi_extrapolate: bad input or too few distinct xi for the degree")
    return v.value, vs.value, c2.value, list(coef)


def pimd_autotune(h, cache_path=None):
    return _check(lib().pimd_autotune(h, cache_path.encode() if cache_path else None), h)


def pimd_tuning(h):
    W, T, H, F, S = (ctypes.c_int() for _ in range(5))
    _check(lib().pimd_tuning(h, ctypes.byref(W), ctypes.byref(T), ctypes.byref(H), ctypes.byref(F),
                             ctypes.byref(S)), h)
    return {"exch_band": W.value, "pair_block": T.value, "helpers": H.value, "force_blocks": F.value,
            "streams": S.value}


def probe_chain_latency(split=2, nblk=4, n_iter=400, seed=0, device="cuda"):
    """Cycles per iteration of the recursion chain's dependent core
    (pimd_probe_chain) on seeded non-negative tiles scaled so the iterate stays
    O(1).  Returns (cycles_per_iteration, y_out, inputs) -- the inputs let a
    test recompute y_out in FP64."""
    import numpy as np
    import torch

    rng = np.random.default_rng(seed)
    Q = rng.random((nblk, 32, 32)) / 32.0
    G = rng.random((nblk, 32, 32)) / 32.0
    y0 = rng.random(32)
    s = rng.random(32)
    dev = torch.device(device)
    t = [torch.tensor(a, dtype=torch.float64, device=dev) for a in (Q, G, y0, s)]
    y = torch.zeros(32, dtype=torch.float64, device=dev)
    cyc = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    pimd_probe_chain(nblk, n_iter, split, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), t[3].data_ptr(),
                     y.data_ptr(), cyc.data_ptr(), stream)
    torch.cuda.synchronize(dev)
    return float(cyc.item()) / n_iter, y.cpu().numpy(), (Q, G, y0, s)


class Batch:
    """R replicas of uneven N, beta, xi in one set of torch-owned device arrays.

    ``rs`` and ``ps`` are lists of particle-major (N_r, P, d) arrays.  Replica
    r's slice-major block [P][d][n_pad_r] sits at element offset offsets[r] of
    the flat float64 tensors.  All arithmetic happens in the C ABI's kernels.
    """

    def __init__(self, Ns, P, d, betas, xis, omega=1.0, g=0.0, s=0.5, rs=None, ps=None, device="cuda",
                 stream=None, **cfg_kw):
        import torch

        self.torch = torch
        self.R, self.P, self.d = len(Ns), P, d
        self.Ns, self.betas, self.xis = list(Ns), list(betas), list(xis)
        self.h = pimd_batch_create(Ns, P, d, betas, xis, omega, g, s)
        cfg = pimd_default_config()
        for k, v in cfg_kw.items():
            setattr(cfg, k, v)
        pimd_batch_configure(self.h, cfg)
        self.cfg = cfg
        self.offsets = pimd_batch_layout(self.h, self.R)
        self.n_pad = [(n + 31) // 32 * 32 for n in Ns]
        dev = torch.device(device)
        f64 = torch.float64
        tot = self.offsets[-1]
        M = cfg.nhc_len
        self.r = torch.zeros(tot, dtype=f64, device=dev)
        self.p = torch.zeros_like(self.r)
        self.f = torch.zeros_like(self.r)
        self.eta = torch.zeros(M * tot, dtype=f64, device=dev)
        self.peta = torch.zeros_like(self.eta)
        nbytes = pimd_batch_workspace_bytes(self.h)
        self.work = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        self.work_ptr = (self.work.data_ptr() + 255) // 256 * 256
        for q in range(self.R):
            if rs is not None:
                self._view(self.r, q)[:, :, :Ns[q]] = torch.as_tensor(rs[q], dtype=f64).permute(1, 2, 0).to(dev)
            if ps is not None:
                self._view(self.p, q)[:, :, :Ns[q]] = torch.as_tensor(ps[q], dtype=f64).permute(1, 2, 0).to(dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.bufs = BatchBuffers(self.r.data_ptr(), self.p.data_ptr(), self.f.data_ptr(), self.eta.data_ptr(),
                                 self.peta.data_ptr(), self.work_ptr, nbytes)
        pimd_batch_bind(self.h, self.bufs, self.stream.cuda_stream)

    def _view(self, flat, q):
        a, b = self.offsets[q], self.offsets[q + 1]
        return flat[a:b].view(self.P, self.d, self.n_pad[q])

    def positions(self, q):
        return self._view(self.r, q)[:, :, :self.Ns[q]].permute(2, 0, 1).cpu().numpy()

    def momenta(self, q):
        return self._view(self.p, q)[:, :, :self.Ns[q]].permute(2, 0, 1).cpu().numpy()

    def forces_array(self, q):
        return self._view(self.f, q)[:, :, :self.Ns[q]].permute(2, 0, 1).cpu().numpy()

    def forces(self):
        pimd_batch_forces(self.h)

    def step(self, n=1, graph=True):
        (pimd_batch_step if graph else pimd_batch_step_eager)(self.h, n)

    def init_state(self, seed):
        """Seeded beads and momenta on the device for every replica (pimd_batch_init_state)."""
        pimd_batch_init_state(self.h, seed)

    def autotune(self, cache_path=None):
        pimd_batch_autotune(self.h, cache_path)
        return pimd_batch_tuning(self.h)

    def estimators(self):
        return pimd_batch_estimators(self.h, self.R)

    def sync(self):
        pimd_batch_sync(self.h)

    def close(self):
        if self.h:
            pimd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- convenience: torch-owned buffers ---------------------------------------

class System:
    """One PIMD system whose device buffers are torch tensors.

    ``r`` and ``p`` are given particle-major, shape (N, P, d) (host numpy or
    torch); the device copies live in slice-major (P, d, n_pad) float64
    tensors.  ``species``: particle counts of consecutive species, each with
    its own exchange recursion (None: one species).  All arithmetic happens
    in the C ABI's kernels.
    """

    def __init__(self, N, P, d, beta, omega=1.0, g=0.0, s=0.5, xi=1.0, r=None, p=None, device="cuda",
                 stream=None, species=None, **cfg_kw):
        import torch

        self.torch = torch
        self.N, self.P, self.d = N, P, d
        self.beta = beta
        self.h = pimd_create(N, P, d, beta, omega, g, s, xi)
        cfg = pimd_default_config()
        for k, v in cfg_kw.items():
            setattr(cfg, k, v)
        pimd_configure(self.h, cfg)
        if species is not None:  # particle counts per species, consecutive (pimd_set_species)
            pimd_set_species(self.h, list(species))
        self.cfg = cfg
        self.n_pad = (N + 31) // 32 * 32
        dev = torch.device(device)
        f64 = torch.float64
        self.r = torch.zeros((P, d, self.n_pad), dtype=f64, device=dev)
        self.p = torch.zeros_like(self.r)
        self.f = torch.zeros_like(self.r)
        M = cfg.nhc_len
        self.eta = torch.zeros((M, P, d, self.n_pad), dtype=f64, device=dev)
        self.peta = torch.zeros_like(self.eta)
        nbytes = pimd_workspace_bytes(self.h, self.n_pad)
        self.work = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self.work.data_ptr()
        self.work_ptr = (base + 255) // 256 * 256
        self.work_bytes = nbytes
        if r is not None:
            self.r[:, :, :N] = torch.as_tensor(r, dtype=f64).permute(1, 2, 0).to(dev)
        if p is not None:
            self.p[:, :, :N] = torch.as_tensor(p, dtype=f64).permute(1, 2, 0).to(dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.bufs = Buffers(self.r.data_ptr(), self.p.data_ptr(), self.f.data_ptr(), self.eta.data_ptr(),
                            self.peta.data_ptr(), self.work_ptr, nbytes, self.n_pad)
        pimd_bind(self.h, self.bufs, self.stream.cuda_stream)

    # particle-major views (host numpy)
    def positions(self):
        return self.r[:, :, :self.N].permute(2, 0, 1).cpu().numpy()

    def momenta(self):
        return self.p[:, :, :self.N].permute(2, 0, 1).cpu().numpy()

    def forces_array(self):
        return self.f[:, :, :self.N].permute(2, 0, 1).cpu().numpy()

    def forces(self):
        return pimd_forces(self.h)

    def exchange_forces(self):
        out = self.torch.zeros_like(self.r)
        V = pimd_exchange_forces(self.h, out.data_ptr())
        return out[:, :, :self.N].permute(2, 0, 1).cpu().numpy(), V

    def interaction_forces(self):
        out = self.torch.zeros_like(self.r)
        U = pimd_interaction_forces(self.h, out.data_ptr())
        return out[:, :, :self.N].permute(2, 0, 1).cpu().numpy(), U

    def step(self, n=1, graph=True):
        (pimd_step if graph else pimd_step_eager)(self.h, n)

    def density(self, nbins, r_max, hist=None):
        """Adds the radial bead density of the current configuration into
        ``hist`` (a float64 CUDA tensor of nbins, created zeroed if None) and
        returns it (pimd_density_accumulate)."""
        if hist is None:
            hist = self.torch.zeros(nbins, dtype=self.torch.float64, device=self.r.device)
        pimd_density_accumulate(self.h, nbins, r_max, hist.data_ptr())
        return hist

    def cycle_energies_naive(self):
        """E[u-1, v-1] = E^[u,v] for u <= v from the definition, one GPU thread
        per entry (pimd_cycle_energies_naive); zeros below the diagonal."""
        E = self.torch.zeros((self.N, self.N), dtype=self.torch.float64, device=self.r.device)
        pimd_cycle_energies_naive(self.h, E.data_ptr(), self.N)
        return E.cpu().numpy()

    def init_state(self, seed):
        """Seeded beads and momenta on the device (pimd_init_state)."""
        pimd_init_state(self.h, seed)

    def autotune(self, cache_path=None):
        pimd_autotune(self.h, cache_path)
        return pimd_tuning(self.h)

    def tuning(self):
        return pimd_tuning(self.h)

    def estimators(self):
        return pimd_estimators(self.h)

    def get_state(self):
        n = pimd_state_bytes(self.h)
        buf = (ctypes.c_char * n)()
        pimd_get_state(self.h, ctypes.addressof(buf), n)
        return bytes(buf)

    def set_state(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        pimd_set_state(self.h, ctypes.addressof(buf), len(blob))

    def sync(self):
        pimd_sync(self.h)

    def close(self):
        if self.h:
            pimd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
