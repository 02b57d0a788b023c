"""Plain FP64 CPU oracle for the bosonic / fictitious-particle PIMD hot path.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
``cpu_baseline`` / ``--impl reference`` legs are the only users.  It shares no
code with the CUDA path (``paper_2404_02628_gb300``) and never imports it.

The arithmetic lives in ``pimd_oracle.c`` (literal formulas of arXiv
2404.02628, Sec. III and IV) and ``exact.py`` (closed-form canonical energies
of trapped ideal bosons).  This module only compiles the C file and marshals
numpy arrays through ctypes.

Configuration layout here is particle-major: ``r[l, j, c]`` = component ``c``
of bead ``j`` of particle ``l`` (shape ``(N, P, d)``, float64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pimd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_LIB_LD = os.path.join(_BUILD, "liborc_ld.so")
_lock = threading.Lock()
_lib = None
_lib_ld = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class ForceInfo(ctypes.Structure):
    _fields_ = [("V_xi", ctypes.c_double), ("V_xi_bwd", ctypes.c_double),
                ("U_over_P", ctypes.c_double), ("spring", ctypes.c_double),
                ("virial", ctypes.c_double)]


class Estimates(ctypes.Structure):
    _fields_ = [("E_prim", ctypes.c_double), ("E_vir", ctypes.c_double),
                ("V_xi", ctypes.c_double), ("U_over_P", ctypes.c_double),
                ("kinetic", ctypes.c_double), ("spring", ctypes.c_double),
                ("H_conserved", ctypes.c_double), ("virial", ctypes.c_double)]


ESTIMATE_FIELDS = [f[0] for f in Estimates._fields_]


def _compile(out, defines, force):
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    tmp = out + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"] + defines + [
        "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, no FMA contraction) into oracle/_build:
    the FP64 library and its extended-precision twin (same source, every
    quantity ``long double``: 64-bit significand on x86-64, IEEE binary128 on
    aarch64)."""
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        _compile(_LIB_LD, ["-DORC_REAL=long double"], force)
        return _compile(_LIB, [], force)


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        L.orc_E_int.restype = ctypes.c_double
        L.orc_E_int.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_int]
        L.orc_cycle_energies.argtypes = [ctypes.c_int] * 3 + [_dp, ctypes.c_double, _dp]
        L.orc_V_forward.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, _dp]
        L.orc_V_backward.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, _dp]
        L.orc_connection_probabilities.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_double,
                                                   ctypes.c_double, _dp]
        L.orc_exchange_forces.argtypes = [ctypes.c_int] * 3 + [_dp, ctypes.c_double, _dp, _dp]
        L.orc_spring_expectation.restype = ctypes.c_double
        L.orc_spring_expectation.argtypes = [ctypes.c_int] * 3 + [_dp, ctypes.c_double, _dp]
        L.orc_interaction.argtypes = [ctypes.c_int] * 3 + [_dp] + [ctypes.c_double] * 3 + [_dp, _dp, _dp]
        L.orc_forces.restype = ctypes.c_int
        L.orc_forces.argtypes = [ctypes.c_int] * 3 + [_dp] + [ctypes.c_double] * 5 + [
            _dp, ctypes.POINTER(ForceInfo), _dp]
        L.orc_md_run.restype = ctypes.c_int
        L.orc_md_run.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_double] * 6 + [ctypes.c_int]
                                 + [ctypes.c_double] * 2 + [ctypes.c_int] + [_dp] * 5
                                 + [_ip, ctypes.c_int, ctypes.POINTER(Estimates)])
        L.orc_estimators.restype = ctypes.c_int
        L.orc_estimators.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_double] * 5 + [ctypes.c_int]
                                     + [ctypes.c_double] * 2 + [ctypes.c_int] + [_dp] * 4
                                     + [ctypes.POINTER(Estimates)])
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_dp)


def _conf(r):
    r = np.ascontiguousarray(r, dtype=np.float64)
    if r.ndim != 3:
        raise ValueError("configuration must have shape (N, P, d)")
    return r


# --------------------------------------------------------------------------
# Sec. III building blocks

def E_int(r, beta, v):
    """E_int^(v) for 1-based particle index v."""
    r = _conf(r)
    N, P, d = r.shape
    return lib().orc_E_int(P, d, _p(r), beta, v)


def cycle_energies(r, beta):
    """E[u-1, v-1] = E^[u,v] for u <= v by the quadratic iteration (zeros below)."""
    r = _conf(r)
    N, P, d = r.shape
    E = np.zeros((N, N))
    lib().orc_cycle_energies(N, P, d, _p(r), beta, _p(E))
    return E


def V_forward(E, beta, xi):
    """Vf[l] = V^[1,l] for l = 0..N."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    N = E.shape[0]
    Vf = np.zeros(N + 1)
    lib().orc_V_forward(N, _p(E), beta, xi, _p(Vf))
    return Vf


def V_backward(E, beta, xi):
    """Vb[u-1] = V^[u,N] for u = 1..N+1."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    N = E.shape[0]
    Vb = np.zeros(N + 1)
    lib().orc_V_backward(N, _p(E), beta, xi, _p(Vb))
    return Vb


def connection_probabilities(E, Vf, Vb, beta, xi):
    """Pr[l-1, l'-1] = Pr[G(l) = l'] for l = 1..N, l' = 1..N+1."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    N = E.shape[0]
    Vf = np.ascontiguousarray(Vf, dtype=np.float64)
    Vb = np.ascontiguousarray(Vb, dtype=np.float64)
    Pr = np.zeros((N, N + 1))
    lib().orc_connection_probabilities(N, _p(E), _p(Vf), _p(Vb), beta, xi, _p(Pr))
    return Pr


def exchange_forces(r, beta, Pr):
    r = _conf(r)
    N, P, d = r.shape
    Pr = np.ascontiguousarray(Pr, dtype=np.float64)
    F = np.zeros_like(r)
    lib().orc_exchange_forces(N, P, d, _p(r), beta, _p(Pr), _p(F))
    return F


def spring_expectation(r, beta, Pr):
    r = _conf(r)
    N, P, d = r.shape
    Pr = np.ascontiguousarray(Pr, dtype=np.float64)
    return lib().orc_spring_expectation(N, P, d, _p(r), beta, _p(Pr))


def interaction(r, omega, A, s):
    """Returns (U, F = -grad(U/P), virial = sum r.grad U)."""
    r = _conf(r)
    N, P, d = r.shape
    F = np.zeros_like(r)
    U = ctypes.c_double()
    vir = ctypes.c_double()
    lib().orc_interaction(N, P, d, _p(r), omega, A, s, ctypes.byref(U), _p(F), ctypes.byref(vir))
    return U.value, F, vir.value


def forces(r, beta, xi, omega=1.0, A=0.0, s=1.0, want_pr=False):
    """F = -grad(V_xi + U/P) and a dict of per-configuration scalars."""
    r = _conf(r)
    N, P, d = r.shape
    F = np.zeros_like(r)
    info = ForceInfo()
    Pr = np.zeros((N, N + 1)) if want_pr else None
    rc = lib().orc_forces(N, P, d, _p(r), beta, xi, omega, A, s, _p(F), ctypes.byref(info),
                          _p(Pr) if want_pr else None)
    if rc:
        raise ValueError("oracle rejected the arguments")
    out = {f[0]: getattr(info, f[0]) for f in ForceInfo._fields_}
    if want_pr:
        return F, out, Pr
    return F, out


def forces_species(r, counts, beta, xi, omega=1.0, A=0.0, s=1.0):
    """Several species (Sec. II, closing paragraph): each species -- counts[k]
    consecutive particles -- carries its own exchange potential from the
    Sec. III recursions over its own particles; the trap and the pairs act
    between all particles.  F = -grad(sum_k V_xi(species k) + U/P) and a dict
    of scalars (V_xi and spring summed over species, per-species V_xi in
    "V_species")."""
    r = _conf(r)
    N, P, d = r.shape
    if sum(counts) != N or min(counts) < 1:
        raise ValueError("species counts must be positive and add up to N")
    F = np.zeros_like(r)
    V, spring, Vs = 0.0, 0.0, []
    off = 0
    for n in counts:
        Fk, ik = forces(r[off:off + n], beta, xi, 0.0, 0.0, s)  # exchange part only (no trap, no pairs)
        F[off:off + n] += Fk
        V += ik["V_xi"]
        spring += ik["spring"]
        Vs.append(ik["V_xi"])
        off += n
    U, Fi, vir = interaction(r, omega, A, s)
    F += Fi
    return F, {"V_xi": V, "spring": spring, "U_over_P": U / P, "virial": vir, "V_species": Vs}


class MDState:
    """Oracle MD state: r, p of shape (N, P, d); eta, peta of shape (N, P, d, M)."""

    def __init__(self, r, p, M):
        self.r = np.array(r, dtype=np.float64, order="C")
        self.p = np.array(p, dtype=np.float64, order="C")
        self.M = int(M)
        self.eta = np.zeros(self.r.shape + (self.M,))
        self.peta = np.zeros(self.r.shape + (self.M,))
        self.F = np.zeros_like(self.r)
        self.have_forces = ctypes.c_int(0)

    def copy(self):
        o = MDState(self.r, self.p, self.M)
        o.eta[...] = self.eta
        o.peta[...] = self.peta
        o.F[...] = self.F
        o.have_forces = ctypes.c_int(self.have_forces.value)
        return o


def md_run(state, beta, xi, omega, A, s, dt, Q, nsteps, mass=1.0, thermostat=True):
    """Advance ``state`` by nsteps; returns a structured array of estimators per step."""
    N, P, d = state.r.shape
    est = (Estimates * max(nsteps, 1))()
    rc = lib().orc_md_run(N, P, d, beta, xi, omega, A, s, dt, state.M, Q, mass,
                          1 if thermostat else 0, _p(state.r), _p(state.p), _p(state.eta),
                          _p(state.peta), _p(state.F), ctypes.byref(state.have_forces),
                          nsteps, est)
    if rc:
        raise ValueError("oracle rejected the arguments")
    flat = np.ctypeslib.as_array(ctypes.cast(est, _dp), shape=(max(nsteps, 1) * len(ESTIMATE_FIELDS),))
    return flat.reshape(max(nsteps, 1), len(ESTIMATE_FIELDS))[:nsteps].copy()


def estimators(state, beta, xi, omega, A, s, Q, mass=1.0, thermostat=True):
    N, P, d = state.r.shape
    est = Estimates()
    rc = lib().orc_estimators(N, P, d, beta, xi, omega, A, s, state.M, Q, mass,
                              1 if thermostat else 0, _p(state.r), _p(state.p), _p(state.eta),
                              _p(state.peta), ctypes.byref(est))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return {f: getattr(est, f) for f in ESTIMATE_FIELDS}


def radial_density(r, nbins, r_max):
    """Radial bead density of one configuration (Sec. IV B density profiles),
    per particle: rho_b = n_b / (N P V_b), where n_b counts the beads with
    floor(sqrt(r2) / dr) = b, dr = r_max / nbins, r2 = x_0^2 + ... summed in
    component order with IEEE rounding after every operation, and V_b is the
    d-dimensional volume of shell b.  Beads at or beyond r_max are dropped.
    Returns (rho[nbins], counts[nbins])."""
    r = np.asarray(r, dtype=np.float64)
    N, P, d = r.shape
    dr = r_max / nbins
    r2 = np.zeros((N, P))
    for c in range(d):
        x = r[:, :, c]
        r2 = r2 + x * x
    t = np.floor(np.sqrt(r2) / dr)
    t = t[t < nbins].astype(np.int64)
    counts = np.bincount(t, minlength=nbins)[:nbins]
    edges = np.arange(nbins + 1) * dr
    if d == 1:
        vol = 2.0 * (edges[1:] - edges[:-1])
    elif d == 2:
        vol = np.pi * (edges[1:] ** 2 - edges[:-1] ** 2)
    else:
        vol = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    return counts / (N * P * vol), counts


# --------------------------------------------------------------------------
# Extended-precision twin (same C source, every quantity long double): how far
# FP64 evaluations of the exchange part sit from the exact value of the same
# formulas.  Inputs are converted exactly (float64 -> long double).

_ldp = ctypes.POINTER(ctypes.c_longdouble)


def lib_ld():
    global _lib_ld
    if _lib_ld is None:
        build()
        L = ctypes.CDLL(_LIB_LD)
        L.orc_cycle_energies.argtypes = [ctypes.c_int] * 3 + [_ldp, ctypes.c_longdouble, _ldp]
        L.orc_V_forward.argtypes = [ctypes.c_int, _ldp, ctypes.c_longdouble, ctypes.c_longdouble, _ldp]
        L.orc_V_backward.argtypes = [ctypes.c_int, _ldp, ctypes.c_longdouble, ctypes.c_longdouble, _ldp]
        L.orc_connection_probabilities.argtypes = [ctypes.c_int, _ldp, _ldp, _ldp, ctypes.c_longdouble,
                                                   ctypes.c_longdouble, _ldp]
        L.orc_exchange_forces.argtypes = [ctypes.c_int] * 3 + [_ldp, ctypes.c_longdouble, _ldp, _ldp]
        L.orc_spring_expectation.restype = ctypes.c_longdouble
        L.orc_spring_expectation.argtypes = [ctypes.c_int] * 3 + [_ldp, ctypes.c_longdouble, _ldp]
        _lib_ld = L
    return _lib_ld


def _pl(a):
    return a.ctypes.data_as(_ldp)


def extended_significand_bits():
    """Significand bits of the extended twin's type (53 would mean no gain)."""
    return int(np.finfo(np.longdouble).nmant) + 1


def exchange_extended(r, beta, xi):
    """Exchange part in extended precision: (F, info) with F = -grad V_xi
    (shape (N, P, d), np.longdouble) and info holding V_xi, V_xi_bwd and the
    expected spring energy as np.longdouble; same formulas and order as the
    FP64 oracle (Sec. III)."""
    r64 = _conf(r)
    N, P, d = r64.shape
    L = lib_ld()
    rl = np.ascontiguousarray(r64, dtype=np.longdouble)
    b = ctypes.c_longdouble(beta)
    x = ctypes.c_longdouble(xi)
    E = np.zeros((N, N), dtype=np.longdouble)
    L.orc_cycle_energies(N, P, d, _pl(rl), b, _pl(E))
    Vf = np.zeros(N + 1, dtype=np.longdouble)
    Vb = np.zeros(N + 1, dtype=np.longdouble)
    L.orc_V_forward(N, _pl(E), b, x, _pl(Vf))
    L.orc_V_backward(N, _pl(E), b, x, _pl(Vb))
    Pr = np.zeros((N, N + 1), dtype=np.longdouble)
    L.orc_connection_probabilities(N, _pl(E), _pl(Vf), _pl(Vb), b, x, _pl(Pr))
    del E
    F = np.zeros_like(rl)
    L.orc_exchange_forces(N, P, d, _pl(rl), b, _pl(Pr), _pl(F))
    spring = L.orc_spring_expectation(N, P, d, _pl(rl), b, _pl(Pr))
    return F, {"V_xi": Vf[N], "V_xi_bwd": Vb[0], "spring": np.longdouble(spring)}
