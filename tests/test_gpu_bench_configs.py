"""Oracle parity on the exact configurations bench.py times.

- gauss1600 (N=1600, P=32, beta=3, xi=1, Gaussian g=1, s=0.5): mixed precision
  (FP32 springs, pairs and thermostat chain) with the autotuned launch shape
  against the FP64 oracle at 1e-5, forces and three MD steps; the same
  workload in FP64 mode, both exchange arithmetics, against the oracle's
  extended-precision twin at 1e-10.  The FP64 oracle itself sits about 1e-9
  from the extended result here (its probability exponents are differences
  of numbers of size beta*|V_xi|), so the FP64 bar is checked against the
  extended twin, which evaluates the same formulas in the same order.
- ideal10000 (N=10000, P=32, beta=3, g=0, mixed, autotuned): forces at 1e-5
  and V_xi at 1e-10 against the FP64 oracle.
- the 64-replica batch as benched (uneven N, beta, xi; g=3; mixed with the
  FP32 thermostat; autotuned): every replica's forces against the oracle at
  bind and after five graph-replayed steps.
"""
import numpy as np
import pytest

import oracle
from gpu_common import amplitude, rel_inf
from workloads import BATCH64, WORKLOADS, batch_replicas, beads, momenta

pytestmark = pytest.mark.gpu
TOL64 = 1e-10
TOLMIX = 1e-5


def _system(pkg, w, **kw):
    r = beads(w["N"], w["P"], w["d"], w["seed"])
    p = momenta(w["N"], w["P"], w["d"], w["beta"], w["seed"])
    prec = kw.pop("precision", pkg.PREC_MIXED if w["precision"] == "mixed" else pkg.PREC_FP64)
    kw.setdefault("nhc_fp32", w.get("nhc_fp32", 0))
    S = pkg.System(w["N"], w["P"], w["d"], w["beta"], w["omega"], w["g"], w["s"], w["xi"], r=r, p=p,
                   precision=prec, nhc_len=w["M"], dt=w["dt"], **kw)
    return S, r


def test_gauss1600_mixed_as_benched():
    import paper_2404_02628_gb300 as pkg
    w = WORKLOADS["gauss1600"]
    S, r = _system(pkg, w)
    S.autotune(None)
    V = S.forces()
    F = S.forces_array()
    Fo, info = oracle.forces(r, w["beta"], w["xi"], w["omega"], amplitude(w["g"], w["s"]), w["s"])
    assert rel_inf(F, Fo) < TOLMIX
    Vo = info["V_xi"] + info["U_over_P"]
    assert abs(V - Vo) < TOLMIX * abs(Vo)
    est = S.estimators()
    # the exchange potential and the spring expectation are FP64-accurate in mixed mode
    assert abs(est["V_xi"] - info["V_xi"]) < TOL64 * abs(info["V_xi"])
    assert abs(est["U_over_P"] - info["U_over_P"]) < TOLMIX * abs(info["U_over_P"])
    S.close()


@pytest.fixture(scope="module")
def gauss1600_extended():
    w = WORKLOADS["gauss1600"]
    r = beads(w["N"], w["P"], w["d"], w["seed"])
    Fx, info = oracle.exchange_extended(r, w["beta"], w["xi"])
    U, Fi, vir = oracle.interaction(r, w["omega"], amplitude(w["g"], w["s"]), w["s"])
    F64, i64 = oracle.forces(r, w["beta"], w["xi"], w["omega"], amplitude(w["g"], w["s"]), w["s"])
    return {"F": Fx + Fi.astype(np.longdouble), "V_xi": info["V_xi"], "spring": info["spring"],
            "U_over_P": U / w["P"], "F64": F64, "i64": i64}


@pytest.mark.parametrize("arith", [0, 1])
def test_gauss1600_fp64_against_extended_oracle(gauss1600_extended, arith):
    import paper_2404_02628_gb300 as pkg
    ref = gauss1600_extended
    w = WORKLOADS["gauss1600"]
    S, r = _system(pkg, w, precision=pkg.PREC_FP64, exchange_arith=arith, nhc_fp32=0)
    S.autotune(None)
    S.forces()
    F = S.forces_array().astype(np.longdouble)
    Fref = ref["F"]
    err = float(np.abs(F - Fref).max() / np.abs(Fref).max())
    # the FP64 oracle's own distance from the extended result, for the record
    err64 = float(np.abs(ref["F64"].astype(np.longdouble) - Fref).max() / np.abs(Fref).max())
    print("arith %d: GPU vs extended %.3e, FP64 oracle vs extended %.3e" % (arith, err, err64))
    assert err < TOL64
    est = S.estimators()
    assert abs(est["V_xi"] - float(ref["V_xi"])) < TOL64 * abs(float(ref["V_xi"]))
    assert abs(est["spring"] - float(ref["spring"])) < TOL64 * abs(float(ref["spring"]))
    assert abs(est["U_over_P"] - ref["U_over_P"]) < TOL64 * abs(ref["U_over_P"])
    S.close()


def test_gauss1600_md_steps_as_benched():
    """Three MD steps of the benched gauss1600 system (mixed precision with the
    FP32 thermostat chain, autotuned) against three FP64 steps of the oracle
    from the same state: positions within 1e-7 and momenta within 1e-5
    (infinity norm, relative), the energies within 1e-5."""
    import paper_2404_02628_gb300 as pkg
    w = WORKLOADS["gauss1600"]
    S, r = _system(pkg, w)
    S.autotune(None)
    S.forces()
    S.step(3)
    x, p, est = S.positions(), S.momenta(), S.estimators()
    S.close()
    st = oracle.MDState(r, momenta(w["N"], w["P"], w["d"], w["beta"], w["seed"]), w["M"])
    oest = oracle.md_run(st, w["beta"], w["xi"], w["omega"], amplitude(w["g"], w["s"]), w["s"], w["dt"],
                         w["beta"] / w["P"], 3)
    assert rel_inf(x, st.r) < 1e-7
    assert rel_inf(p, st.p) < 1e-5
    for k in ("E_prim", "E_vir", "H_conserved"):
        ref = oest[-1, oracle.ESTIMATE_FIELDS.index(k)]
        assert abs(est[k] - ref) < 1e-5 * abs(ref), k


def test_ideal10000_as_benched():
    import paper_2404_02628_gb300 as pkg
    w = WORKLOADS["ideal10000"]
    S, r = _system(pkg, w)
    S.autotune(None)
    S.forces()
    F = S.forces_array()
    est = S.estimators()
    S.close()
    Fo, info = oracle.forces(r, w["beta"], w["xi"], w["omega"], 0.0, w["s"])
    assert rel_inf(F, Fo) < TOLMIX
    assert abs(est["V_xi"] - info["V_xi"]) < TOL64 * abs(info["V_xi"])
    assert abs(est["V_xi_bwd"] - info["V_xi"]) < TOL64 * abs(info["V_xi"])


def test_batch64_as_benched():
    import paper_2404_02628_gb300 as pkg
    reps = batch_replicas()
    cfg = BATCH64
    P, d = cfg["P"], cfg["d"]
    rs = [beads(q["N"], P, d, q["seed"]) for q in reps]
    ps = [momenta(q["N"], P, d, q["beta"], q["seed"]) for q in reps]
    B = pkg.Batch([q["N"] for q in reps], P, d, [q["beta"] for q in reps], [q["xi"] for q in reps],
                  cfg["omega"], cfg["g"], cfg["s"], rs=rs, ps=ps, precision=pkg.PREC_MIXED,
                  nhc_len=cfg["M"], dt=cfg["dt"], nhc_fp32=1)
    B.autotune(None)
    B.forces()
    A = amplitude(cfg["g"], cfg["s"])
    for q, rep in enumerate(reps):
        Fo, _ = oracle.forces(rs[q], rep["beta"], rep["xi"], cfg["omega"], A, cfg["s"])
        assert rel_inf(B.forces_array(q), Fo) < TOLMIX, q
    B.step(5)
    est = B.estimators()
    for q, rep in enumerate(reps):
        x = B.positions(q)
        Fo, info = oracle.forces(x, rep["beta"], rep["xi"], cfg["omega"], A, cfg["s"])
        assert rel_inf(B.forces_array(q), Fo) < TOLMIX, q
        assert abs(est[q]["V_xi"] - info["V_xi"]) < TOL64 * max(1.0, abs(info["V_xi"])), q
        assert est[q]["step"] == 5
    B.close()
