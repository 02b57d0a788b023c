"""bench.py's multi-rank logic on CPU: world_size 2 over gloo (no GPU)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench

    dist = bench.init_dist("gloo")
    bench.barrier(None)
    m = bench.max_over_ranks(1.5 * (rank + 1))
    info = bench.dist_info()
    dist.destroy_process_group()
    q.put((rank, m, info))


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [3.0, 3.0]
    assert out[0][2] == (2, 0, 0) and out[1][2] == (2, 1, 1)


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(2.5) == 2.5


def test_kernel_work_table():
    import bench
    from workloads import WORKLOADS

    w = WORKLOADS["gauss1600"]
    rates = {"fp64_tflops": 1.2, "fp32_tflops": 74.0, "ex2_per_s": 1.0e13, "sms": 152}
    for name in ("exch_recursion", "exch_table", "pair", "md_pre", "md_post", "springs"):
        for r in (None, rates):
            bound, work, unit, peak, src = bench.kernel_work(name, w, r)
            assert bound in ("alu", "hbm", "mufu") and work > 0 and peak > 0
    assert bench.kernel_work("exch_finalize", w, rates) is None
    fr = bench.kernel_fractions({"md_pre": 15.0, "exch_band": 12.0, "exch_table": 16.0}, w, rates)
    assert set(fr) == {"md_pre", "exch_table"} and 0 < fr["md_pre"]["frac"] < 1


def test_reference_arm_line(capsys):
    """The reference arm (the oracle on the host cores) prints one JSON line
    with the contract's keys and the same workload config as the CUDA arm."""
    import json
    import types

    import bench
    from workloads import WORKLOADS

    args = types.SimpleNamespace(steps=1, warmup=1, workload="gauss1600")
    bench.run_reference(args)
    line = capsys.readouterr().out.strip().splitlines()[-1]
    d = json.loads(line)
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["value"] > 0
    assert d["config"] == bench.workload_config(dict(WORKLOADS["gauss1600"]), 1)
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
