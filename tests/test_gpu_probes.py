"""Measurement probes behind the roofline fractions: the throughput kernels
give plausible GB300 rates, and the chain-latency probe computes exactly the
product it claims to (checked against an FP64 numpy iteration), so its cycle
count belongs to real work."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    import torch

    import paper_2404_02628_gb300 as pkg
    sink = torch.zeros(4, dtype=torch.float64, device="cuda")
    r = pkg.pimd_probe_rates(sink.data_ptr(), torch.cuda.current_stream().cuda_stream)
    print(r)
    assert r["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 0.2 < r["fp64_tflops"] < 10.0
    assert 10.0 < r["fp32_tflops"] < 200.0
    assert 1e12 < r["ex2_per_s"] < 1e14


@pytest.mark.parametrize("split", [1, 2, 4])
def test_probe_chain_computes_the_chain_product(split):
    import paper_2404_02628_gb300 as pkg
    nblk, n_iter = 4, 64
    cyc, y, (Q, G, y0, s) = pkg.probe_chain_latency(split=split, nblk=nblk, n_iter=n_iter, seed=split)
    x = y0.copy()
    for it in range(n_iter):
        k = it % nblk
        x = Q[k] @ x + G[k] @ s
    assert np.abs(y - x).max() < 1e-12 * np.abs(x).max()
    print("split %d: %.0f cycles per chain iteration" % (split, cyc))
    assert 50 < cyc < 100000
