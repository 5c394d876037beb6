"""Theorem 2 (Sec. 3.1) through the GPU path on the plain-method shape.

A, B 256 x 256 with i.i.d. N(0, 1) entries stored as FP64, b = 1024, d = 1,
2000 independent hash draws (seeds 1..2000): every draw runs the library's
sketch (hash tables -> fused sketch kernel -> inverse) and the dense decode,
and the estimates' mean and variance over the draws are compared with what
the theorem fixes: the estimator is unbiased, with variance at most
||AB||_F^2 / b (exactly (||AB||_F^2 - AB_ij^2) / b for a collision
probability of 1/b).  AB itself is formed on the host in float64.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_1320_gb300 import build as b
    b.build()
    import paper_1108_1320_gb300 as m
    m.lib()
    return m


def test_theorem2_mean_and_variance_over_2000_draws(cms):
    dev = torch.device("cuda", torch.cuda.current_device())
    n, b, seeds = 256, 1024, 2000
    A = W.gaussian(n, n, 1)
    B = W.gaussian(n, n, 2)
    AB = A @ B
    fro2 = float((AB ** 2).sum())
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev).T      # column-major, float64
    Bd = torch.from_numpy(B).to(dev)
    h = cms.make_hashes(1, n, b, 1)
    ws = cms.alloc_workspace(cms.workspace_size(h, n, n, n, torch.float64), dev)
    c = torch.empty((1, b), dtype=torch.float32, device=dev)
    est = torch.empty((n, n), dtype=torch.float32, device=dev)
    s1 = torch.zeros((n, n), dtype=torch.float64, device=dev)
    s2 = torch.zeros((n, n), dtype=torch.float64, device=dev)
    for seed in range(1, seeds + 1):
        h.reseed(seed)
        cms.sketch_product(Ad, Bd, h, c=c, ws=ws)
        cms.decode_dense(c, h, n, n, out=est)
        e64 = est.double()
        s1 += e64
        s2 += e64 * e64
    torch.cuda.synchronize()
    cms.check_async()
    mean = (s1 / seeds).cpu().numpy()
    var = (s2 / seeds).cpu().numpy() - mean ** 2
    sigma = math.sqrt(fro2 / b)
    assert np.max(np.abs(mean - AB)) < 6.0 * sigma / math.sqrt(seeds)
    avg_var = float(var.mean())
    expected = (fro2 - float((AB ** 2).mean())) / b
    assert avg_var <= 1.08 * fro2 / b
    assert avg_var >= 0.85 * expected
    h.free()
