"""GPU parity at the full sizes of the large covariance and the batched
configurations, in the launch configuration the bench times, on sampled
outputs the oracle computes one by one (c_t[z] for sampled buckets z straight
from the definition of Sec. 2.2) on every repetition, plus the DC-bin identity
sum_z c_t[z] = (s1^T A)(B s2) (Sec. 2.1, the AMS sketch) formed in float64.
Tolerance: relative L2 1e-5 per repetition (BF16 storage against the BF16
values themselves); the DC bin within 1e-5 of sum_z |c_t[z]|."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cms_oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def cms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_1320_gb300 import build as b
    b.build()
    import paper_1108_1320_gb300 as m
    m.lib()
    return m


def dev():
    return torch.device("cuda", torch.cuda.current_device())


def test_large_covariance_full_size(cms):
    # X 16384 x 32768 stored as BF16, 4096 planted pairs rho = 0.3, A = X^T,
    # B = X, b = 2^20, d = 7: the cluster kernel
    m, n, b, d = 16384, 32768, 1 << 20, 7
    cov = W.covariance(m, n, 4096, 0.3, seed=5, dtype=np.float32)
    X = torch.from_numpy(cov.X).to(dev(), torch.bfloat16)
    Xb = X.float().cpu().numpy()          # the stored BF16 values, exactly
    del cov
    h = cms.make_hashes(5, n, b, d)
    assert cms.plan_kernel(X.T, X, h) == "cluster"
    c = cms.sketch_product(X.T, X, h).cpu().numpy().astype(np.float64)
    cms.check_async()
    tab = O.make_tables(5, n, b, d)
    XT = np.ascontiguousarray(Xb.T)       # rows of A = X^T and columns of B = X
    for t in range(d):
        zs = W.rng(57 + t).choice(b, 64, replace=False)
        want = O.sketch_bucket_values_rows(XT, XT, tab, t, zs)
        assert np.linalg.norm(c[t, zs] - want) / np.linalg.norm(want) < TOL, t
        # (s1^T A)_k = sum_i s1(i) X_ki and (B s2)_k = sum_j s2(j) X_kj, in float64
        s1 = tab.s1[t].astype(np.float64)
        s2 = tab.s2[t].astype(np.float64)
        u = np.concatenate([Xb[r:r + 1024].astype(np.float64) @ s1 for r in range(0, m, 1024)])
        v = np.concatenate([Xb[r:r + 1024].astype(np.float64) @ s2 for r in range(0, m, 1024)])
        dc = float(np.dot(u, v))
        assert abs(c[t].sum() - dc) < TOL * np.abs(c[t]).sum(), t
    h.free()


def test_batched_full_range(cms):
    # 64 covariance instances, n log-uniform in [512, 8192] (5-smooth),
    # m = 2 n, half FP32 / half BF16, b = 16 n, d = 3, one persistent launch
    specs = W.batched_specs(64, seed=4, n_lo=512, n_hi=8192)
    items, host = [], []
    for q, sp in enumerate(specs):
        cov = W.covariance(sp.m, sp.n, sp.n_pairs, sp.rho, sp.seed, dtype=np.float32)
        dt = torch.bfloat16 if sp.dtype == "bf16" else torch.float32
        X = torch.from_numpy(cov.X).to(dev(), dt)
        host.append(X.float().cpu().numpy() if dt == torch.bfloat16 else cov.X)
        h = cms.make_hashes(1000 + q, sp.n, 16 * sp.n, 3)
        items.append((X.T, X, h))
    batch = cms.Batch(items)
    assert batch.info()["fast_instances"] == 64
    batch.run()
    torch.cuda.synchronize()
    cms.check_async()
    for q, sp in enumerate(specs):
        c = batch.c[q].cpu().numpy().astype(np.float64)
        tab = O.make_tables(1000 + q, sp.n, 16 * sp.n, 3)
        XqT = np.ascontiguousarray(host[q].T)
        for t in range(3):
            zs = W.rng(200 + 3 * q + t).choice(16 * sp.n, 16, replace=False)
            want = O.sketch_bucket_values_rows(XqT, XqT, tab, t, zs)
            assert np.linalg.norm(c[t, zs] - want) / np.linalg.norm(want) < TOL, (q, t)
    batch.free()
    for _, _, h in items:
        h.free()
