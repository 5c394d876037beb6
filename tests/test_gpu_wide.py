"""GPU parity of the cluster kernel for long sketches against the FP64 oracle.

When b is a multiple of 2^16 the row length of the b = R x C split is
C = 2^16 and each row is computed by a cluster of 8 CTAs (k_sketch_wide):
bucket records dealt to threads in tensor memory, a local length-8192 FFT
per CTA, the length-8 DFT across the cluster through distributed shared
memory, Kahan accumulators in tensor memory, and a two-pass inverse of the
length-2^16 rows.  Tolerance: relative L2 1e-5 per repetition (FP32 data;
BF16 storage against the BF16 values themselves).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cms_oracle as O

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


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


def run(cms, A, B, h):
    """Sketch through the C ABI; returns c (host) and the launched kernels."""
    cms.profile_enable(True)
    c = cms.sketch_product(A, B, h)
    torch.cuda.synchronize()
    kernels = cms.profile_summary()
    cms.profile_enable(False)
    cms.check_async()
    return c.cpu().numpy().astype(np.float64), kernels


def per_rep_err(c, ref):
    return max(O.rel_l2(c[t], ref[t]) for t in range(ref.shape[0]))


@pytest.mark.parametrize("n1,n2,n3,b,d,bf16,alias", [
    (2048, 40, 2048, 1 << 18, 3, False, True),    # R = 4: rows f1 = 0..2
    (1200, 33, 1000, 5 << 16, 2, False, False),   # R = 5 (odd), two operands
    (4096, 24, 4096, 3 << 18, 2, True, True),     # R = 12, BF16 storage
    (2048, 19, 4096, 1 << 18, 3, True, False),    # BF16, two operands, n1 != n3
    (1024, 1, 1024, 1 << 18, 1, False, True),     # a single inner index
])
def test_wide_kernel_matches_oracle(cms, n1, n2, n3, b, d, bf16, alias):
    n = max(n1, n3)
    seed = 31 + n1 + n2
    h = cms.make_hashes(seed, n, b, d)
    tab = O.make_tables(seed, n, b, d)
    dt = torch.bfloat16 if bf16 else torch.float32
    if alias:
        X = W.gaussian(n2, n1, seed).astype(np.float32)
        Xr = W.bf16_round(X)[0] if bf16 else X
        xt = torch.from_numpy(X).to(dev(), dt)
        c, kernels = run(cms, xt.T, xt, h)
        ref = O.sketch_definition(Xr.T.astype(np.float64), Xr.astype(np.float64), tab)
    else:
        A = W.gaussian(n1, n2, seed).astype(np.float32)
        B = W.gaussian(n2, n3, seed + 1).astype(np.float32)
        Ar = W.bf16_round(A)[0] if bf16 else A
        Br = W.bf16_round(B)[0] if bf16 else B
        at = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev(), dt).T
        bt = torch.from_numpy(B).to(dev(), dt)
        c, kernels = run(cms, at, bt, h)
        ref = O.sketch_definition(Ar.astype(np.float64), Br.astype(np.float64), tab)
    assert "k_sketch_wide" in kernels and "k_winv_a" in kernels
    assert per_rep_err(c, ref) < TOL_F32
    h.free()


def test_wide_kernel_spill_list(cms):
    # every side-1 bucket of these tables has (h mod 2^16) mod 8 = 0, so one
    # CTA of each cluster holds about n + n / 8 entries, beyond the records
    # its tensor memory keeps: the rest runs through the spill list
    n, m, b, d = 16384, 12, 1 << 18, 2
    rng = W.rng(77)
    h1 = 8 * rng.integers(0, b // 8, size=(d, n))
    s1 = rng.choice(np.array([-1, 1]), size=(d, n))
    h2 = rng.integers(0, b, size=(d, n))
    s2 = rng.choice(np.array([-1, 1]), size=(d, n))
    h = cms.Hashes.from_tables(h1.astype(np.uint32), s1.astype(np.int8), h2.astype(np.uint32),
                               s2.astype(np.int8), b)
    tab = O.Tables(h1, s1, h2, s2, b)
    X = W.gaussian(m, n, 78).astype(np.float32)
    xt = torch.from_numpy(X).to(dev())
    c, kernels = run(cms, xt.T, xt, h)
    assert "k_sketch_wide" in kernels
    Xd = X.astype(np.float64)
    zs = W.rng(79).choice(b, 48, replace=False)
    for t in range(d):
        want = O.sketch_bucket_values(Xd.T, Xd, tab, t, zs)
        assert np.linalg.norm(c[t, zs] - want) / np.linalg.norm(want) < TOL_F32, t
        dc = (tab.s1[t] @ Xd.T) @ (Xd @ tab.s2[t])
        assert abs(c[t].sum() - dc) < 1e-5 * np.abs(c[t]).sum()
    h.free()


def test_large_covariance_shape_runs_the_cluster_kernel(cms):
    # the large covariance configuration's shape (n = 32768 BF16 variables,
    # b = 2^20, d = 7) with 16 samples: the cluster kernel, checked on
    # sampled buckets and the DC identity
    m, n, b, d = 16, 32768, 1 << 20, 7
    cov = W.covariance(m, n, 64, 0.3, seed=5, dtype=np.float32)
    Xb, _ = W.bf16_round(cov.X)
    X = torch.from_numpy(cov.X).to(dev(), torch.bfloat16)
    h = cms.make_hashes(5, n, b, d)
    c, kernels = run(cms, X.T, X, h)
    assert "k_sketch_wide" in kernels
    tab = O.make_tables(5, n, b, d)
    Xd = Xb.astype(np.float64)
    zs = W.rng(56).choice(b, 48, replace=False)
    for t in range(d):
        want = O.sketch_bucket_values(Xd.T, Xd, tab, t, zs)
        assert np.linalg.norm(c[t, zs] - want) / np.linalg.norm(want) < TOL_F32, t
        dc = (tab.s1[t] @ Xd.T) @ (Xd @ tab.s2[t])
        assert abs(c[t].sum() - dc) < 1e-5 * np.abs(c[t]).sum()
    h.free()
