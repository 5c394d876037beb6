"""Batched products (many uneven (A, B) pairs in one persistent launch) and
their CUDA-graph replay, against the FP64 oracle instance by instance."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cms_oracle as O

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


def dev():
    return torch.device("cuda", torch.cuda.current_device())


def make_instances(cms, specs, d=3):
    """Covariance-shaped instances: X (m x n), A = X^T, B = X, b = 16 n."""
    items, refs = [], []
    for q, sp in enumerate(specs):
        cov = W.covariance(sp.m, sp.n, sp.n_pairs, sp.rho, sp.seed, dtype=np.float32)
        if sp.dtype == "bf16":
            xr, _ = W.bf16_round(cov.X)
            X = torch.from_numpy(cov.X).to(dev(), torch.bfloat16)
        elif sp.dtype == "f64":
            xr = cov.X
            X = torch.from_numpy(cov.X).to(dev(), torch.float64)
        else:
            xr = cov.X
            X = torch.from_numpy(cov.X).to(dev())
        b = 16 * sp.n
        h = cms.make_hashes(100 + q, sp.n, b, d)
        items.append((X.T, X, h))
        refs.append((xr.astype(np.float64), O.make_tables(100 + q, sp.n, b, d)))
    return items, refs


def specs_small(count=8, seed=4):
    out = W.batched_specs(count, seed, n_lo=256, n_hi=1600)
    return out


def check(c, ref, tol=1e-5):
    Xd, tab = ref
    want = O.sketch_definition(Xd.T, Xd, tab)
    assert O.rel_l2(c.cpu().numpy(), want) < tol


def test_batch_matches_oracle_and_graph_replays(cms):
    specs = specs_small()
    items, refs = make_instances(cms, specs)
    batch = cms.Batch(items)
    info = batch.info()
    assert info["instances"] == len(specs) and info["tasks"] > 0
    cs = [c.clone() for c in batch.run()]
    torch.cuda.synchronize()
    cms.check_async()
    for c, ref in zip(cs, refs):
        check(c, ref)
    s = torch.cuda.Stream()
    for _ in range(2):
        batch.run_graph(s)
        s.synchronize()
        for c0, c1 in zip(cs, batch.c):
            assert torch.equal(c0, c1)          # deterministic whatever block ran which task
    batch.free()


def test_batch_graph_follows_reseeded_hashes(cms):
    specs = specs_small(4, seed=9)
    items, refs = make_instances(cms, specs)
    batch = cms.Batch(items)
    s = torch.cuda.Stream()
    batch.run_graph(s)
    s.synchronize()
    for q, (_, _, h) in enumerate(items):
        h.reseed(500 + q, stream=s)
    batch.run_graph(s)
    s.synchronize()
    for q, (c, (Xd, tab)) in enumerate(zip(batch.c, refs)):
        sp = specs[q]
        check(c, (Xd, O.make_tables(500 + q, sp.n, 16 * sp.n, 3)))
    batch.free()


def test_batch_autotune_writes_cache(cms, tmp_path):
    specs = specs_small(3, seed=11)
    items, refs = make_instances(cms, specs)
    cache = tmp_path / "tune.txt"
    batch = cms.Batch(items, autotune=True, tune_cache=str(cache))
    batch.run()
    torch.cuda.synchronize()
    for c, ref in zip(batch.c, refs):
        check(c, ref)
    lines = cache.read_text().strip().splitlines()
    assert len(lines) >= 1 and all("b=" in ln and "kernel=" in ln for ln in lines)
    batch.free()
    # a second batch reads the tuned choices back
    batch2 = cms.Batch(items, autotune=True, tune_cache=str(cache))
    batch2.run()
    torch.cuda.synchronize()
    for c, ref in zip(batch2.c, refs):
        check(c, ref)
    assert cache.read_text().strip().splitlines() == lines
    batch2.free()


def test_batch_mixes_kernel_kinds(cms):
    # FP32 and BF16 storage on the register-FFT body (odd n: rows copied as
    # their 16-byte aligned supersets, C = P Q), FP64 storage on the
    # generic body; all in one launch
    class Sp:
        def __init__(self, n, dtype, seed):
            self.n, self.m, self.dtype, self.seed, self.n_pairs, self.rho = n, 2 * n, dtype, seed, n // 100, 0.5
    specs = [Sp(512, "f32", 1), Sp(1000, "f32", 2), Sp(768, "bf16", 3), Sp(640, "f32", 4), Sp(675, "f32", 5),
             Sp(625, "bf16", 6), Sp(600, "f64", 7)]
    items, refs = make_instances(cms, specs)
    batch = cms.Batch(items)
    assert batch.info()["fast_instances"] == 6
    batch.run()
    torch.cuda.synchronize()
    for c, ref in zip(batch.c, refs):
        check(c, ref)
    batch.free()


def test_batch_c_32l_instances_run_the_fast_body(cms):
    # b = 16 n with n even: C = 32 L (L = 30, 27, 25, 24, 32), every FP32
    # instance on the register-FFT body, X^T X against the oracle
    class Sp:
        def __init__(self, n, seed):
            self.n, self.m, self.dtype, self.seed, self.n_pairs, self.rho = n, 2 * n, "f32", seed, n // 100, 0.5
    specs = [Sp(600, 1), Sp(648, 2), Sp(1000, 3), Sp(576, 4), Sp(1024, 5), Sp(864, 6)]
    items, refs = make_instances(cms, specs)
    batch = cms.Batch(items)
    assert batch.info()["fast_instances"] == len(specs)
    batch.run()
    torch.cuda.synchronize()
    for c, ref in zip(batch.c, refs):
        check(c, ref)
    batch.free()


def test_batch_large_instances_keep_records_in_tensor_memory(cms):
    # n up to 7776 (the configuration's upper range): the two-row twiddle
    # records no longer fit in shared memory and go to tensor memory; every
    # instance still runs the register-FFT body; checked on sampled buckets
    class Sp:
        def __init__(self, n, dtype, seed):
            self.n, self.m, self.dtype, self.seed, self.n_pairs, self.rho = n, 48, dtype, seed, n // 100, 0.5
    specs = [Sp(7776, "f32", 1), Sp(6912, "bf16", 2), Sp(1000, "f32", 3), Sp(5760, "f32", 4)]
    items, refs = make_instances(cms, specs)
    batch = cms.Batch(items)
    assert batch.info()["fast_instances"] == len(specs)
    batch.run()
    torch.cuda.synchronize()
    cms.check_async()
    for q, (Xd, tab) in enumerate(refs):
        c = batch.c[q].cpu().numpy().astype(np.float64)
        zs = W.rng(70 + q).choice(tab.b, 32, replace=False)
        for t in range(tab.d):
            want = O.sketch_bucket_values(Xd.T, Xd, tab, t, zs)
            assert np.linalg.norm(c[t, zs] - want) / np.linalg.norm(want) < 1e-5, (q, t)
    batch.free()
    for _, _, h in items:
        h.free()


def test_batch_inverse_is_two_launches_for_all_instances(cms):
    # the reduction and inverse of every instance run as one row launch and
    # one column launch (not two per instance), with the oracle's results
    specs = specs_small(count=6, seed=9)
    items, refs = make_instances(cms, specs)
    batch = cms.Batch(items)
    info = batch.info()
    cms.profile_enable(True)
    batch.run()
    torch.cuda.synchronize()
    kernels = cms.profile_summary()
    cms.profile_enable(False)
    cms.check_async()
    assert kernels["k_rows_inverse_batched"]["launches"] == 1
    assert kernels["k_cols_inverse_batched"]["launches"] == 1
    assert "k_rows_inverse" not in kernels and "k_cols_inverse" not in kernels
    fast = info["fast_instances"]
    assert info["launches"] == 4 + (len(specs) - fast)
    for c, ref in zip(batch.c, refs):
        check(c, ref)
    batch.free()
