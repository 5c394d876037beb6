"""GPU parity of the sparse-input path (A by columns, B by rows) against the
FP64 oracle: integer-valued block-sparse products (Theorem 5's setting) must
come out exact after rounding; real-valued inputs within relative L2 1e-5."""
import math

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


def to_dev(sb: W.SparseBlocks, dtype=torch.float32):
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev(), dt)   # noqa: E731
    return (t(sb.a_colptr, torch.int64), t(sb.a_rowidx, torch.int32), t(sb.a_val, dtype),
            t(sb.b_rowptr, torch.int64), t(sb.b_colidx, torch.int32), t(sb.b_val, dtype))


@pytest.mark.parametrize("n,blocks,b,d", [(1 << 16, 64, 1 << 16, 3), (5000, 10, 4096, 2), (3000, 4, 1024, 5)])
def test_sparse_blocks_exact(cms, n, blocks, b, d):
    sb = W.sparse_blocks(n, n_blocks=blocks, inner=8, rows=32, cols=32, seed=n + blocks)
    A, B = sb.scipy()
    h = cms.make_hashes(7 + b, n, b, d)
    c = cms.sketch_product_csr(*to_dev(sb), n, n, h).cpu().numpy()
    ref = O.sketch_definition_sparse(A, B, O.make_tables(7 + b, n, b, d))
    np.testing.assert_array_equal(np.rint(c), ref)
    assert O.rel_l2(c, ref) < 1e-5
    h.free()


def test_sparse_real_values_match_dense_path(cms):
    n, n2, b, d = 700, 300, 8192, 3
    g = W.rng(4)
    A = np.where(g.random((n, n2)) < 0.05, g.standard_normal((n, n2)), 0.0).astype(np.float32)
    B = np.where(g.random((n2, n)) < 0.05, g.standard_normal((n2, n)), 0.0).astype(np.float32)
    import scipy.sparse as sp
    Ac = sp.csc_matrix(A)
    Br = sp.csr_matrix(B)
    h = cms.make_hashes(5, n, b, d)
    T = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev(), dt)   # noqa: E731
    c_sp = cms.sketch_product_csr(T(Ac.indptr, torch.int64), T(Ac.indices, torch.int32),
                                  T(Ac.data, torch.float32), T(Br.indptr, torch.int64),
                                  T(Br.indices, torch.int32), T(Br.data, torch.float32), n, n, h)
    c_dn = cms.sketch_product(T(A.T, torch.float32).T, T(B, torch.float32), h)
    ref = O.sketch_definition(A.astype(np.float64), B.astype(np.float64), O.make_tables(5, n, b, d))
    assert O.rel_l2(c_sp.cpu().numpy(), ref) < 1e-5
    assert O.rel_l2(c_dn.cpu().numpy(), ref) < 1e-5
    h.free()


@pytest.mark.parametrize("K", [1, 2, 3, 5, 7, 9, 13])
def test_sparse_few_nonempty_inner_indices(cms, K):
    # K nonempty inner indices (a column of A and a row of B both nonzero)
    # among n2 = 500: partial groups of the FFT route's four inner indices,
    # the prefetch of the next two groups running past the list's end, and
    # chunks of the fixed launch left empty
    n, n2, b, d = 600, 500, 4096, 3
    g = W.rng(60 + K)
    ks = np.sort(g.choice(n2, size=K, replace=False))
    A = np.zeros((n, n2), np.float32)
    B = np.zeros((n2, n), np.float32)
    for k in ks:
        ra = g.choice(n, size=int(g.integers(1, 40)), replace=False)
        rb = g.choice(n, size=int(g.integers(1, 40)), replace=False)
        A[ra, k] = g.standard_normal(ra.size)
        B[k, rb] = g.standard_normal(rb.size)
    # inner indices with only one side nonzero add nothing and are skipped
    A[g.integers(0, n, 20), g.integers(0, n2, 20)] = 1.0
    import scipy.sparse as sp
    Ac = sp.csc_matrix(A)
    Br = sp.csr_matrix(B)
    h = cms.make_hashes(70 + K, n, b, d)
    T = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev(), dt)   # noqa: E731
    c = cms.sketch_product_csr(T(Ac.indptr, torch.int64), T(Ac.indices, torch.int32),
                               T(Ac.data, torch.float32), T(Br.indptr, torch.int64),
                               T(Br.indices, torch.int32), T(Br.data, torch.float32), n, n, h)
    ref = O.sketch_definition(A.astype(np.float64), B.astype(np.float64), O.make_tables(70 + K, n, b, d))
    assert O.rel_l2(c.cpu().numpy(), ref) < 1e-5
    h.free()


@pytest.mark.parametrize("density", [0.02, 0.08])
def test_sparse_scatter_buffers_in_place_and_separate(cms, monkeypatch, density):
    # the FFT route scatters into per-warp Y buffers kept zero between groups
    # (each lane clears its bucket after the FFT reads it; columns of more
    # than 32 nonzeros, common at density 0.08, clear the whole buffer), or,
    # when those do not fit (forced here by the library's debug switch),
    # into the FFT region zeroed every group: the same sketch bit for bit,
    # and the oracle's
    n, n2, b, d = 900, 200, 16384, 2
    g = W.rng(41)
    A = np.where(g.random((n, n2)) < density, g.standard_normal((n, n2)), 0.0).astype(np.float32)
    B = np.where(g.random((n2, n)) < density, g.standard_normal((n2, n)), 0.0).astype(np.float32)
    import scipy.sparse as sp
    Ac = sp.csc_matrix(A)
    Br = sp.csr_matrix(B)
    h = cms.make_hashes(42, n, b, d)
    T = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev(), dt)   # noqa: E731
    args = (T(Ac.indptr, torch.int64), T(Ac.indices, torch.int32), T(Ac.data, torch.float32),
            T(Br.indptr, torch.int64), T(Br.indices, torch.int32), T(Br.data, torch.float32), n, n, h)
    c_sep = cms.sketch_product_csr(*args)
    monkeypatch.setenv("CMS_SPARSE_INPLACE_Y", "1")
    c_inp = cms.sketch_product_csr(*args)
    monkeypatch.delenv("CMS_SPARSE_INPLACE_Y")
    cms.check_async()
    assert torch.equal(c_sep, c_inp)
    ref = O.sketch_definition(A.astype(np.float64), B.astype(np.float64), O.make_tables(42, n, b, d))
    assert O.rel_l2(c_sep.cpu().numpy(), ref) < 1e-5
    h.free()


def test_sparse_without_common_inner_index_is_zero(cms):
    n, b = 200, 2048
    colptr = np.zeros(11, np.int64)
    colptr[1:] = np.arange(1, 11)            # A: one nonzero in each column k = 0..9
    rowptr = np.zeros(11, np.int64)          # B: all rows empty
    T = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev(), dt)   # noqa: E731
    h = cms.make_hashes(1, n, b, 2)
    c = cms.sketch_product_csr(T(colptr, torch.int64), T(np.arange(10), torch.int32),
                               T(np.ones(10), torch.float32), T(rowptr, torch.int64),
                               T(np.zeros(1), torch.int32), T(np.zeros(1), torch.float32), n, n, h)
    assert torch.count_nonzero(c).item() == 0
    h.free()


def test_sparse_bf16_values_exact(cms):
    n, b, d = 4096, 4096, 3
    sb = W.sparse_blocks(n, n_blocks=16, inner=4, rows=16, cols=16, seed=12)
    A, B = sb.scipy()
    h = cms.make_hashes(3, n, b, d)
    c = cms.sketch_product_csr(*to_dev(sb, torch.bfloat16), n, n, h).cpu().numpy()
    ref = O.sketch_definition_sparse(A, B, O.make_tables(3, n, b, d))
    np.testing.assert_array_equal(np.rint(c), ref)   # small integers are exact in BF16
    h.free()


def test_exact_sparse_full_size(cms):
    # n = 2^20; 256 disjoint blocks of 8 inner indices x 32 rows of A x 32
    # columns of B, integer values in [-8, 8] \ {0}; b = 2^20, d = 3.
    n, b, d = 1 << 20, 1 << 20, 3
    sb = W.sparse_blocks(n, n_blocks=256, inner=8, rows=32, cols=32, seed=3)
    A, B = sb.scipy()
    h = cms.make_hashes(3, n, b, d)
    c = cms.sketch_product_csr(*to_dev(sb), n, n, h)
    tab = O.make_tables(3, n, b, d)
    ref = O.sketch_definition_sparse(A, B, tab)
    np.testing.assert_array_equal(np.rint(c.cpu().numpy()), ref)      # c bit-exact after rounding
    # decode at every nonzero of AB and at as many random positions: the GPU's
    # medians equal the oracle's medians exactly (both decode integer sketches)
    AB = (A @ B).tocoo()
    g = W.rng(33)
    zi = g.integers(0, n, AB.nnz)
    zj = g.integers(0, n, AB.nnz)
    ii = np.concatenate([AB.row, zi]).astype(np.int64)
    jj = np.concatenate([AB.col, zj]).astype(np.int64)
    ij = torch.from_numpy(np.stack([ii, jj], 1)).to(dev())
    est = cms.decode(c, h, ij).cpu().numpy()
    want = O.decompress(ref, tab, ii, jj)
    np.testing.assert_array_equal(np.rint(est), want)
    # how often the median equals AB (Theorem 5 regime needs d >= 6 lg n; d = 3 here)
    exact = np.mean(np.rint(est[:AB.nnz]) == AB.data)
    assert exact > 0.8
    h.free()


# ------------------------------------------------------ sparse-k hybrid ----
def run_hybrid(cms, args, n1, n3, h, limit):
    cms.profile_enable(True)
    c = cms.sketch_product_csr(*args, n1, n3, h, direct_max_pairs=limit)
    torch.cuda.synchronize()
    kernels = cms.profile_summary()
    cms.profile_enable(False)
    cms.check_async()
    return c.cpu().numpy(), kernels


@pytest.mark.parametrize("limit", [-1, 0, 1024, 1 << 40])
def test_hybrid_blocks_exact(cms, limit):
    # integer blocks: every outer product has 32 x 32 = 1024 terms, so the
    # default split and limit >= 1024 sketch them all directly, 0 none
    n, b, d = 1 << 16, 1 << 16, 3
    sb = W.sparse_blocks(n, n_blocks=64, inner=8, rows=32, cols=32, seed=n + 64)
    A, B = sb.scipy()
    h = cms.make_hashes(7 + b, n, b, d)
    c, kernels = run_hybrid(cms, to_dev(sb), n, n, h, limit)
    ref = O.sketch_definition_sparse(A, B, O.make_tables(7 + b, n, b, d))
    np.testing.assert_array_equal(np.rint(c), ref)
    assert O.rel_l2(c, ref) < 1e-5
    # the split is made on the device (the call never waits for it): both
    # routes' kernels launch, and the one whose list is empty returns at once
    assert kernels["k_sketch_sparse"]["launches"] == 1
    assert kernels["k_direct_scatter"]["launches"] == 1
    h.free()


def test_hybrid_mixed_split_real_values(cms):
    # columns of A / rows of B with very different nonzero counts: the split
    # sends the small outer products to the direct route, the large ones to
    # the FFT route; their sum matches the oracle
    n, n2, b, d = 900, 240, 8192, 3
    g = W.rng(41)
    dens = np.where(np.arange(n2) % 3 == 0, 0.2, 0.01)
    A = np.where(g.random((n, n2)) < dens[None, :], g.standard_normal((n, n2)), 0.0).astype(np.float32)
    B = np.where(g.random((n2, n)) < dens[:, None], g.standard_normal((n2, n)), 0.0).astype(np.float32)
    import scipy.sparse as sp
    Ac = sp.csc_matrix(A)
    Br = sp.csr_matrix(B)
    pairs = np.diff(Ac.indptr) * np.diff(Br.indptr)
    limit = int(np.median(pairs[pairs > 0]))
    assert (pairs > limit).sum() > 10 and ((pairs > 0) & (pairs <= limit)).sum() > 10
    T = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev(), dt)   # noqa: E731
    args = (T(Ac.indptr, torch.int64), T(Ac.indices, torch.int32), T(Ac.data, torch.float32),
            T(Br.indptr, torch.int64), T(Br.indices, torch.int32), T(Br.data, torch.float32))
    h = cms.make_hashes(9, n, b, d)
    c, kernels = run_hybrid(cms, args, n, n, h, limit)
    assert "k_sketch_sparse" in kernels and "k_direct_scatter" in kernels
    ref = O.sketch_definition(A.astype(np.float64), B.astype(np.float64), O.make_tables(9, n, b, d))
    assert max(O.rel_l2(c[t], ref[t]) for t in range(d)) < 1e-5
    h.free()


def test_hybrid_without_common_inner_index_is_zero(cms):
    n, b = 200, 2048
    colptr = np.zeros(11, np.int64)
    colptr[1:] = np.arange(1, 11)
    rowptr = np.zeros(11, np.int64)
    T = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev(), dt)   # noqa: E731
    h = cms.make_hashes(1, n, b, 2)
    c = torch.full((2, b), 7.0, device=dev())
    cms.sketch_product_csr(T(colptr, torch.int64), T(np.arange(10), torch.int32),
                           T(np.ones(10), torch.float32), T(rowptr, torch.int64),
                           T(np.zeros(1), torch.int32), T(np.zeros(1), torch.float32), n, n, h, c=c,
                           direct_max_pairs=-1)
    assert torch.count_nonzero(c).item() == 0
    h.free()


def test_hybrid_exact_sparse_full_size(cms):
    # the exact sparse configuration (n = b = 2^20, d = 3) through the direct
    # route: c bit-exact after rounding, as on the FFT route
    n, b, d = 1 << 20, 1 << 20, 3
    sb = W.sparse_blocks(n, n_blocks=256, inner=8, rows=32, cols=32, seed=3)
    A, B = sb.scipy()
    h = cms.make_hashes(3, n, b, d)
    c, kernels = run_hybrid(cms, to_dev(sb), n, n, h, -1)
    # every inner index goes direct: the FFT route's blocks return at once
    # (its full run on this configuration takes about 18 ms)
    assert kernels["k_sketch_sparse"]["ms"] < 1.0
    ref = O.sketch_definition_sparse(A, B, O.make_tables(3, n, b, d))
    np.testing.assert_array_equal(np.rint(c), ref)
    h.free()


@pytest.mark.parametrize("hybrid", [False, True])
def test_sparse_calls_return_without_waiting_and_capture_in_a_graph(cms, hybrid):
    # the nonempty-inner-index count stays on the device: the call returns
    # while the stream is still busy with earlier work, and the whole call can
    # be captured in a CUDA graph whose replay gives the same (exact) sketch
    n, b, d = 5000, 4096, 2
    sb = W.sparse_blocks(n, n_blocks=10, inner=8, rows=32, cols=32, seed=77)
    A, B = sb.scipy()
    args = to_dev(sb)
    h = cms.make_hashes(9, n, b, d)
    ref = O.sketch_definition_sparse(A, B, O.make_tables(9, n, b, d))
    ws = cms.alloc_workspace(cms.sparse_workspace_size(h, n, A.shape[1], n), dev())
    c = torch.zeros((d, b), dtype=torch.float32, device=dev())
    dmp = -1 if hybrid else None
    s = torch.cuda.Stream(device=dev())
    with torch.cuda.stream(s):
        cms.sketch_product_csr(*args, n, n, h, c=c, ws=ws, stream=s, direct_max_pairs=dmp)   # warm
        torch.cuda._sleep(200_000_000)                 # ~0.1 s of GPU time ahead of the call
        cms.sketch_product_csr(*args, n, n, h, c=c, ws=ws, stream=s, direct_max_pairs=dmp)
        busy = not s.query()
    s.synchronize()
    assert busy, "the sparse call waited for the stream"
    np.testing.assert_array_equal(np.rint(c.cpu().numpy()), ref)
    c.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        cms.sketch_product_csr(*args, n, n, h, c=c, ws=ws, stream=s, direct_max_pairs=dmp)
    for _ in range(2):
        c.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(np.rint(c.cpu().numpy()), ref)
    cms.check_async()
    h.free()


def test_hybrid_with_every_inner_index_direct_or_none(cms):
    # the FFT route's list empty (everything direct: its kernels return at
    # once) and the direct list empty (everything on the FFT route)
    n, b, d = 3000, 2048, 3
    sb = W.sparse_blocks(n, n_blocks=4, inner=8, rows=32, cols=32, seed=5)
    A, B = sb.scipy()
    h = cms.make_hashes(3, n, b, d)
    ref = O.sketch_definition_sparse(A, B, O.make_tables(3, n, b, d))
    for limit in (1 << 40, 0):
        c = cms.sketch_product_csr(*to_dev(sb), n, n, h, direct_max_pairs=limit)
        np.testing.assert_array_equal(np.rint(c.cpu().numpy()), ref)
    h.free()
