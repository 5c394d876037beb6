"""GPU parity of the Sec. 5.2 estimator: the AMS sketches X_t of AB under
4-wise independent signs (FP64 sums; equal to the oracle's to 1e-9 of the
sum of |terms|) and the bound 32 median X_t^2."""
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


@pytest.mark.parametrize("n1,n2,n3,d,dtype,alias", [
    (2048, 512, 2048, 9, torch.float32, True),
    (700, 333, 500, 5, torch.float32, False),
    (1024, 128, 1024, 4, torch.bfloat16, True),
    (300, 77, 450, 3, torch.float64, False),
    (64, 1, 64, 1, torch.float32, True),
])
def test_frobenius_estimate_matches_oracle(cms, n1, n2, n3, d, dtype, alias):
    seed = 1000 + n1 + d
    if alias:
        X = W.gaussian(n2, n1, seed).astype(np.float32)
        Xr = W.bf16_round(X)[0] if dtype == torch.bfloat16 else X
        xt = torch.from_numpy(X).to(dev(), dtype)
        A, B = xt.T, xt
        Ad, Bd = Xr.T.astype(np.float64), Xr.astype(np.float64)
    else:
        Ah = W.gaussian(n1, n2, seed).astype(np.float32)
        Bh = W.gaussian(n2, n3, seed + 1).astype(np.float32)
        A = torch.from_numpy(np.ascontiguousarray(Ah.T)).to(dev(), dtype).T
        B = torch.from_numpy(Bh).to(dev(), dtype)
        Ad, Bd = Ah.astype(np.float64), Bh.astype(np.float64)
    est, bound = cms.frobenius_estimate(A, B, seed, d)
    cms.check_async()
    want = O.ams_frobenius(Ad, Bd, seed, d)
    scale = np.abs(Ad).sum(axis=0) @ np.abs(Bd).sum(axis=1)      # sum_k |a_k|_1 |b_k|_1
    np.testing.assert_allclose(est.cpu().numpy(), want, rtol=0, atol=1e-9 * scale)
    assert abs(bound - O.frobenius_bound(want)) <= 1e-9 * 32 * scale ** 2
    if d >= 5:
        assert bound >= np.sum((Ad @ Bd) ** 2)


def to_dev(sb: W.SparseBlocks):
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev(), dt)   # noqa: E731
    return (t(sb.a_colptr, torch.int64), t(sb.a_rowidx, torch.int32), t(sb.a_val, torch.float32),
            t(sb.b_rowptr, torch.int64), t(sb.b_colidx, torch.int32), t(sb.b_val, torch.float32))


@pytest.mark.parametrize("blocks,d", [(16, 3), (64, 5), (3, 1)])
def test_nnz_doubling_matches_oracle(cms, blocks, d):
    n = 1 << 16
    sb = W.sparse_blocks(n, n_blocks=blocks, inner=8, rows=32, cols=32, seed=blocks + 7)
    A, B = sb.scipy()
    AB = (A @ B).tocoo()
    AB.eliminate_zeros()
    seed = 500 + blocks
    got = cms.nnz_estimate(*to_dev(sb), n, n, seed, d, 1 << 22)
    want = O.nnz_doubling(AB.row, AB.col, seed, d, 1 << 22)
    assert got == want
    assert got[0] >= AB.nnz or d < 3


def test_nnz_doubling_sees_cancellation(cms):
    # two inner indices with the same column of A and opposite rows of B: the
    # block's product cancels exactly and its entries are zero; the search
    # counts only the entries that remain
    import scipy.sparse as sp
    n, n2 = 4096, 6
    g = W.rng(120)
    A = np.zeros((n, n2))
    B = np.zeros((n2, n))
    r = g.choice(n, 40, replace=False)
    cl = g.choice(n, 40, replace=False)
    A[r, 0] = g.integers(1, 9, 40)
    A[r, 1] = A[r, 0]
    B[0, cl] = g.integers(1, 9, 40)
    B[1, cl] = -B[0, cl]
    r2 = g.choice(n, 10, replace=False)
    c2 = g.choice(n, 12, replace=False)
    A[r2, 4] = g.integers(1, 9, 10)
    B[4, c2] = g.integers(1, 9, 12)
    Ac = sp.csc_matrix(A.astype(np.float32))
    Br = sp.csr_matrix(B.astype(np.float32))
    AB = (sp.csc_matrix(A) @ sp.csr_matrix(B)).tocoo()
    AB.eliminate_zeros()
    assert AB.nnz == 120
    T = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev(), dt)   # noqa: E731
    args = (T(Ac.indptr, torch.int64), T(Ac.indices, torch.int32), T(Ac.data, torch.float32),
            T(Br.indptr, torch.int64), T(Br.indices, torch.int32), T(Br.data, torch.float32))
    got = cms.nnz_estimate(*args, n, n, 77, 5, 1 << 16)
    assert got == O.nnz_doubling(AB.row, AB.col, 77, 5, 1 << 16)
