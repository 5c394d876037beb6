"""GPU parity of the covariance post-steps (Sec. 3.2, Fig. 2) against the
FP64 oracle: the sketch with the diagonal's contribution removed (relative
L2 1e-5 per repetition) and the thresholded decode (the same pairs, in the
same row-major order, and the same FP32 estimates, when both sides decode
the oracle's sketch rounded to FP32)."""
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


def per_rep_err(c, ref):
    return max(O.rel_l2(c[t], ref[t]) for t in range(ref.shape[0]))


@pytest.mark.parametrize("n,m,b,d,dtype", [(1024, 300, 65536, 5, torch.float32),
                                           (1000, 200, 16000, 3, torch.float32),
                                           (768, 100, 12288, 4, torch.bfloat16)])
def test_remove_diagonal_matches_oracle(cms, n, m, b, d, dtype):
    cov = W.covariance(m, n, n // 100, 0.5, seed=n + d, dtype=np.float32)
    Xr = W.bf16_round(cov.X)[0] if dtype == torch.bfloat16 else cov.X
    X = torch.from_numpy(cov.X).to(dev(), dtype)
    h = cms.make_hashes(n + b, n, b, d)
    tab = O.make_tables(n + b, n, b, d)
    c = cms.sketch_product(X.T, X, h)
    cms.remove_diagonal(X.T, X, h, c)
    cms.check_async()
    Xd = Xr.astype(np.float64)
    ref = O.remove_diagonal(O.sketch_definition(Xd.T, Xd, tab), O.product_diagonal(Xd.T, Xd), tab)
    assert per_rep_err(c.cpu().numpy(), ref) < TOL_F32
    h.free()


def test_remove_diagonal_rectangular_operands(cms):
    n1, n2, n3, b, d = 700, 57, 500, 8192, 3
    A = W.gaussian(n1, n2, 81).astype(np.float32)
    B = W.gaussian(n2, n3, 82).astype(np.float32)
    h = cms.make_hashes(83, n1, b, d)
    tab = O.make_tables(83, n1, b, d)
    At = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev()).T
    Bt = torch.from_numpy(B).to(dev())
    c = cms.sketch_product(At, Bt, h)
    cms.remove_diagonal(At, Bt, h, c)
    ref = O.remove_diagonal(O.sketch_definition(A.astype(np.float64), B.astype(np.float64), tab),
                            O.product_diagonal(A, B), tab)
    assert per_rep_err(c.cpu().numpy(), ref) < TOL_F32
    h.free()


@pytest.mark.parametrize("d,skip", [(5, True), (4, True), (3, False)])
def test_decode_threshold_matches_oracle(cms, d, skip):
    # both sides decode the oracle's sketch (rounded to FP32)
    n, m, b = 600, 400, 32768
    cov = W.covariance(m, n, 6, 0.5, seed=90 + d, dtype=np.float32)
    Xd = cov.X.astype(np.float64)
    tab = O.make_tables(91 + d, n, b, d)
    c_ref = O.remove_diagonal(O.sketch_definition(Xd.T, Xd, tab), O.product_diagonal(Xd.T, Xd), tab)
    c32 = c_ref.astype(np.float32)
    h = cms.make_hashes(91 + d, n, b, d)
    tau = 0.5 * 0.5 * m
    ij, val, count = cms.decode_threshold(torch.from_numpy(c32).to(dev()), h, n, n, tau, skip_diagonal=skip,
                                          capacity=n * n)
    want = O.candidates(c32, tab, n, n, tau, skip_diagonal=skip)
    assert count == len(want) > 10
    np.testing.assert_array_equal(ij.cpu().numpy(), want)
    est = O.estimates(c32, tab, want[:, 0], want[:, 1]).astype(np.float32)
    est.sort(axis=0)
    mid = d // 2
    want_val = est[mid] if d % 2 else np.float32(0.5) * (est[mid - 1] + est[mid])
    np.testing.assert_array_equal(val.cpu().numpy(), want_val)
    # a buffer smaller than the hit count: the count stays exact, the
    # returned hits are the first ones in row-major order
    ij2, _, count2 = cms.decode_threshold(torch.from_numpy(c32).to(dev()), h, n, n, tau, skip_diagonal=skip,
                                          capacity=7)
    assert count2 == count
    np.testing.assert_array_equal(ij2.cpu().numpy(), want[:7])
    h.free()


def test_covariance_pipeline_recovers_planted_pairs(cms):
    # the covariance configuration (X 4096 x 2048 FP32, 32 pairs rho = 0.5,
    # b = 2^16, d = 5): sketch, remove the diagonal, threshold at rho m / 2
    m, n, b, d, rho = 4096, 2048, 65536, 5, 0.5
    cov = W.covariance(m, n, 32, rho, seed=2, dtype=np.float32)
    X = torch.from_numpy(cov.X).to(dev())
    h = cms.make_hashes(2, n, b, d)
    c = cms.sketch_product(X.T, X, h)
    cms.remove_diagonal(X.T, X, h, c)
    ij, val, count = cms.decode_threshold(c, h, n, n, 0.5 * rho * m, capacity=1 << 20)
    hits = set(map(tuple, ij.cpu().numpy().tolist()))
    planted = [(int(u), int(v)) for u, v in cov.pairs] + [(int(v), int(u)) for u, v in cov.pairs]
    recall = sum(p in hits for p in planted) / len(planted)
    assert recall >= 0.9, recall
    assert count < 0.002 * n * n, count
    h.free()
