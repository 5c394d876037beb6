"""GPU parity of FINDSIGNIFICANTENTRIES (Sec. 4, Fig. 3): the decode and vote
on the oracle's masked sketches (rounded to FP32) give exactly the oracle's
positions; end to end (2 l masked sketch products on the GPU) the planted
large entries of a product with a clear margin are found exactly."""
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


def planted(n1, n2, n3, seed, big):
    g = W.rng(seed)
    A = 0.01 * g.standard_normal((n1, n2))
    B = 0.01 * g.standard_normal((n2, n3))
    for q, (i, j) in enumerate(big):
        A[i, q] += 10.0
        B[q, j] += 10.0 + q
    return A.astype(np.float32), B.astype(np.float32)


@pytest.mark.parametrize("rho,b,d", [(1, 8192, 5), (3, 4096, 4), (2, 2048, 3)])
def test_decode_significant_matches_oracle(cms, rho, b, d):
    n1, n2, n3 = 60, 8, 50
    big = [(3, 5), (17, 30), (59, 0), (21, 21), (40, 49), (7, 7)]
    A, B = planted(n1, n2, n3, 140 + rho, big)
    tab = O.make_tables(141, max(n1, n3), b, d)
    P = O.masked_sketches(A, B, tab, rho).astype(np.float32)
    h = cms.make_hashes(141, max(n1, n3), b, d)
    delta = 50.0
    got, count = cms.decode_significant(torch.from_numpy(P).to(dev()), h, n1, n3, delta, rho)
    want = O.significant_from_sketches(P, n1, n3, delta, rho)
    assert count == len(want)
    np.testing.assert_array_equal(got.cpu().numpy(), want)
    h.free()


@pytest.mark.parametrize("rho", [1, 2])
def test_find_significant_end_to_end(cms, rho):
    n1, n2, n3, b, d = 300, 16, 280, 16384, 5
    big = [(3, 5), (117, 230), (299, 0), (21, 21), (150, 279), (8, 9), (200, 100)]
    A, B = planted(n1, n2, n3, 150 + rho, big)
    AB = A.astype(np.float64) @ B.astype(np.float64)
    delta = 50.0
    want = sorted((int(i), int(j)) for i, j in zip(*np.nonzero(np.abs(AB) > delta)))
    h = cms.make_hashes(151, max(n1, n3), b, d)
    At = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev()).T
    Bt = torch.from_numpy(B).to(dev())
    cms.profile_enable(True)
    got, count = cms.find_significant(At, Bt, h, delta, rho)
    kernels = cms.profile_summary()
    cms.profile_enable(False)
    cms.check_async()
    assert [tuple(p) for p in got.cpu().numpy().tolist()] == want
    L, ell = O.code_length(n1, n3, rho)
    assert kernels["k_mask_copy"]["launches"] == 2 * ell
    assert kernels["k_sig_decode"]["launches"] == 1
    h.free()


def test_find_significant_covariance_entries(cms):
    # X^T X of a covariance-shaped sample: the diagonal (about m) and the
    # planted pairs (about rho m) stand above the sketch's noise; with
    # rho = 3 copies per bit the decode corrects the bits that noise flips
    m, n, b, d, rho_c = 2000, 256, 1 << 16, 5, 3
    cov = W.covariance(m, n, 8, 0.8, seed=160, dtype=np.float32)
    X = torch.from_numpy(cov.X).to(dev())
    h = cms.make_hashes(161, n, b, d)
    got, count = cms.find_significant(X.T, X, h, 0.5 * 0.8 * m, rho_c)
    hits = set(map(tuple, got.cpu().numpy().tolist()))
    want = [(i, i) for i in range(n)] + [(int(u), int(v)) for u, v in cov.pairs] + \
        [(int(v), int(u)) for u, v in cov.pairs]
    recall = sum(p in hits for p in want) / len(want)
    assert recall >= 0.9, recall
    assert count <= len(want) + 20, count
    h.free()
