"""CPU checks of the seeded input generators (the input recipe the tests and
the benchmark share): planted covariance pairs, block-sparse operands for
the exact-recovery regime (Theorem 5), 5-smooth batch sizes, bfloat16
rounding and reproducibility of every stream."""
import math

import numpy as np
import torch

import workloads as W


def test_streams_are_reproducible():
    a = W.gaussian(64, 32, 7)
    np.testing.assert_array_equal(a, W.gaussian(64, 32, 7))
    assert not np.array_equal(a, W.gaussian(64, 32, 8))
    np.testing.assert_array_equal(W.sample_pairs(10, 20, 50, 3), W.sample_pairs(10, 20, 50, 3))


def test_covariance_pairs_are_disjoint_and_correlated():
    m, n, k, rho = 20000, 64, 8, 0.5
    cov = W.covariance(m, n, k, rho, seed=11, dtype=np.float64, chunk_rows=4096)
    assert cov.X.shape == (m, n) and cov.pairs.shape == (k, 2)
    flat = cov.pairs.reshape(-1)
    assert len(set(flat.tolist())) == 2 * k                    # disjoint pairs, u != v
    X = cov.X
    for u, v in cov.pairs:
        r = np.corrcoef(X[:, u], X[:, v])[0, 1]
        assert abs(r - rho) < 0.05, (u, v, r)                   # sampling error ~ 1/sqrt(m)
    others = [c for c in range(n) if c not in set(flat.tolist())]
    r0 = np.corrcoef(X[:, others[0]], X[:, others[1]])[0, 1]
    assert abs(r0) < 0.05
    # unit variance for planted and free columns alike
    assert np.all(np.abs(X.var(axis=0) - 1.0) < 0.05)


def test_sparse_blocks_have_disjoint_supports_and_exact_integer_product():
    sb = W.sparse_blocks(256, n_blocks=6, inner=3, rows=5, cols=4, seed=2)
    A, B = sb.scipy()
    ks = np.concatenate([blk[0] for blk in sb.blocks])
    rs = np.concatenate([blk[1] for blk in sb.blocks])
    cs = np.concatenate([blk[2] for blk in sb.blocks])
    assert len(set(ks.tolist())) == len(ks)
    assert len(set(rs.tolist())) == len(rs)
    assert len(set(cs.tolist())) == len(cs)
    vals = np.concatenate([sb.a_val, sb.b_val])
    assert np.all(vals != 0) and np.all(np.abs(vals) <= 8) and np.all(vals == np.round(vals))
    C = (A @ B).toarray()
    assert np.count_nonzero(C) <= 6 * 5 * 4
    np.testing.assert_array_equal(C, np.round(C))               # integer product
    # the product lives on the blocks' rows x columns only
    mask = np.zeros_like(C, dtype=bool)
    for k_, r_, c_ in sb.blocks:
        mask[np.ix_(r_, c_)] = True
    assert not np.any(C[~mask])


def _is_5_smooth(v: int) -> bool:
    for p in (2, 3, 5):
        while v % p == 0:
            v //= p
    return v == 1


def test_five_smooth_near_and_batch_specs():
    for x in (1.0, 7.0, 511.3, 700.0, 1000.0, 4095.0, 8192.0):
        v = W.five_smooth_near(x)
        assert _is_5_smooth(v)
        # no 5-smooth integer lies closer in log scale (brute force)
        cands = [c for c in range(1, 4 * int(x) + 2) if _is_5_smooth(c)]
        best = min(cands, key=lambda c: abs(math.log(c) - math.log(x)))
        assert abs(math.log(v) - math.log(x)) <= abs(math.log(best) - math.log(x)) + 1e-12
    specs = W.batched_specs(64, 4)
    assert len(specs) == 64
    assert [s.dtype for s in specs] == ["f32"] * 32 + ["bf16"] * 32
    for q, s in enumerate(specs):
        assert 512 <= s.n <= 8192 and _is_5_smooth(s.n) and _is_5_smooth(16 * s.n)
        assert s.m == 2 * s.n and s.n_pairs == s.n // 100 and s.seed == 4 + q


def test_bf16_round_matches_torch_round_to_nearest_even():
    g = np.random.default_rng(5)
    x = np.concatenate([g.standard_normal(10000).astype(np.float32) * 1e3,
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.4e38, 1e-40], np.float32)])
    got, bits = W.bf16_round(x)
    want = torch.from_numpy(x).to(torch.bfloat16)
    np.testing.assert_array_equal(got, want.float().numpy())
    np.testing.assert_array_equal(bits, want.view(torch.int16).numpy().view(np.uint16))
