"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test names what fixes the expected value: a published generator output,
a hand-worked hash value, an independent computation route of the paper's
identities (Sec. 2.2), a special case that reduces to brute force, the AMS
identity of Sec. 2.1, or Theorems 2 and 5.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import cms_oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- seeding ---
def test_splitmix64_matches_published_outputs():
    g = _load("splitmix64_seed0.json")
    state = g["state"]
    for hx in g["outputs_hex"]:
        state, out = O.splitmix64(state)
        assert out == int(hx, 16)


def test_coefficients_in_range_and_ordered():
    coef = O.draw_coefficients(12345, 7)
    assert coef.shape == (7, 4, 2)
    assert np.all(coef[:, :, 0] >= 1) and np.all(coef[:, :, 0] <= O.P31 - 1)
    assert np.all(coef[:, :, 1] >= 0) and np.all(coef[:, :, 1] <= O.P31 - 1)
    # draw order: the first published splitmix64 output of state 0 is h1.a of t=0
    g = _load("splitmix64_seed0.json")
    r = [int(h, 16) for h in g["outputs_hex"]]
    c0 = O.draw_coefficients(0, 1)
    assert c0[0, 0, 0] == 1 + r[0] % (O.P31 - 1)
    assert c0[0, 0, 1] == r[1] % O.P31
    assert c0[0, 1, 0] == 1 + r[2] % (O.P31 - 1)
    # different seeds give different functions
    assert not np.array_equal(O.draw_coefficients(1, 3), O.draw_coefficients(2, 3))


# ------------------------------------------------------------ hash family ---
def test_hash_hand_worked_values():
    g = _load("hash_hand.json")
    for e in g["bucket"]:
        got = O.hash_bucket(e["a"], e["c"], np.array([e["x"]]), e["b"])[0]
        assert got == e["h"], e
    for e in g["sign"]:
        got = O.hash_sign(e["a"], e["c"], np.array([e["x"]]))[0]
        assert got == e["s"], e


def test_hash_uniform_and_pairwise():
    # Sec. 2.2 needs Pr[h(x) = h(y)] = 1/b for x != y; check the family gets
    # close over many draws (chi-square-style bounds, loose).
    b = 64
    x = np.arange(4096)
    hist = np.zeros(b)
    coll = 0
    trials = 400
    for s in range(trials):
        coef = O.draw_coefficients(s, 1)
        h = O.hash_bucket(coef[0, 0, 0], coef[0, 0, 1], x, b)
        hist += np.bincount(h, minlength=b)
        coll += int(h[3] == h[77])
    exp = hist.sum() / b
    chi2 = float(((hist - exp) ** 2 / exp).sum())
    assert chi2 < 3 * b
    assert abs(coll / trials - 1 / b) < 5 * math.sqrt((1 / b) / trials)
    # signs are balanced
    sg = O.hash_sign(*O.draw_coefficients(9, 1)[0, 1], np.arange(100000))
    assert abs(sg.mean()) < 0.02


# ------------------------------------------------------------ count sketch --
def test_count_sketch_hand_example():
    # p_u(x) = sum_i s(i) u_i x^{h(i)}: u = (1, 2, 3), h = (0, 2, 0), s = (+, -, +)
    # gives 1*x^0 - 2*x^2 + 3*x^0 = 4 - 2 x^2.
    got = O.count_sketch(np.array([1.0, 2.0, 3.0]), np.array([0, 2, 0]),
                         np.array([1, -1, 1]), 3)
    np.testing.assert_array_equal(got, [4.0, 0.0, -2.0])


def _random_problem(n1, n2, n3, b, d, seed):
    A = W.gaussian(n1, n2, seed)
    B = W.gaussian(n2, n3, seed + 1)
    tab = O.make_tables(seed + 2, max(n1, n3), b, d)
    return A, B, tab


# ------------------------------------------- three routes of Sec. 2.2 agree --
@pytest.mark.parametrize("n1,n2,n3,b,d", [
    (16, 9, 16, 32, 2),       # power-of-two b
    (23, 17, 11, 64, 3),      # ragged rectangular shapes
    (40, 12, 40, 100, 1),     # b not a power of two (5-smooth)
    (10, 5, 10, 7, 2),        # prime b
    (30, 8, 30, 2000, 1),     # b as in the Fig. 2 demonstration
])
def test_fft_route_equals_definition_and_convolution(n1, n2, n3, b, d):
    A, B, tab = _random_problem(n1, n2, n3, b, d, 100 + b)
    cf, imag = O.sketch_fft(A, B, tab, return_imag=True)
    cd = O.sketch_definition(A, B, tab)
    np.testing.assert_allclose(cf, cd, rtol=0, atol=1e-10 * np.abs(cd).max())
    assert imag < 1e-9 * np.abs(cd).max()
    if b <= 256:
        cc = O.sketch_convolution(A, B, tab)
        np.testing.assert_allclose(cc, cd, rtol=0, atol=1e-10 * np.abs(cd).max())


def test_fft_route_equals_convolution_at_b1024():
    # the plain-method shape (b = 1024, d = 1) scaled down in n: direct
    # O(b^2) convolution vs the FFT route at b = 1024
    A, B, tab = _random_problem(64, 32, 64, 1024, 1, 7)
    cf = O.sketch_fft(A, B, tab)
    cc = O.sketch_convolution(A, B, tab)
    assert O.rel_l2(cf, cc) < 1e-12


def test_bucket_values_match_full_definition():
    A, B, tab = _random_problem(50, 20, 45, 128, 2, 3)
    cd = O.sketch_definition(A, B, tab)
    zs = np.array([0, 5, 64, 127, 99])
    for t in range(2):
        np.testing.assert_allclose(O.sketch_bucket_values(A, B, tab, t, zs), cd[t, zs],
                                   rtol=1e-12, atol=1e-12)


def test_batched_bucket_values_match_full_definition():
    # the many-bucket form (rows of A and columns of B, chunked dot products)
    # gives every bucket of the definition, with chunks that split buckets,
    # float32 rows widened exactly, and a bucket list with repeats
    A, B, tab = _random_problem(61, 23, 47, 96, 3, 5)
    cd = O.sketch_definition(A, B, tab)
    zs = np.array(list(range(96)) + [7, 7])
    for t in range(3):
        got = O.sketch_bucket_values_rows(np.ascontiguousarray(A), np.ascontiguousarray(B.T), tab, t, zs,
                                          chunk=17)
        np.testing.assert_allclose(got, cd[t, zs], rtol=1e-12, atol=1e-12 * np.abs(cd).max())
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    cd32 = O.sketch_definition(A32.astype(np.float64), B32.astype(np.float64), tab)
    got = O.sketch_bucket_values_rows(np.ascontiguousarray(A32), np.ascontiguousarray(B32.T), tab, 1,
                                      np.arange(96))
    np.testing.assert_allclose(got, cd32[1], rtol=1e-12, atol=1e-12 * np.abs(cd32).max())


# ------------------------------------------- special cases -> brute force ---
def test_injective_hash_gives_exact_product():
    # h1(i) = i, h2(j) = n1 j, b = n1 n3: every (i, j) has its own bucket
    # i + n1 j, so c is vec(AB) with the signs s1(i) s2(j) (Sec. 2.2).
    n1, n2, n3 = 6, 5, 4
    A = W.gaussian(n1, n2, 1)
    B = W.gaussian(n2, n3, 2)
    n = max(n1, n3)
    g = W.rng(3)
    s1 = g.choice([-1, 1], size=(1, n))
    s2 = g.choice([-1, 1], size=(1, n))
    h1 = np.arange(n)[None, :]
    h2 = (n1 * np.arange(n))[None, :]
    tab = O.Tables(h1, s1, h2, s2, n1 * n3)
    c = O.sketch_fft(A, B, tab)[0]
    AB = np.array([[sum(A[i, k] * B[k, j] for k in range(n2)) for j in range(n3)]
                   for i in range(n1)])
    for i in range(n1):
        for j in range(n3):
            assert abs(c[i + n1 * j] - s1[0, i] * s2[0, j] * AB[i, j]) < 1e-12
    # and decoding recovers AB exactly
    est = O.decompress_dense(c[None, :], tab, n1, n3)
    np.testing.assert_allclose(est, AB, atol=1e-12)


def test_b1_is_ams_sketch():
    # b = 1: every entry in one bucket; c_0 = sum_ij s1(i)s2(j)(AB)_ij
    # = (sum_i s1(i) a_i)(sum_j s2(j) b_j) summed over k (Sec. 2.1).
    A, B, tab = _random_problem(20, 7, 13, 1, 3, 11)
    c = O.sketch_fft(A, B, tab)
    for t in range(3):
        lhs = sum((tab.s1[t, :20] @ A[:, k]) * (B[k, :] @ tab.s2[t, :13]) for k in range(7))
        assert abs(c[t, 0] - lhs) < 1e-10 * max(1.0, abs(lhs))


def test_dc_bin_sum_is_ams_sketch():
    # sum_z c_z = (s1^T A)(B s2) for any b (the t = 0 spectral bin; Sec. 2.1/2.2)
    A, B, tab = _random_problem(31, 9, 27, 64, 2, 5)
    c = O.sketch_fft(A, B, tab)
    for t in range(2):
        lhs = (tab.s1[t, :31] @ A) @ (B @ tab.s2[t, :27])
        assert abs(c[t].sum() - lhs) < 1e-10 * max(1.0, abs(lhs))


def test_linearity_and_k_permutation():
    # the sketch is linear in each outer product a_k b_k (eq. (1), Sec. 2.2)
    A, B, tab = _random_problem(20, 10, 20, 32, 2, 21)
    A2 = W.gaussian(20, 10, 99)
    c1 = O.sketch_fft(A, B, tab)
    c2 = O.sketch_fft(A2, B, tab)
    c12 = O.sketch_fft(2.0 * A - 3.0 * A2, B, tab)
    np.testing.assert_allclose(c12, 2.0 * c1 - 3.0 * c2, atol=1e-10)
    perm = W.rng(4).permutation(10)
    cp = O.sketch_fft(A[:, perm], B[perm, :], tab)
    np.testing.assert_allclose(cp, c1, atol=1e-10)
    # split over k: sketch(A,B) = sketch(A[:, :4], B[:4]) + sketch(A[:, 4:], B[4:])
    cs = O.sketch_fft(A[:, :4], B[:4], tab) + O.sketch_fft(A[:, 4:], B[4:], tab)
    np.testing.assert_allclose(cs, c1, atol=1e-10)


def test_median_convention():
    assert O.median(np.array([3.0, 1.0, 2.0])) == 2.0
    assert O.median(np.array([1.0, 2.0, 3.0, 10.0])) == 2.5
    assert O.median(np.array([[5.0, -1.0], [4.0, 7.0], [6.0, 0.0]]), axis=0).tolist() == [5.0, 0.0]


def test_decompress_formula_on_hand_sketch():
    # DECOMPRESS of Fig. 1 with hand-chosen tables and sketch.
    h1 = np.array([[0, 1], [1, 1], [2, 0]])
    s1 = np.array([[1, -1], [1, 1], [-1, 1]])
    h2 = np.array([[2, 0], [0, 3], [1, 1]])
    s2 = np.array([[-1, 1], [1, 1], [1, -1]])
    tab = O.Tables(h1, s1, h2, s2, 4)
    c = np.array([[10., 20., 30., 40.], [1., 2., 3., 4.], [-5., 6., -7., 8.]])
    # (i, j) = (1, 0): t0: s=-1*-1=1, z=(1+2)%4=3 -> 40; t1: 1*1, z=(1+0)=1 -> 2;
    # t2: 1*1, z=(0+1)=1 -> 6.  median(40, 2, 6) = 6.
    assert O.decompress(c, tab, [1], [0])[0] == 6.0
    # (0, 1): t0: 1*1, z=(0+0)=0 -> 10; t1: 1*1, z=(1+3)%4=0 -> 1; t2: -1*-1, z=(2+1)=3 -> 8
    assert O.decompress(c, tab, [0], [1])[0] == 8.0


# ------------------------------------------------------ Theorem 2 (Sec 3.1) --
def test_theorem2_unbiased_and_variance_bound():
    # d = 1, many independent hash draws: the estimator C_ij is unbiased and
    # Var <= ||AB||_F^2 / b.  Data: 64 x 64 N(0,1), b = 256, 2000 seeds.
    n, b, seeds = 64, 256, 2000
    A = W.gaussian(n, n, 1)
    B = W.gaussian(n, n, 2)
    AB = A @ B
    fro2 = float((AB ** 2).sum())
    s = np.zeros((n, n))
    s2 = np.zeros((n, n))
    for seed in range(1, seeds + 1):
        tab = O.make_tables(seed, n, b, 1)
        c = O.sketch_definition(A, B, tab)
        est = O.decompress_dense(c, tab, n, n)
        s += est
        s2 += est * est
    mean = s / seeds
    var = s2 / seeds - mean ** 2
    sigma = math.sqrt(fro2 / b)
    assert np.max(np.abs(mean - AB)) < 6.0 * sigma / math.sqrt(seeds)
    # per-entry exact variance for a collision probability of 1/b is
    # (||AB||_F^2 - AB_ij^2)/b; check the average against the bound
    avg_var = float(var.mean())
    expected = (fro2 - float((AB ** 2).mean())) / b
    assert avg_var <= 1.08 * fro2 / b
    assert avg_var >= 0.85 * expected


def test_theorem2_fft_route_single_seed_matches_definition():
    # the statistical test above uses the definition route; it equals the
    # FFT route seed by seed
    A = W.gaussian(64, 64, 1)
    B = W.gaussian(64, 64, 2)
    tab = O.make_tables(17, 64, 256, 1)
    assert O.rel_l2(O.sketch_fft(A, B, tab), O.sketch_definition(A, B, tab)) < 1e-12


# --------------------------------------------------- Theorem 5 (Sec 3.3.1) --
def test_theorem5_sparse_product_recovered_exactly():
    # AB with at most b/8 nonzeros and d >= 6 lg n: median decoding returns AB.
    n, b = 64, 1024
    d = 6 * int(math.log2(n))
    sb = W.sparse_blocks(n, n_blocks=2, inner=3, rows=8, cols=8, seed=5)
    A, B = sb.scipy()
    AB = (A @ B).toarray()
    assert np.count_nonzero(AB) <= b // 8
    tab = O.make_tables(2024, n, b, d)
    c = O.sketch_definition(A.toarray(), B.toarray(), tab)
    est = O.decompress_dense(c, tab, n, n)
    np.testing.assert_array_equal(np.rint(est), AB)


def test_sparse_routes_agree_and_are_integers():
    sb = W.sparse_blocks(512, n_blocks=8, inner=4, rows=6, cols=5, seed=9)
    A, B = sb.scipy()
    tab = O.make_tables(3, 512, 256, 3)
    cd = O.sketch_definition_sparse(A, B, tab)
    cf = O.sketch_fft_sparse(A, B, tab)
    cdense = O.sketch_definition(A.toarray(), B.toarray(), tab)
    np.testing.assert_array_equal(cd, np.rint(cd))
    np.testing.assert_allclose(cf, cd, atol=1e-9)
    np.testing.assert_array_equal(cdense, cd)


# ---------------------------------------------------------- Fig. 2 (qual.) --
def test_fig2_planted_pair_stands_out():
    # Fig. 2: 100 x 100 uniform[-1, 1] data, rows 21 and 66 positively
    # correlated, b = 2000; after removing the diagonal's contribution and
    # thresholding, the planted pair is among the candidates.  Qualitative.
    n, m, b = 100, 100, 2000
    X = W.uniform_pm1(n, m, 42)
    X[66] = 0.9 * X[21] + 0.1 * X[66]
    tab = O.make_tables(7, n, b, 3)
    c = O.sketch_definition(X, X.T, tab)
    c = O.remove_diagonal(c, O.product_diagonal(X, X.T), tab)
    est = O.decompress_dense(c, tab, n, n)
    thr = 0.5 * est[21, 66]
    cand = set(map(tuple, O.candidates(c, tab, n, n, thr)))
    assert (21, 66) in cand and (66, 21) in cand
    assert len(cand) < 0.02 * n * n


# ----------------------------------------- covariance post-steps (Sec. 3.2) --
def test_product_diagonal_brute_force():
    A = W.gaussian(7, 5, 61)
    B = W.gaussian(5, 9, 62)
    want = [sum(A[i, k] * B[k, i] for k in range(5)) for i in range(7)]
    np.testing.assert_allclose(O.product_diagonal(A, B), want, rtol=1e-13)


def test_remove_diagonal_is_the_sketch_of_the_offdiagonal_part():
    # the sketch of Q~ computed from its definition (AB with a zero
    # diagonal, sketched as the product (AB - D) I) equals the sketch of AB
    # with the diagonal's contributions removed
    n1, n2, n3, b, d = 30, 11, 26, 97, 3
    A = W.gaussian(n1, n2, 63)
    B = W.gaussian(n2, n3, 64)
    tab = O.make_tables(65, max(n1, n3), b, d)
    AB = A @ B
    off = AB.copy()
    m = min(n1, n3)
    off[np.arange(m), np.arange(m)] = 0.0
    want = O.sketch_definition(off, np.eye(n3), tab)
    got = O.remove_diagonal(O.sketch_definition(A, B, tab), O.product_diagonal(A, B), tab)
    np.testing.assert_allclose(got, want, atol=1e-11)


@pytest.mark.parametrize("skip", [True, False])
def test_candidates_with_injective_hashes_are_the_large_entries(skip):
    # with an injective splitting function every estimate is (AB)_ij itself
    # (Sec. 2.2), so the candidates are exactly the entries above the
    # threshold, found here by brute force
    n1, n2, n3 = 9, 4, 8
    A = np.round(W.gaussian(n1, n2, 66) * 4)
    B = np.round(W.gaussian(n2, n3, 67) * 4)
    n = max(n1, n3)
    g = W.rng(68)
    tab = O.Tables(np.arange(n)[None, :].repeat(3, 0), g.choice([-1, 1], size=(3, n)),
                   (n1 * np.arange(n))[None, :].repeat(3, 0), g.choice([-1, 1], size=(3, n)), n1 * n3)
    c = O.sketch_definition(A, B, tab)
    AB = A @ B
    tau = 10.5
    want = [(i, j) for i in range(n1) for j in range(n3) if abs(AB[i, j]) > tau and (i != j or not skip)]
    got = [tuple(p) for p in O.candidates(c, tab, n1, n3, tau, skip_diagonal=skip)]
    assert got == want


# ------------------------------------------------ Sec. 5.2 (AMS, 4-wise) ----
def test_sign4_hand_worked_values():
    # a0..a3 = 5, 3, 2, 7: x = 0 -> 5 (odd, -1); x = 1 -> 17 (odd, -1);
    # x = 2 -> 5 + 6 + 8 + 56 = 75 (odd, -1); x = 3 -> 5 + 9 + 18 + 189 = 221 (odd);
    # x = 4 -> 5 + 12 + 32 + 448 = 497 (odd); x = 5 -> 5 + 15 + 50 + 875 = 945 (odd)
    coef = np.array([5, 3, 2, 7])
    assert O.sign4(coef, np.arange(6)).tolist() == [-1] * 6
    # a3 x^3 wraps the modulus: x = 2^11, a3 = 1: 2^33 mod (2^31 - 1) = 4 (even, +1)
    assert O.sign4(np.array([0, 0, 0, 1]), np.array([1 << 11])).tolist() == [1]
    # x = 2^11 with a1 = 1 only: 2048 (even, +1); a0 = p - 1 (even): +1; a0 = p - 2: -1
    assert O.sign4(np.array([0, 1, 0, 0]), np.array([1 << 11])).tolist() == [1]
    assert O.sign4(np.array([(1 << 31) - 2, 0, 0, 0]), np.array([9])).tolist() == [1]
    assert O.sign4(np.array([(1 << 31) - 3, 0, 0, 0]), np.array([9])).tolist() == [-1]


def test_sign4_coefficients_in_range_and_ordered():
    coef = O.draw_sign4_coefficients(123, 3)
    assert coef.shape == (3, 2, 4)
    assert coef.min() >= 0 and coef.max() < (1 << 31) - 1
    state = 123
    flat = []
    for _ in range(24):
        state, r = O.splitmix64(state)
        flat.append(r % ((1 << 31) - 1))
    assert coef.reshape(-1).tolist() == flat


def test_ams_estimate_is_the_signed_sum_of_ab():
    A = W.gaussian(9, 4, 71)
    B = W.gaussian(4, 7, 72)
    X = O.ams_frobenius(A, B, 73, 3)
    coef = O.draw_sign4_coefficients(73, 3)
    AB = A @ B
    for t in range(3):
        s1 = O.sign4(coef[t, 0], np.arange(9))
        s2 = O.sign4(coef[t, 1], np.arange(7))
        want = sum(s1[i] * s2[j] * AB[i, j] for i in range(9) for j in range(7))
        assert abs(X[t] - want) < 1e-10


def test_ams_square_unbiased_and_variance_bound():
    # Sec. 5.2: E[X^2] = ||AB||_F^2, Var[X^2] <= 8 E[X^2]^2 (4-wise signs)
    A = W.gaussian(12, 5, 74)
    B = W.gaussian(5, 10, 75)
    fro2 = float(np.sum((A @ B) ** 2))
    X = O.ams_frobenius(A, B, 76, 4000)
    sq = X ** 2
    se = np.sqrt(8.0) * fro2 / np.sqrt(len(sq))      # the standard error the bound allows
    assert abs(sq.mean() - fro2) < 4 * se
    assert sq.var() <= 8 * fro2 ** 2 * 1.3
    # and the bound of 32 medians is above ||AB||_F^2 for most seeds
    ok = sum(O.frobenius_bound(O.ams_frobenius(A, B, 1000 + q, 9)) >= fro2 for q in range(60))
    assert ok >= 57


def test_sign4_four_wise_products_vanish_on_average():
    # for 4 distinct points the product of the signs has mean 0 over draws
    xs = np.array([0, 1, 2, 3])
    prods = []
    for q in range(3000):
        c = O.draw_sign4_coefficients(5000 + q, 1)[0, 0]
        s = O.sign4(c, xs)
        prods.append(int(np.prod(s)))
    assert abs(np.mean(prods)) < 4 / np.sqrt(3000)


# ------------------------------------------- Sec. 5.1 (doubling search) ----
def _distinct_buckets(rows, cols, seed, d, b):
    coef = O.draw_coefficients(seed, d)
    out = []
    for t in range(d):
        h1 = [((int(coef[t, 0, 0]) * int(i) + int(coef[t, 0, 1])) % ((1 << 31) - 1)) % b for i in rows]
        h2 = [((int(coef[t, 2, 0]) * int(j) + int(coef[t, 2, 1])) % ((1 << 31) - 1)) % b for j in cols]
        out.append(len({(x + y) % b for x, y in zip(h1, h2)}))
    return out


def test_nnz_doubling_stops_at_the_first_b_with_a_fifth_occupied():
    # brute force with Python integers: the returned b is the first power of
    # two whose every repetition occupies at most b/5 buckets
    g = W.rng(101)
    rows = g.integers(0, 500, 60)
    cols = g.integers(0, 500, 60)
    b, worst = O.nnz_doubling(rows, cols, 102, 4, 1 << 16)
    assert b > 0
    assert max(_distinct_buckets(rows, cols, 102, 4, b)) == worst and 5 * worst <= b
    bb = 2
    while bb < b:
        assert 5 * max(_distinct_buckets(rows, cols, 102, 4, bb)) > bb
        bb *= 2


def test_nnz_doubling_is_a_five_approximation():
    # the search ends by the time b/5 reaches the number of nonzeros, so
    # b <= 10 nnz; and (whp, Sec. 5.1) b is at least the number of nonzeros
    g = W.rng(103)
    ok = 0
    for q in range(40):
        nnz = int(g.integers(20, 400))
        flat = g.choice(1000 * 1000, nnz, replace=False)
        b, worst = O.nnz_doubling(flat // 1000, flat % 1000, 200 + q, 5, 1 << 20)
        assert 0 < b <= 10 * nnz and worst <= nnz
        ok += b >= nnz
    assert ok >= 36


# ------------------------------------- Sec. 4 (FINDSIGNIFICANTENTRIES) -----
def test_code_round_trip_and_error_correction():
    L, rho = 7, 3
    g = W.rng(130)
    for x in [0, 1, 77, 127] + g.integers(0, 128, 20).tolist():
        e = O.code_bits(x, L, rho)
        assert len(e) == 2 * rho * L and e.sum() == rho * L
        assert O.decode_code(e, L, rho) == x
        # one flip in every bit's group of 2 rho is corrected (votes stay a majority)
        f = e.copy()
        for q in range(L):
            f[q * 2 * rho + g.integers(0, 2 * rho)] ^= 1
        assert O.decode_code(f, L, rho) == x
    # an empty bucket (all bits 0) and an all-ones string decode to nothing
    assert O.decode_code(np.zeros(2 * rho * L, dtype=np.int64), L, rho) == -1
    assert O.decode_code(np.ones(2 * rho * L, dtype=np.int64), L, rho) == -1
    # rho = 1: a flip makes a tie, which is rejected
    e = O.code_bits(5, 3, 1)
    e[0] ^= 1
    assert O.decode_code(e, 3, 1) == -1


def test_find_significant_returns_the_planted_entries():
    # AB with a few large entries over small noise, b large enough that the
    # large entries rarely share a bucket: the result is the set of entries
    # above Delta, found by brute force
    n1, n2, n3, b, d = 40, 6, 36, 8192, 5
    g = W.rng(131)
    A = 0.01 * g.standard_normal((n1, n2))
    B = 0.01 * g.standard_normal((n2, n3))
    big = [(3, 5), (17, 30), (39, 0), (21, 21)]
    for q, (i, j) in enumerate(big):
        A[i, q] += 10.0
        B[q, j] += 10.0 + q
    AB = A @ B
    delta = 50.0
    want = sorted((int(i), int(j)) for i, j in zip(*np.nonzero(np.abs(AB) > delta)))
    assert len(want) >= len(big)
    tab = O.make_tables(132, max(n1, n3), b, d)
    for rho in (1, 2):
        got = [tuple(p) for p in O.find_significant(A, B, tab, delta, rho)]
        assert got == want


# ------------------------------------ single row and column; Parseval (FFT) --
def test_single_row_and_column_is_one_bucket():
    # n1 = n3 = 1: AB is the number sum_k A_0k B_k0, and every route of the
    # sketch puts s1(0) s2(0) AB into bucket (h1(0) + h2(0)) mod b alone
    b, d = 40, 3
    A = W.gaussian(1, 13, 61)
    B = W.gaussian(13, 1, 62)
    tab = O.make_tables(63, 1, b, d)
    ab = float(sum(A[0, k] * B[k, 0] for k in range(13)))
    for route in (O.sketch_fft, O.sketch_definition, O.sketch_convolution):
        c = route(A, B, tab)
        for t in range(d):
            z = (int(tab.h1[t][0]) + int(tab.h2[t][0])) % b
            want = np.zeros(b)
            want[z] = int(tab.s1[t][0]) * int(tab.s2[t][0]) * ab
            np.testing.assert_allclose(c[t], want, rtol=1e-12, atol=1e-12)


def test_parseval_holds_for_the_fft_route():
    # energy of c = (1/b) x energy of the product spectrum sum_k PA_k PB_k,
    # with the count sketches built here by loops and their spectra taken with
    # an explicit DFT matrix (no FFT routine): pins the FFT route's inverse
    # scaling and its real output
    n1, n2, n3, b, d = 12, 7, 9, 24, 2
    A, B, tab = _random_problem(n1, n2, n3, b, d, 71)
    c = O.sketch_fft(A, B, tab)
    F = np.exp(-2j * np.pi * np.outer(np.arange(b), np.arange(b)) / b)
    for t in range(d):
        spec = np.zeros(b, dtype=np.complex128)
        for k in range(n2):
            pa = np.zeros(b)
            pb = np.zeros(b)
            for i in range(n1):
                pa[tab.h1[t][i]] += tab.s1[t][i] * A[i, k]
            for j in range(n3):
                pb[tab.h2[t][j]] += tab.s2[t][j] * B[k, j]
            spec += (F @ pa) * (F @ pb)
        assert abs(np.sum(c[t] ** 2) - np.sum(np.abs(spec) ** 2) / b) <= 1e-9 * np.sum(np.abs(spec) ** 2) / b
