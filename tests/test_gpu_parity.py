"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: hash tables and bucket indices bit-exact; the sketch c within
relative L2 1e-5 per repetition for FP32 (and FP64-stored) inputs, 3e-3 for
BF16 storage against the unrounded data and 1e-5 against the BF16 values
themselves; the plain FP64 path within 1e-10; decoding exact when fed the
oracle's own sketch.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import cms_oracle as O

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_BF16 = 3e-3


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


def colmajor(A: np.ndarray, dtype=torch.float32) -> torch.Tensor:
    """Device copy of A (n1 x n2) in column-major order."""
    return torch.from_numpy(np.ascontiguousarray(A.T)).to(dev(), dtype).T


def rowmajor(B: np.ndarray, dtype=torch.float32) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(B)).to(dev(), dtype)


# ------------------------------------------------------------ hash tables --
@pytest.mark.parametrize("seed,n,b,d", [(1, 256, 1024, 1), (2, 2048, 65536, 5), (3, 1000, 2000, 3),
                                        (4, 37, 7, 2), (5, 5000, 1, 1), (6, 70000, 1 << 20, 3),
                                        (2**64 - 1, 64, 16384, 64)])
def test_hash_tables_bit_exact(cms, seed, n, b, d):
    h = cms.make_hashes(seed, n, b, d)
    h1, s1, h2, s2 = h.tables()
    tab = O.make_tables(seed, n, b, d)
    np.testing.assert_array_equal(h1, tab.h1)
    np.testing.assert_array_equal(s1, tab.s1)
    np.testing.assert_array_equal(h2, tab.h2)
    np.testing.assert_array_equal(s2, tab.s2)
    coef = O.draw_coefficients(seed, d)
    for t in range(d):
        np.testing.assert_array_equal(h.coeffs(t), coef[t].reshape(-1))
    h.free()


@pytest.mark.parametrize("seed,n,b,d", [(2, 2048, 65536, 5), (3, 1000, 2000, 3), (6, 70000, 1 << 20, 2),
                                        (7, 5000, 1, 1), (8, 333, 3 * 1024, 2)])
def test_bucket_lists_are_the_stable_sort(cms, seed, n, b, d):
    # the gather front ends read each bucket class z = h(x) mod C in the order
    # of a stable sort of x by z: perm and off must equal numpy's stable
    # argsort and class counts of the oracle's tables, bit for bit
    h = cms.make_hashes(seed, n, b, d)
    C = h.info()["C"]
    tab = O.make_tables(seed, n, b, d)
    for t in range(d):
        for side, hh in ((0, tab.h1), (1, tab.h2)):
            perm, off = h.buckets(t, side)
            key = np.asarray(hh[t], dtype=np.int64) % C
            np.testing.assert_array_equal(perm, np.argsort(key, kind="stable"))
            np.testing.assert_array_equal(off, np.concatenate([[0], np.cumsum(np.bincount(key, minlength=C))]))
    h.free()


def test_bucket_lists_need_a_factorisation(cms):
    h = cms.make_hashes(1, 64, 7, 1)            # prime b: no FFT split, no lists
    with pytest.raises(cms.CmsError) as e:
        h.buckets(0, 0)
    assert e.value.status == 2
    h.free()


def test_reseed_matches_fresh_tables(cms):
    h = cms.make_hashes(10, 3000, 4096, 3)
    h.reseed(11)
    torch.cuda.synchronize()
    h1, s1, h2, s2 = h.tables()
    tab = O.make_tables(11, 3000, 4096, 3)
    np.testing.assert_array_equal(h1, tab.h1)
    np.testing.assert_array_equal(s2, tab.s2)
    h.free()


# ------------------------------------------------------- sketch parity -----
CASES = [
    # n1, n2, n3, b, d  (A n1 x n2, B n2 x n3)
    (256, 256, 256, 1024, 1),      # the plain-method configuration, b = 1024
    (100, 37, 77, 4096, 3),        # ragged shapes, R = 4 rows of C = 1024
    (2048, 40, 2048, 65536, 5),    # the covariance configuration's n and b, few k
    (500, 64, 300, 2000, 2),       # b = 2000 as in Fig. 2 (5-smooth, C = 1000)
    (64, 10, 64, 1, 2),            # b = 1: the AMS sketch
    (33, 5, 17, 12, 3),            # tiny mixed-radix b
    (300, 129, 301, 3 * 1024, 4),  # R = 3 (odd), ragged k tail
    (1, 9, 1, 8, 1),               # single row / column
]


@pytest.mark.parametrize("n1,n2,n3,b,d", CASES)
def test_sketch_f32_matches_oracle(cms, n1, n2, n3, b, d):
    A = W.gaussian(n1, n2, 1000 + n1)
    B = W.gaussian(n2, n3, 2000 + n3)
    Af = A.astype(np.float32)
    Bf = B.astype(np.float32)
    n = max(n1, n3)
    h = cms.make_hashes(77 + b, n, b, d)
    c = cms.sketch_product(colmajor(Af), rowmajor(Bf), h).cpu().numpy()
    cms.check_async()
    tab = O.make_tables(77 + b, n, b, d)
    ref = O.sketch_definition(Af.astype(np.float64), Bf.astype(np.float64), tab)
    assert O.rel_l2(c, ref) < TOL_F32
    h.free()


def test_sketch_empty_inner_dimension_is_zero(cms):
    h = cms.make_hashes(1, 50, 1024, 2)
    A = torch.zeros((50, 0), device=dev())
    B = torch.zeros((0, 40), device=dev())
    c = cms.sketch_product(A, B, h)
    assert torch.count_nonzero(c).item() == 0
    h.free()


def test_sketch_is_deterministic(cms):
    A = W.gaussian(700, 90, 5).astype(np.float32)
    h = cms.make_hashes(3, 700, 8192, 3)
    a = colmajor(A)
    bm = rowmajor(A.T)
    c1 = cms.sketch_product(a, bm, h)
    c2 = cms.sketch_product(a, bm, h)
    assert torch.equal(c1, c2)
    h.free()


def test_sketch_bf16_storage(cms):
    n, m, b, d = 600, 200, 8192, 3
    X = W.gaussian(m, n, 31).astype(np.float32)
    Xb, _ = W.bf16_round(X)
    h = cms.make_hashes(4, n, b, d)
    xt = torch.from_numpy(X).to(dev(), torch.bfloat16)
    c = cms.sketch_product(xt.T, xt, h).cpu().numpy()
    tab = O.make_tables(4, n, b, d)
    ref_bf16 = O.sketch_definition(Xb.T.astype(np.float64), Xb.astype(np.float64), tab)
    ref_f32 = O.sketch_definition(X.T.astype(np.float64), X.astype(np.float64), tab)
    assert O.rel_l2(c, ref_bf16) < TOL_F32
    assert O.rel_l2(c, ref_f32) < TOL_BF16
    h.free()


@pytest.mark.parametrize("n1,n2,n3,b,d", [
    (304, 45, 296, 3840, 2),      # C = 960, two operands
    (512, 33, 504, 4096, 2),      # C = 1024, two operands
])
def test_sketch_bf16_storage_two_operands(cms, n1, n2, n3, b, d):
    # BF16 rows staged as BF16 by the register-FFT kernel; the sketch of the
    # BF16 values within the FP32 tolerance
    A = W.gaussian(n1, n2, 3 + n1).astype(np.float32)
    B = W.gaussian(n2, n3, 5 + n3).astype(np.float32)
    Ab, _ = W.bf16_round(A)
    Bb, _ = W.bf16_round(B)
    n = max(n1, n3)
    h = cms.make_hashes(7 + b, n, b, d)
    c = cms.sketch_product(colmajor(A, torch.bfloat16), rowmajor(B, torch.bfloat16), h).cpu().numpy()
    ref = O.sketch_definition(Ab.astype(np.float64), Bb.astype(np.float64), O.make_tables(7 + b, n, b, d))
    assert O.rel_l2(c, ref) < TOL_F32
    h.free()


def test_sketch_f64_storage_fused(cms):
    A = W.gaussian(128, 50, 8)
    B = W.gaussian(50, 96, 9)
    h = cms.make_hashes(6, 128, 2048, 2)
    c = cms.sketch_product(colmajor(A, torch.float64), rowmajor(B, torch.float64), h).cpu().numpy()
    ref = O.sketch_definition(A, B, O.make_tables(6, 128, 2048, 2))
    assert O.rel_l2(c, ref) < TOL_F32
    h.free()


def test_sketch_strided_leading_dimensions(cms):
    # lda > n1 and ldb > n3: slices of larger buffers
    big_a = W.gaussian(70, 200, 3).astype(np.float32)      # stored as (n2, lda) rows
    big_b = W.gaussian(70, 150, 4).astype(np.float32)      # (n2, ldb)
    ta = torch.from_numpy(big_a).to(dev())
    tb = torch.from_numpy(big_b).to(dev())
    A = ta[:, :120].T            # n1 = 120, n2 = 70, lda = 200
    B = tb[:, :100]              # n3 = 100, ldb = 150
    h = cms.make_hashes(8, 120, 4096, 2)
    c = cms.sketch_product(A, B, h).cpu().numpy()
    ref = O.sketch_definition(big_a[:, :120].T.astype(np.float64), big_b[:, :100].astype(np.float64),
                              O.make_tables(8, 120, 4096, 2))
    assert O.rel_l2(c, ref) < TOL_F32
    h.free()


def test_sketch_on_side_stream_and_merge(cms):
    # linearity over k (eq. (1)): sketches of two k-ranges merge to the whole
    A = W.gaussian(300, 80, 12).astype(np.float32)
    B = W.gaussian(80, 260, 13).astype(np.float32)
    h = cms.make_hashes(9, 300, 16384, 3)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = colmajor(A)
        bm = rowmajor(B)
        c_all = cms.sketch_product(a, bm, h, stream=s)
        c1 = cms.sketch_product(a[:, :33], bm[:33], h, stream=s)
        c2 = cms.sketch_product(a[:, 33:], bm[33:], h, stream=s)
        cm = cms.merge([c1, c2], stream=s)
    s.synchronize()
    ref = O.sketch_definition(A.astype(np.float64), B.astype(np.float64), O.make_tables(9, 300, 16384, 3))
    assert O.rel_l2(c_all.cpu().numpy(), ref) < TOL_F32
    assert O.rel_l2(cm.cpu().numpy(), ref) < TOL_F32
    h.free()


def test_injective_hash_recovers_product(cms):
    # h1(i) = i, h2(j) = n1 j, b = n1 n3: c = vec(AB) with signs (Sec. 2.2)
    n1, n2, n3 = 16, 20, 8
    A = W.gaussian(n1, n2, 1).astype(np.float32)
    B = W.gaussian(n2, n3, 2).astype(np.float32)
    n = n1
    g = W.rng(3)
    s1 = g.choice([-1, 1], size=(1, n)).astype(np.int8)
    s2 = g.choice([-1, 1], size=(1, n)).astype(np.int8)
    h1 = np.arange(n, dtype=np.uint32)[None, :]
    h2 = (n1 * np.arange(n, dtype=np.uint32))[None, :]
    h2 = np.minimum(h2, n1 * n3 - 1).astype(np.uint32)   # columns >= n3 are never used
    h = cms.Hashes.from_tables(h1, s1, h2, s2, n1 * n3)
    c = cms.sketch_product(colmajor(A), rowmajor(B), h)
    ii, jj = np.meshgrid(np.arange(n1), np.arange(n3), indexing="ij")
    ij = torch.from_numpy(np.stack([ii.ravel(), jj.ravel()], 1).astype(np.int64)).to(dev())
    est = cms.decode(c, h, ij).cpu().numpy().reshape(n1, n3)
    AB = A.astype(np.float64) @ B.astype(np.float64)
    np.testing.assert_allclose(est, AB, atol=2e-5 * np.abs(AB).max())
    h.free()


# ------------------------------------------------------------ plain FP64 --
@pytest.mark.parametrize("n1,n2,n3,b,d", [(256, 256, 256, 1024, 1), (100, 37, 77, 4096, 3),
                                          (500, 64, 300, 2000, 2), (64, 10, 64, 1, 2)])
def test_plain_f64_matches_oracle(cms, n1, n2, n3, b, d):
    A = W.gaussian(n1, n2, 10 + n1)
    B = W.gaussian(n2, n3, 20 + n3)
    n = max(n1, n3)
    h = cms.make_hashes(55, n, b, d)
    c = cms.sketch_product_plain_f64(colmajor(A, torch.float64), rowmajor(B, torch.float64), h)
    ref = O.sketch_definition(A, B, O.make_tables(55, n, b, d))
    assert O.rel_l2(c.cpu().numpy(), ref) < 1e-10
    h.free()


# ----------------------------------------------------------------- decode --
@pytest.mark.parametrize("d", [1, 2, 3, 5, 7, 8, 36])
def test_decode_exact_on_oracle_sketch(cms, d):
    # feed the oracle's sketch (rounded to FP32) to both decoders: median is a
    # selection, so odd d matches exactly; even d averages in FP32
    n1, n3, b = 300, 200, 4096
    rng = W.rng(d)
    c_ref = rng.standard_normal((d, b)).astype(np.float32)
    h = cms.make_hashes(100 + d, max(n1, n3), b, d)
    tab = O.make_tables(100 + d, max(n1, n3), b, d)
    ij = W.sample_pairs(n1, n3, 5000, 4)
    got = cms.decode(torch.from_numpy(c_ref).to(dev()), h, torch.from_numpy(ij).to(dev())).cpu().numpy()
    want = O.decompress(c_ref.astype(np.float64), tab, ij[:, 0], ij[:, 1])
    if d % 2:
        np.testing.assert_array_equal(got, want.astype(np.float32))
    else:
        np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-6)
    dense = cms.decode_dense(torch.from_numpy(c_ref).to(dev()), h, n1, n3).cpu().numpy()
    want_dense = O.decompress_dense(c_ref.astype(np.float64), tab, n1, n3)
    np.testing.assert_allclose(dense, want_dense, rtol=1e-6, atol=1e-6)
    h.free()


def test_decode_f64(cms):
    d, b = 5, 2048
    c_ref = W.rng(1).standard_normal((d, b))
    h = cms.make_hashes(3, 100, b, d)
    tab = O.make_tables(3, 100, b, d)
    ij = W.sample_pairs(100, 100, 1000, 2)
    got = cms.decode(torch.from_numpy(c_ref).to(dev()), h, torch.from_numpy(ij).to(dev())).cpu().numpy()
    np.testing.assert_array_equal(got, O.decompress(c_ref, tab, ij[:, 0], ij[:, 1]))
    h.free()


def test_decode_out_of_range_pair_raises(cms):
    h = cms.make_hashes(3, 10, 64, 1)
    c = torch.zeros((1, 64), device=dev())
    ij = torch.tensor([[0, 0], [10, 0]], dtype=torch.int64, device=dev())
    out = cms.decode(c, h, ij)
    with pytest.raises(cms.CmsError) as e:
        cms.check_async()
    assert e.value.status == 6
    assert math.isnan(out[1].item())
    cms.check_async()   # the word was cleared
    h.free()


# ---------------------------------------------------- argument checking ----
def test_invalid_arguments(cms):
    h = cms.make_hashes(1, 64, 1024, 1)
    A = torch.zeros((64, 8), device=dev()).T.contiguous().T  # column-major
    B = torch.zeros((8, 64), device=dev())
    with pytest.raises(ValueError):
        cms.sketch_product(A.contiguous(), B, h)            # row-major A rejected by binding
    ws = torch.empty(16, dtype=torch.uint8, device=dev())
    with pytest.raises(cms.CmsError) as e:
        cms.sketch_product(A, B, h, ws=ws)
    assert e.value.status == 4
    h7 = cms.make_hashes(1, 64, 7, 1)                       # prime b: no FFT factorisation
    with pytest.raises(cms.CmsError) as e:
        cms.sketch_product(A, B, h7)
    assert e.value.status == 2
    big = torch.zeros((65, 8), device=dev()).T.contiguous().T
    with pytest.raises(cms.CmsError) as e:
        cms.sketch_product(big, B, h)                        # n1 > n
    assert e.value.status == 1
    h.free()
    h7.free()


def test_binding_rejects_bad_buffers(cms):
    # the library sees only pointers: the binding checks every caller buffer
    # (device, dtype, layout, size) before a call can reach a kernel
    n, b, d = 64, 1024, 3
    h = cms.make_hashes(2, n, b, d)
    A = torch.zeros((n, 8), device=dev()).T.contiguous().T
    B = torch.zeros((8, n), device=dev())
    c = cms.sketch_product(A, B, h)
    bad_c = [torch.zeros((d, b - 1), device=dev()),                  # too small
             torch.zeros((d, b), device=dev(), dtype=torch.float64),  # wrong dtype
             torch.zeros((d, b)),                                     # host memory
             torch.zeros((b, d), device=dev()).T]                     # not contiguous
    for cc in bad_c:
        with pytest.raises(ValueError):
            cms.sketch_product(A, B, h, c=cc)
        with pytest.raises(ValueError):
            cms.remove_diagonal(A, B, h, cc)
    with pytest.raises(ValueError):
        cms.sketch_product(A, B, h, ws=torch.empty(1 << 20, dtype=torch.uint8))   # host workspace
    with pytest.raises(ValueError):
        cms.sketch_product(A, B.cpu(), h)                                         # B on the host
    ij = torch.zeros((10, 2), dtype=torch.int64, device=dev())
    with pytest.raises(ValueError):
        cms.decode(c[:, : b // 2], h, ij)                                         # c shorter than d b
    with pytest.raises(ValueError):
        cms.decode(c, h, ij, out=torch.empty(9, device=dev()))                    # out too small
    with pytest.raises(ValueError):
        cms.decode(c, h, ij.cpu())                                                # pairs on the host
    with pytest.raises(ValueError):
        cms.decode_dense(c, h, n, n, out=torch.empty((n, n - 1), device=dev()))  # wrong out shape
    with pytest.raises(ValueError):
        cms.decode_threshold(c[:1], h, n, n, 1.0)                                 # one repetition only
    with pytest.raises(ValueError):
        cms.merge([c, torch.zeros((d, b - 1), device=dev())])                     # parts disagree
    with pytest.raises(ValueError):
        cms.merge([c], out=torch.zeros((d, b), device=dev(), dtype=torch.float64))
    h.free()


# ------------------------------------------------- Theorem 5, on the GPU ---
def test_theorem5_exact_sparse_on_gpu(cms):
    n, b = 64, 1024
    d = 6 * int(math.log2(n))
    sb = W.sparse_blocks(n, n_blocks=2, inner=3, rows=8, cols=8, seed=5)
    A, B = sb.scipy()
    Ad = A.toarray()
    Bd = B.toarray()
    h = cms.make_hashes(2024, n, b, d)
    c = cms.sketch_product(colmajor(Ad), rowmajor(Bd), h)
    tab = O.make_tables(2024, n, b, d)
    ref = O.sketch_definition(Ad, Bd, tab)
    np.testing.assert_array_equal(np.rint(c.cpu().numpy()), ref)
    est = cms.decode_dense(c, h, n, n).cpu().numpy()
    np.testing.assert_array_equal(np.rint(est), Ad @ Bd)
    h.free()


# ------------------------------------------ full-size covariance workload --
def test_covariance_full_size_sampled(cms):
    # X 4096 samples x 2048 variables FP32, 32 planted pairs rho = 0.5,
    # A = X^T, B = X, b = 65536, d = 5 (the benchmarked configuration).
    m, n, b, d = 4096, 2048, 65536, 5
    cov = W.covariance(m, n, 32, 0.5, seed=2, dtype=np.float32)
    X = torch.from_numpy(cov.X).to(dev())
    h = cms.make_hashes(2, n, b, d)
    c = cms.sketch_product(X.T, X, h).cpu().numpy().astype(np.float64)
    tab = O.make_tables(2, n, b, d)
    Xd = cov.X.astype(np.float64)
    zs = W.rng(22).choice(b, 128, replace=False)
    for t in range(d):
        want = O.sketch_bucket_values(Xd.T, Xd, tab, t, zs)
        err = np.linalg.norm(c[t, zs] - want) / np.linalg.norm(want)
        assert err < TOL_F32, (t, err)
        # the DC bin: sum_z c_z = (s1^T X^T)(X s2)  (Sec. 2.1)
        dc = (tab.s1[t] @ Xd.T) @ (Xd @ tab.s2[t])
        assert abs(c[t].sum() - dc) < 1e-5 * np.abs(c[t]).sum()
    h.free()


# ------------------------------------- C = 1024 register-FFT kernel cases --
@pytest.mark.parametrize("n1,n2,n3,b,d", [
    (300, 130, 304, 3 * 1024, 3),     # R = 3 (odd), ragged inner tail (130 = 4*32 + 2)
    (256, 7, 256, 1024, 2),           # R = 1, fewer k than one group
    (1024, 64, 512, 65536, 2),        # R = 64, rectangular
    (2044, 33, 2044, 1 << 20, 1),     # R = 1024 rows
])
def test_fast_kernel_cases_match_oracle(cms, n1, n2, n3, b, d):
    A = W.gaussian(n1, n2, 7 + n1).astype(np.float32)
    B = W.gaussian(n2, n3, 9 + n3).astype(np.float32)
    n = max(n1, n3)
    h = cms.make_hashes(31 + b, n, b, d)
    c = cms.sketch_product(colmajor(A), rowmajor(B), h).cpu().numpy()
    ref = O.sketch_definition(A.astype(np.float64), B.astype(np.float64), O.make_tables(31 + b, n, b, d))
    assert O.rel_l2(c, ref) < TOL_F32
    h.free()


# C = P Q for the other register-FFT lengths (b chosen so that P Q is the
# largest supported factor): P = 32 with Q = 30, 27, 25, 24, 20, 18, 16, and
# P, Q < 32
@pytest.mark.parametrize("n1,n2,n3,b,d", [
    (300, 70, 296, 3840, 2),      # C = 960, R = 4
    (500, 33, 500, 2592, 2),      # C = 864, R = 3
    (256, 41, 260, 4000, 3),      # C = 800, R = 5
    (400, 64, 400, 1536, 2),      # C = 768, R = 2
    (200, 29, 204, 1280, 2),      # C = 640, R = 2
    (300, 50, 300, 1152, 1),      # C = 576, R = 2
    (100, 17, 100, 512, 2),       # C = 512, R = 1
    (300, 40, 296, 10800, 2),     # C = 900 = 30 x 30, R = 12
    (256, 30, 256, 10000, 2),     # C = 625 = 25 x 25, R = 16
    (200, 25, 200, 11664, 1),     # C = 729 = 27 x 27, R = 16
    (100, 20, 100, 2000, 2),      # C = 500 = 25 x 20, R = 4
])
def test_fast_kernel_c_32l_match_oracle(cms, n1, n2, n3, b, d):
    A = W.gaussian(n1, n2, 17 + n1).astype(np.float32)
    B = W.gaussian(n2, n3, 19 + n3).astype(np.float32)
    n = max(n1, n3)
    h = cms.make_hashes(41 + b, n, b, d)
    c = cms.sketch_product(colmajor(A), rowmajor(B), h).cpu().numpy()
    ref = O.sketch_definition(A.astype(np.float64), B.astype(np.float64), O.make_tables(41 + b, n, b, d))
    assert O.rel_l2(c, ref) < TOL_F32
    h.free()


def test_fast_kernel_overflow_buckets(cms):
    # 32 entries per occupied bucket class: half of each goes through the
    # overflow list of the gather front end
    n, n2, b = 256, 40, 1024
    A = W.gaussian(n, n2, 1).astype(np.float32)
    B = W.gaussian(n2, n, 2).astype(np.float32)
    g = W.rng(5)
    h1 = (np.arange(n) % 8)[None, :].astype(np.uint32)
    h2 = g.integers(0, b, size=(1, n)).astype(np.uint32)
    s1 = g.choice([-1, 1], size=(1, n)).astype(np.int8)
    s2 = g.choice([-1, 1], size=(1, n)).astype(np.int8)
    h = cms.Hashes.from_tables(h1, s1, h2, s2, b)
    c = cms.sketch_product(colmajor(A), rowmajor(B), h).cpu().numpy()
    tab = O.Tables(h1.astype(np.int64), s1.astype(np.int64), h2.astype(np.int64), s2.astype(np.int64), b)
    ref = O.sketch_definition(A.astype(np.float64), B.astype(np.float64), tab)
    assert O.rel_l2(c, ref) < TOL_F32
    h.free()


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_fast_kernel_overflow_with_unaligned_rows(cms, dtype):
    # rows not in whole 16-byte units (n1, n3 not multiples of the 16-byte
    # element count; staged as aligned supersets) and side-a buckets of 31
    # or 32 entries: the overflow entries are walked per lane with the
    # staging offsets of unaligned rows, odd inner dimension
    n1, n2, n3, b = 250, 37, 253, 1024
    n = max(n1, n3)
    A = W.gaussian(n1, n2, 81).astype(np.float32)
    B = W.gaussian(n2, n3, 82).astype(np.float32)
    Ar = W.bf16_round(A)[0] if dtype == torch.bfloat16 else A
    Br = W.bf16_round(B)[0] if dtype == torch.bfloat16 else B
    g = W.rng(83)
    h1 = (np.arange(n) % 8 * 129)[None, :].astype(np.uint32)
    h2 = g.integers(0, b, size=(1, n)).astype(np.uint32)
    s1 = g.choice([-1, 1], size=(1, n)).astype(np.int8)
    s2 = g.choice([-1, 1], size=(1, n)).astype(np.int8)
    h = cms.Hashes.from_tables(h1, s1, h2, s2, b)
    Ad, Bd = colmajor(A, dtype), rowmajor(B, dtype)
    assert cms.plan_kernel(Ad, Bd, h) == "lockstep"
    c = cms.sketch_product(Ad, Bd, h).cpu().numpy()
    cms.check_async()
    tab = O.Tables(h1.astype(np.int64), s1.astype(np.int64), h2.astype(np.int64), s2.astype(np.int64), b)
    ref = O.sketch_definition(Ar.astype(np.float64), Br.astype(np.float64), tab)
    assert O.rel_l2(c, ref) < TOL_F32
    h.free()


@pytest.mark.parametrize("smem_swap", [False, True])
def test_warp_specialised_overflow_records_in_tensor_memory(cms, monkeypatch, smem_swap):
    # side-a hash with 128 buckets of 16 entries (8 past the records each)
    # and the other 896 empty: the warp-specialised front end keeps those
    # overflow entries as records in its free tensor-memory columns (192
    # per warp, or 256 in blocks that swap spectra through shared memory,
    # forced here by the library's debug switch); odd inner dimension,
    # X^T X (aliased operands)
    if smem_swap:
        monkeypatch.setenv("CMS_WS_SMEM_SWAP", "1")
    n, m, b = 2048, 45, 65536
    X = W.gaussian(m, n, 91).astype(np.float32)
    g = W.rng(92)
    h1 = ((np.arange(n) % 128) * 8 + 3 + 1024 * g.integers(0, 64, size=n))[None, :].astype(np.uint32)
    h2 = g.integers(0, b, size=(1, n)).astype(np.uint32)
    s1 = g.choice([-1, 1], size=(1, n)).astype(np.int8)
    s2 = g.choice([-1, 1], size=(1, n)).astype(np.int8)
    h = cms.Hashes.from_tables(h1, s1, h2, s2, b)
    xt = torch.from_numpy(X).to(dev())
    assert cms.plan_kernel(xt.T, xt, h) == "warp_specialised"
    c = cms.sketch_product(xt.T, xt, h).cpu().numpy()
    cms.check_async()
    tab = O.Tables(h1.astype(np.int64), s1.astype(np.int64), h2.astype(np.int64), s2.astype(np.int64), b)
    ref = O.sketch_definition(X.T.astype(np.float64), X.astype(np.float64), tab)
    assert O.rel_l2(c, ref) < TOL_F32
    h.free()


def test_overflow_lists_beyond_the_twiddle_cache(cms):
    # side-a hash with 2 buckets of 1024 entries each: 2032 entries go through
    # the overflow lists, more than the fused kernel caches per task (at most
    # 1024), so both the cached and the on-the-fly twiddles are used; X^T X
    # (aliased operands) as in the covariance workload
    n, m, b = 2048, 20, 2048
    X = W.gaussian(m, n, 31).astype(np.float32)
    g = W.rng(6)
    h1 = (np.arange(n) % 2 * 517)[None, :].astype(np.uint32)
    h2 = g.integers(0, b, size=(1, n)).astype(np.uint32)
    s1 = g.choice([-1, 1], size=(1, n)).astype(np.int8)
    s2 = g.choice([-1, 1], size=(1, n)).astype(np.int8)
    h = cms.Hashes.from_tables(h1, s1, h2, s2, b)
    xt = torch.from_numpy(X).to(dev())
    c = cms.sketch_product(xt.T, xt, h).cpu().numpy()
    tab = O.Tables(h1.astype(np.int64), s1.astype(np.int64), h2.astype(np.int64), s2.astype(np.int64), b)
    ref = O.sketch_definition(X.T.astype(np.float64), X.astype(np.float64), tab)
    assert O.rel_l2(c, ref) < TOL_F32
    h.free()


def test_fast_and_generic_kernels_agree(cms):
    # the same product through the register-FFT kernel with 16-byte aligned
    # rows (TMA copies of the rows), with rows that are not (A's leading
    # dimension n1 + 1: copies of the aligned supersets) and through the
    # shared-memory kernel (FP64 storage)
    n1, n2, n3, b, d = 512, 96, 512, 16384, 3
    A = W.gaussian(n1, n2, 3).astype(np.float32)
    B = W.gaussian(n2, n3, 4).astype(np.float32)
    h = cms.make_hashes(12, 512, b, d)
    c_fast = cms.sketch_product(colmajor(A), rowmajor(B), h).cpu().numpy()
    pad_a = torch.zeros((n2, n1 + 1), device=dev())
    pad_a[:, :n1] = torch.from_numpy(A.T)
    c_unal = cms.sketch_product(pad_a[:, :n1].T, rowmajor(B), h).cpu().numpy()
    c_gen = cms.sketch_product(colmajor(A, torch.float64), rowmajor(B, torch.float64), h).cpu().numpy()
    ref = O.sketch_definition(A.astype(np.float64), B.astype(np.float64), O.make_tables(12, 512, b, d))
    assert O.rel_l2(c_fast, ref) < TOL_F32
    assert O.rel_l2(c_unal, ref) < TOL_F32
    assert O.rel_l2(c_gen, ref) < TOL_F32
    h.free()


@pytest.mark.parametrize("n1,n2,n3,b,d,dtype", [
    (301, 37, 299, 3840, 2, torch.float32),    # odd row lengths, C = 960
    (301, 37, 299, 3840, 2, torch.bfloat16),
    (675, 29, 675, 10800, 2, torch.float32),   # X^T X with odd n (aliased), C = 900
])
def test_fast_kernel_unaligned_rows(cms, n1, n2, n3, b, d, dtype):
    n = max(n1, n3)
    h = cms.make_hashes(5 + b, n, b, d)
    tab = O.make_tables(5 + b, n, b, d)
    if n1 == n3:
        X = W.gaussian(n2, n1, 9).astype(np.float32)
        Xr = W.bf16_round(X)[0] if dtype == torch.bfloat16 else X
        xt = torch.from_numpy(X).to(dev(), dtype)
        c = cms.sketch_product(xt.T, xt, h).cpu().numpy()
        ref = O.sketch_definition(Xr.T.astype(np.float64), Xr.astype(np.float64), tab)
    else:
        A = W.gaussian(n1, n2, 7).astype(np.float32)
        B = W.gaussian(n2, n3, 8).astype(np.float32)
        Ar = W.bf16_round(A)[0] if dtype == torch.bfloat16 else A
        Br = W.bf16_round(B)[0] if dtype == torch.bfloat16 else B
        c = cms.sketch_product(colmajor(A, dtype), rowmajor(B, dtype), h).cpu().numpy()
        ref = O.sketch_definition(Ar.astype(np.float64), Br.astype(np.float64), tab)
    assert O.rel_l2(c, ref) < TOL_F32
    h.free()


def test_reseeded_fast_path(cms):
    # reseed rebuilds the front-end records on the device
    X = W.gaussian(96, 1024, 8).astype(np.float32)
    h = cms.make_hashes(1, 1024, 65536, 2)
    xt = torch.from_numpy(X).to(dev())
    h.reseed(99)
    c = cms.sketch_product(xt.T, xt, h).cpu().numpy()
    ref = O.sketch_definition(X.T.astype(np.float64), X.astype(np.float64), O.make_tables(99, 1024, 65536, 2))
    assert O.rel_l2(c, ref) < TOL_F32
    h.free()


def test_workspace_query_covers_aliased_operands(cms):
    # n = 2304: with A = X^T and B = X the same bytes the fast kernel stages
    # each row once and fits in shared memory, while the two-operand form
    # does not; a workspace of exactly cms_workspace_size() must serve both
    m, n, b, d = 40, 2304, 32768, 2
    X = W.gaussian(m, n, 21).astype(np.float32)
    h = cms.make_hashes(5, n, b, d)
    xt = torch.from_numpy(X).to(dev())
    ws = cms.alloc_workspace(cms.workspace_size(h, n, m, n))
    c = cms.sketch_product(xt.T, xt, h, ws=ws).cpu().numpy()
    ref = O.sketch_definition(X.T.astype(np.float64), X.astype(np.float64), O.make_tables(5, n, b, d))
    assert O.rel_l2(c, ref) < TOL_F32
    h.free()


# --------------------------------------------- large hash domain (BF16) ----
def test_large_domain_bf16_reduced_inner(cms):
    # the large covariance shape (n = 32768 variables, b = 2^20, d = 7, BF16
    # storage) with the inner dimension cut to 48 samples so the oracle and
    # the test stay fast: checked on sampled buckets and the DC identity
    m, n, b, d = 48, 32768, 1 << 20, 7
    cov = W.covariance(m, n, 64, 0.3, seed=5, dtype=np.float32)
    Xb, _ = W.bf16_round(cov.X)
    X = torch.from_numpy(cov.X).to(dev(), torch.bfloat16)
    h = cms.make_hashes(5, n, b, d)
    c = cms.sketch_product(X.T, X, h).cpu().numpy().astype(np.float64)
    tab = O.make_tables(5, n, b, d)
    Xd = Xb.astype(np.float64)
    zs = W.rng(55).choice(b, 64, replace=False)
    for t in range(d):
        want = O.sketch_bucket_values(Xd.T, Xd, tab, t, zs)
        assert np.linalg.norm(c[t, zs] - want) / np.linalg.norm(want) < TOL_F32, t
        dc = (tab.s1[t] @ Xd.T) @ (Xd @ tab.s2[t])
        assert abs(c[t].sum() - dc) < 1e-5 * np.abs(c[t]).sum()
    h.free()


# ------------------------------------- records in tensor memory (large n) ----
@pytest.mark.parametrize("n1,n2,n3,b,d,dtype,alias", [
    (6000, 24, 6000, 96000, 2, torch.float32, True),     # C = 960
    (4096, 20, 4096, 65536, 3, torch.bfloat16, True),    # C = 1024, BF16 (not the FP32-only warp-specialised kernel)
    (5000, 17, 4400, 80000, 2, torch.float32, False),    # C = 800, two operands
])
def test_lockstep_kernel_with_tensor_memory_records(cms, n1, n2, n3, b, d, dtype, alias):
    n = max(n1, n3)
    h = cms.make_hashes(60 + d, n, b, d)
    tab = O.make_tables(60 + d, n, b, d)
    if alias:
        X = W.gaussian(n2, n1, 61).astype(np.float32)
        Xr = W.bf16_round(X)[0] if dtype == torch.bfloat16 else X
        xt = torch.from_numpy(X).to(dev(), dtype)
        A, B = xt.T, xt
        Ad, Bd = Xr.T.astype(np.float64), Xr.astype(np.float64)
    else:
        Ah = W.gaussian(n1, n2, 62).astype(np.float32)
        Bh = W.gaussian(n2, n3, 63).astype(np.float32)
        A, B = colmajor(Ah, dtype), rowmajor(Bh, dtype)
        Ad, Bd = Ah.astype(np.float64), Bh.astype(np.float64)
    assert cms.plan_kernel(A, B, h) == "lockstep_tmem"
    c = cms.sketch_product(A, B, h).cpu().numpy().astype(np.float64)
    cms.check_async()
    zs = W.rng(64).choice(b, 64, replace=False)
    for t in range(d):
        want = O.sketch_bucket_values(Ad, Bd, tab, t, zs)
        assert np.linalg.norm(c[t, zs] - want) / np.linalg.norm(want) < TOL_F32, t
        dc = (tab.s1[t][:n1] @ Ad) @ (Bd @ tab.s2[t][:n3])
        assert abs(c[t].sum() - dc) < 1e-5 * np.abs(c[t]).sum()
    h.free()


@pytest.mark.parametrize("n,b,C", [(12288, 16384, 1024), (10800, 13824, 864)])
def test_lockstep_kernel_long_overflow_lists(cms, n, b, C):
    # 12 to 12.5 entries per bucket class on average (a drawn hash): nearly
    # every bucket holds more than the 8 recorded entries, so every bucket
    # group walks overflow lists of several entries per lane, with twiddles
    # formed on the fly (C = 1024, and C = 864 with items of 27 buckets);
    # the sketch is also bit-identical across two calls
    m, d = 12, 2
    X = W.gaussian(m, n, 71).astype(np.float32)
    Xr = W.bf16_round(X)[0]
    xt = torch.from_numpy(X).to(dev(), torch.bfloat16)
    h = cms.make_hashes(72, n, b, d)
    assert cms.plan_kernel(xt.T, xt, h) == "lockstep_tmem"
    tab = O.make_tables(72, n, b, d)
    assert h.info()["C"] == C
    counts = np.bincount(tab.h1[0] % C, minlength=C)
    assert (counts > 8).mean() > 0.9 and counts.max() - 8 >= 4
    c1 = cms.sketch_product(xt.T, xt, h)
    c2 = cms.sketch_product(xt.T, xt, h)
    cms.check_async()
    assert torch.equal(c1, c2)
    c = c1.cpu().numpy().astype(np.float64)
    Xd = Xr.astype(np.float64)
    zs = W.rng(73).choice(b, 64, replace=False)
    for t in range(d):
        want = O.sketch_bucket_values(Xd.T, Xd, tab, t, zs)
        assert np.linalg.norm(c[t, zs] - want) / np.linalg.norm(want) < TOL_F32, t
        dc = (tab.s1[t] @ Xd.T) @ (Xd @ tab.s2[t])
        assert abs(c[t].sum() - dc) < 1e-5 * np.abs(c[t]).sum()
    h.free()


def test_warp_specialised_kernel_both_spectrum_swaps(cms, monkeypatch):
    # the partner FFT warps swap half spectra through tensor memory; blocks
    # whose front-end records leave no room take the shared-memory swap
    # (forced here by the library's debug switch); both give the oracle's
    # sketch, at an inner dimension that crosses several Kahan folds
    m, n, b, d = 4096, 2048, 65536, 3
    X = W.gaussian(m, n, 17).astype(np.float32)
    xt = torch.from_numpy(X).to(dev())
    h = cms.make_hashes(23, n, b, d)
    assert cms.plan_kernel(xt.T, xt, h) == "warp_specialised"
    tab = O.make_tables(23, n, b, d)
    Xd = X.astype(np.float64)
    ref = O.sketch_definition(Xd.T, Xd, tab)
    c_tm = cms.sketch_product(xt.T, xt, h).cpu().numpy()
    monkeypatch.setenv("CMS_WS_SMEM_SWAP", "1")
    c_sm = cms.sketch_product(xt.T, xt, h).cpu().numpy()
    monkeypatch.delenv("CMS_WS_SMEM_SWAP")
    cms.check_async()
    for c in (c_tm, c_sm):
        assert max(O.rel_l2(c[t], ref[t]) for t in range(d)) < TOL_F32
    h.free()
