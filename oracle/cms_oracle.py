"""FP64 CPU oracle for compressed matrix multiplication (Pagh, "Compressed
Matrix Multiplication", arXiv 1108.1320).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (no kernels, headers, helpers, tables or
constants); the hash definition and its seeding are implemented here a second
time, independently, from their published definitions.

Everything is float64 (numpy) unless stated.  Indices are 0-based: the paper
writes [n] = {1..n} and "for z := 1 to b" in Fig. 1 but maps into {0..b-1}
in Sec. 2.2; we use 0-based row, column, inner and bucket indices and feed the
0-based index to the hash polynomial.

What each function follows:

* ``splitmix64`` / ``draw_coefficients`` - seeding of the hash family.  The
  paper does not say how hash functions are drawn; we use splitmix64 (Steele,
  Lea, Flood, OOPSLA 2014) and draw, for t = 0..d-1, the (a, c) pairs of
  h1, s1, h2, s2 in that order, a = 1 + (r mod (p-1)), c = r mod p.
* ``hash_bucket`` / ``hash_sign`` - the degree-1 polynomial family of Sec. 2.2
  and the paper's reference [13]: h(x) = ((a x + c) mod p) mod b with
  p = 2^31 - 1; the sign function (unspecified in Sec. 2.1) is the same family
  with range 2, mapped to {+1, -1}.
* ``sketch_fft`` - COMPRESSEDPRODUCT of Fig. 1: per repetition t and inner
  index k, count-sketch column k of A with (h1, s1) and row k of B with
  (h2, s2), FFT both, multiply pointwise, accumulate over k, and apply one
  inverse FFT (Sec. 2.2, the identity p*_{uv}(w^t) = p*_t).  The second
  scatter in Fig. 1 writes ``pa[h_2(j)] := pb[h_2(j)] + ...``; it is read as
  ``pb[h_2(j)] := pb[h_2(j)] + s_2(j) B_kj``.
* ``sketch_definition`` - the same sketch from its definition (Sec. 2.2,
  polynomial p*_{uv}; abstract: c = (p mod x^b) + (p div x^b)): the count
  sketch of AB under the decomposed splitting function
  h(i,j) = (h1(i) + h2(j)) mod b and sign s(i,j) = s1(i) s2(j).
* ``sketch_convolution`` - the same sketch as an explicit length-b cyclic
  convolution summed over k (Sec. 2.2, polynomial multiplication), with no
  FFT: the "2-D sketch" M = sum_k pa_k pb_k^T folded along wrapped
  anti-diagonals.
* ``sketch_bucket_values`` - c_t[z] for a few buckets z straight from the
  definition, one bucket at a time (for full-size spot checks).
* ``sketch_bucket_values_rows`` - the same values for many buckets at once,
  from A's rows and B's columns given as contiguous row arrays (the rows of
  X^T for the covariance use), each (AB)_ij a float64 dot product.
* ``decompress`` / ``decompress_dense`` - DECOMPRESS of Fig. 1:
  X_t = s1_t(i) s2_t(j) c_t[(h1_t(i) + h2_t(j)) mod b], median over t.  The
  median of an even number of values is the mean of the two middle ones.

* ``product_diagonal`` / ``remove_diagonal`` / ``candidates`` - the
  covariance post-steps of Sec. 3.2 and Fig. 2: the diagonal of AB, the
  sketch of AB with its diagonal's contribution removed, and the entries
  whose estimate exceeds a threshold.

* ``draw_sign4_coefficients`` / ``sign4`` / ``ams_frobenius`` /
  ``frobenius_bound`` - Sec. 5.2: AMS sketches X = (s1^T A)(B s2) of AB
  with 4-wise independent signs and the bound 32 median X^2 on ||AB||_F^2.

* ``nnz_doubling`` - Sec. 5.1: the doubling search over b that stops when
  at most b/5 buckets are nonzero for every repetition.

* ``code_bits`` / ``decode_code`` / ``masked_sketches`` /
  ``significant_from_sketches`` / ``find_significant`` - Sec. 4, Fig. 3
  (FINDSIGNIFICANTENTRIES) with a balanced repetition code in place of the
  expander code the paper leaves undefined.

Every function here is pinned by tests under ``-m "not gpu"`` against facts
that do not come from this module (published splitmix64 outputs, hand-worked
hash values, the three independent sketch routes, the injective-hash and b=1
special cases, the AMS identity of Sec. 2.1, Theorem 2's mean and variance,
Theorem 5's exact recovery).
"""
from __future__ import annotations

import numpy as np

P31 = (1 << 31) - 1          # the Mersenne prime p = 2^31 - 1 of the hash family
_MASK64 = (1 << 64) - 1
_GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_MIX1 = 0xBF58476D1CE4E5B9
_MIX2 = 0x94D049BB133111EB

HASH_NAMES = ("h1", "s1", "h2", "s2")


# --------------------------------------------------------------------------
# Seeding: splitmix64 (Steele, Lea, Flood 2014), plain Python integers.
# --------------------------------------------------------------------------
def splitmix64(state: int) -> tuple[int, int]:
    """One splitmix64 step: returns (next_state, output)."""
    state = (state + _GOLDEN_GAMMA) & _MASK64
    z = state
    z = ((z ^ (z >> 30)) * _MIX1) & _MASK64
    z = ((z ^ (z >> 27)) * _MIX2) & _MASK64
    return state, z ^ (z >> 31)


def draw_coefficients(seed: int, d: int) -> np.ndarray:
    """Coefficients (a, c) of h1, s1, h2, s2 for each repetition t.

    Returns an int64 array of shape (d, 4, 2): [t][function][a or c], the
    functions in the order h1, s1, h2, s2.
    """
    out = np.zeros((d, 4, 2), dtype=np.int64)
    state = seed & _MASK64
    for t in range(d):
        for f in range(4):
            state, r = splitmix64(state)
            out[t, f, 0] = 1 + r % (P31 - 1)
            state, r = splitmix64(state)
            out[t, f, 1] = r % P31
    return out


# --------------------------------------------------------------------------
# Hash family of Sec. 2.2 / [13]: h(x) = ((a x + c) mod p) mod b.
# --------------------------------------------------------------------------
def hash_bucket(a: int, c: int, x: np.ndarray, b: int) -> np.ndarray:
    """Splitting function value in {0..b-1} for 0-based indices x."""
    x = np.asarray(x, dtype=np.uint64)
    v = (np.uint64(a) * x + np.uint64(c)) % np.uint64(P31)
    return (v % np.uint64(b)).astype(np.int64)


def hash_sign(a: int, c: int, x: np.ndarray) -> np.ndarray:
    """Sign function value in {+1, -1}: 1 - 2 * (((a x + c) mod p) mod 2)."""
    x = np.asarray(x, dtype=np.uint64)
    v = (np.uint64(a) * x + np.uint64(c)) % np.uint64(P31)
    return (1 - 2 * (v % np.uint64(2)).astype(np.int64)).astype(np.int64)


class Tables:
    """Hash tables of d repetitions over the domain {0..n-1}.

    h1[t], s1[t] index rows of A (the i of A_ik); h2[t], s2[t] index columns
    of B (the j of B_kj).  Shapes (d, n), int64.
    """

    def __init__(self, h1, s1, h2, s2, b: int):
        self.h1 = np.asarray(h1, dtype=np.int64)
        self.s1 = np.asarray(s1, dtype=np.int64)
        self.h2 = np.asarray(h2, dtype=np.int64)
        self.s2 = np.asarray(s2, dtype=np.int64)
        self.b = int(b)
        self.d = self.h1.shape[0]

    def rep(self, t: int) -> "Tables":
        return Tables(self.h1[t:t + 1], self.s1[t:t + 1], self.h2[t:t + 1],
                      self.s2[t:t + 1], self.b)


def make_tables(seed: int, n: int, b: int, d: int) -> Tables:
    """Fig. 1's per-repetition draws of s1, s2, h1, h2, as tables over {0..n-1}."""
    coef = draw_coefficients(seed, d)
    x = np.arange(n, dtype=np.int64)
    h1 = np.stack([hash_bucket(coef[t, 0, 0], coef[t, 0, 1], x, b) for t in range(d)])
    s1 = np.stack([hash_sign(coef[t, 1, 0], coef[t, 1, 1], x) for t in range(d)])
    h2 = np.stack([hash_bucket(coef[t, 2, 0], coef[t, 2, 1], x, b) for t in range(d)])
    s2 = np.stack([hash_sign(coef[t, 3, 0], coef[t, 3, 1], x) for t in range(d)])
    return Tables(h1, s1, h2, s2, b)


# --------------------------------------------------------------------------
# COMPRESSEDPRODUCT, Fig. 1: sketch -> FFT -> pointwise product -> sum over k
# -> one inverse FFT.
# --------------------------------------------------------------------------
def count_sketch(u: np.ndarray, h: np.ndarray, s: np.ndarray, b: int) -> np.ndarray:
    """Coefficients of p_u^{h,s}(x) = sum_i s(i) u_i x^{h(i)} (Sec. 2.2)."""
    return np.bincount(h, weights=s * np.asarray(u, dtype=np.float64), minlength=b)


def sketch_fft(A: np.ndarray, B: np.ndarray, tab: Tables, return_imag: bool = False):
    """COMPRESSEDPRODUCT(A, B, b, d) of Fig. 1, in float64.

    A is n1 x n2, B is n2 x n3 (any memory order).  Returns c of shape (d, b):
    c[t] = FFT^{-1}( sum_k FFT(pa_k) * FFT(pb_k) ), the real part (the sketch
    of a real matrix is real; with ``return_imag`` the largest |imag| is also
    returned as a consistency check).
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    n1, n2 = A.shape
    n2b, n3 = B.shape
    assert n2 == n2b
    b = tab.b
    c = np.zeros((tab.d, b), dtype=np.float64)
    max_imag = 0.0
    for t in range(tab.d):
        h1, s1 = tab.h1[t, :n1], tab.s1[t, :n1]
        h2, s2 = tab.h2[t, :n3], tab.s2[t, :n3]
        p = np.zeros(b, dtype=np.complex128)
        for k in range(n2):
            pa = count_sketch(A[:, k], h1, s1, b)       # column k of A
            pb = count_sketch(B[k, :], h2, s2, b)       # row k of B
            p += np.fft.fft(pa) * np.fft.fft(pb)        # p[t][z] += pa[z] pb[z]
        q = np.fft.ifft(p)                              # p[t] := FFT^{-1}(p[t])
        c[t] = q.real
        max_imag = max(max_imag, float(np.max(np.abs(q.imag))) if b else 0.0)
    return (c, max_imag) if return_imag else c


def sketch_definition(A: np.ndarray, B: np.ndarray, tab: Tables) -> np.ndarray:
    """Count sketch of AB from its definition (Sec. 2.2).

    c_t[z] = sum over (i, j) with (h1(i) + h2(j)) mod b = z of
    s1(i) s2(j) (AB)_ij, with AB formed in float64.
    """
    AB = np.asarray(A, dtype=np.float64) @ np.asarray(B, dtype=np.float64)
    n1, n3 = AB.shape
    b = tab.b
    c = np.zeros((tab.d, b), dtype=np.float64)
    for t in range(tab.d):
        z = (tab.h1[t, :n1, None] + tab.h2[t, None, :n3]) % b
        w = (tab.s1[t, :n1, None] * tab.s2[t, None, :n3]) * AB
        c[t] = np.bincount(z.ravel(), weights=w.ravel(), minlength=b)
    return c


def sketch_convolution(A: np.ndarray, B: np.ndarray, tab: Tables) -> np.ndarray:
    """Sketch as a direct length-b cyclic convolution summed over k (no FFT).

    With PA[x, k] = pa_k[x] and PB[k, y] = pb_k[y], M = PA PB holds
    sum_k pa_k[x] pb_k[y]; c[z] = sum_x M[x, (z - x) mod b].  This is
    (p mod x^b) + (p div x^b) for p = sum_k p_{a_k} p_{b_k} (abstract, Sec. 2.2).
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    n1, n2 = A.shape
    n3 = B.shape[1]
    b = tab.b
    c = np.zeros((tab.d, b), dtype=np.float64)
    xs = np.arange(b)
    for t in range(tab.d):
        PA = np.zeros((b, n2))
        np.add.at(PA, tab.h1[t, :n1], tab.s1[t, :n1, None] * A)
        PB = np.zeros((n2, b))
        np.add.at(PB.T, tab.h2[t, :n3], tab.s2[t, :n3, None] * B.T)
        M = PA @ PB
        for z in range(b):
            c[t, z] = M[xs, (z - xs) % b].sum()
    return c


def sketch_bucket_values(A: np.ndarray, B: np.ndarray, tab: Tables, t: int,
                         zs: np.ndarray) -> np.ndarray:
    """c_t[z] for the listed buckets z only, straight from the definition.

    For each z, every pair (i, j) with (h1(i) + h2(j)) mod b = z contributes
    s1(i) s2(j) sum_k A_ik B_kj.  Cost ~ (n1 n3 / b) n2 per bucket, so this
    works at full problem size on a sample of buckets.
    """
    A = np.asarray(A)
    B = np.asarray(B)
    n1 = A.shape[0]
    n3 = B.shape[1]
    b = tab.b
    h1, s1 = tab.h1[t, :n1], tab.s1[t, :n1]
    h2, s2 = tab.h2[t, :n3], tab.s2[t, :n3]
    order = np.argsort(h2, kind="stable")
    h2_sorted = h2[order]
    out = np.zeros(len(zs), dtype=np.float64)
    for q, z in enumerate(np.asarray(zs, dtype=np.int64)):
        need = (z - h1) % b                      # h2(j) each i needs
        lo = np.searchsorted(h2_sorted, need, side="left")
        hi = np.searchsorted(h2_sorted, need, side="right")
        counts = hi - lo
        ii = np.repeat(np.arange(n1), counts)
        if len(ii) == 0:
            continue
        # positions lo[i] .. hi[i]-1 of the sorted h2 table, for every i
        starts = np.repeat(lo, counts)
        within = np.arange(len(ii)) - np.repeat(np.cumsum(counts) - counts, counts)
        jj = order[starts + within]
        ab = np.einsum("pk,kp->p", A[ii, :].astype(np.float64), B[:, jj].astype(np.float64))
        out[q] = np.sum(s1[ii] * s2[jj] * ab)
    return out


def sketch_bucket_values_rows(A_rows: np.ndarray, B_cols: np.ndarray, tab: Tables, t: int,
                              zs: np.ndarray, chunk: int = 1024) -> np.ndarray:
    """c_t[z] for the listed buckets z straight from the definition (Sec. 2.2).

    ``A_rows[i]`` is row i of A (n1 x n2) and ``B_cols[j]`` is column j of B
    (n2 x n3), both as C-contiguous row arrays of any float dtype.  Every pair
    (i, j) with (h1(i) + h2(j)) mod b = z contributes s1(i) s2(j) (AB)_ij,
    where (AB)_ij = sum_k A_ik B_kj is accumulated in float64.  The pairs of
    all listed buckets are collected first and their dot products formed in
    chunks, so that thousands of buckets of a large product cost one pass over
    the needed rows.
    """
    n1 = A_rows.shape[0]
    n3 = B_cols.shape[0]
    b = tab.b
    zs = np.asarray(zs, dtype=np.int64)
    h1, s1 = tab.h1[t, :n1].astype(np.int64), tab.s1[t, :n1].astype(np.float64)
    h2, s2 = tab.h2[t, :n3].astype(np.int64), tab.s2[t, :n3].astype(np.float64)
    order = np.argsort(h2, kind="stable")
    h2_sorted = h2[order]
    ii_all, jj_all, qq_all = [], [], []
    for q, z in enumerate(zs):
        need = (z - h1) % b                      # the h2(j) that row i needs
        lo = np.searchsorted(h2_sorted, need, side="left")
        hi = np.searchsorted(h2_sorted, need, side="right")
        counts = hi - lo
        ii = np.repeat(np.arange(n1), counts)
        if len(ii) == 0:
            continue
        starts = np.repeat(lo, counts)
        within = np.arange(len(ii)) - np.repeat(np.cumsum(counts) - counts, counts)
        ii_all.append(ii)
        jj_all.append(order[starts + within])
        qq_all.append(np.full(len(ii), q, dtype=np.int64))
    out = np.zeros(len(zs), dtype=np.float64)
    if not ii_all:
        return out
    ii = np.concatenate(ii_all)
    jj = np.concatenate(jj_all)
    qq = np.concatenate(qq_all)
    for p0 in range(0, len(ii), chunk):
        i_c, j_c = ii[p0:p0 + chunk], jj[p0:p0 + chunk]
        ab = np.einsum("pk,pk->p", A_rows[i_c], B_cols[j_c], dtype=np.float64, casting="safe")
        np.add.at(out, qq[p0:p0 + chunk], s1[i_c] * s2[j_c] * ab)
    return out


# --------------------------------------------------------------------------
# DECOMPRESS, Fig. 1.
# --------------------------------------------------------------------------
def median(values: np.ndarray, axis: int = 0) -> np.ndarray:
    """Median over ``axis``; an even count takes the mean of the two middle values."""
    return np.median(values, axis=axis)


def estimates(c: np.ndarray, tab: Tables, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    """X_t = s1_t(i) s2_t(j) c_t[(h1_t(i) + h2_t(j)) mod b], shape (d, len(i))."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    X = np.empty((tab.d, len(i)), dtype=np.float64)
    for t in range(tab.d):
        z = (tab.h1[t, i] + tab.h2[t, j]) % tab.b
        X[t] = tab.s1[t, i] * tab.s2[t, j] * np.asarray(c[t], dtype=np.float64)[z]
    return X


def decompress(c: np.ndarray, tab: Tables, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    """DECOMPRESS(i, j) for a list of pairs: median over t of X_t."""
    return median(estimates(c, tab, i, j), axis=0)


def decompress_dense(c: np.ndarray, tab: Tables, n1: int, n3: int) -> np.ndarray:
    """All n1 x n3 estimates (Sec. 2.2, O(n^2) decoding of every entry)."""
    ii, jj = np.meshgrid(np.arange(n1), np.arange(n3), indexing="ij")
    return decompress(c, tab, ii.ravel(), jj.ravel()).reshape(n1, n3)


# --------------------------------------------------------------------------
# Error metric used for parity: relative L2 per repetition, max over t.
# --------------------------------------------------------------------------
def rel_l2(x: np.ndarray, ref: np.ndarray) -> float:
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    ref = np.atleast_2d(np.asarray(ref, dtype=np.float64))
    num = np.linalg.norm(x - ref, axis=-1)
    den = np.maximum(np.linalg.norm(ref, axis=-1), np.finfo(np.float64).tiny)
    return float(np.max(num / den))


# --------------------------------------------------------------------------
# Sparse inputs (Sec. 2.2 "sparse or rectangular"; Theorem 5): A given by
# columns (CSC), B given by rows (CSR).  Exact for integer-valued data.
# --------------------------------------------------------------------------
def sketch_definition_sparse(A_csc, B_csr, tab: Tables) -> np.ndarray:
    """Definition route for sparse A (CSC) and B (CSR) as scipy matrices.

    AB is formed with a sparse product; for integer-valued inputs every
    bucket is an exact integer (float64 sums of integers below 2^53).
    """
    AB = (A_csc @ B_csr).tocoo()
    b = tab.b
    c = np.zeros((tab.d, b), dtype=np.float64)
    i = AB.row.astype(np.int64)
    j = AB.col.astype(np.int64)
    v = AB.data.astype(np.float64)
    for t in range(tab.d):
        z = (tab.h1[t, i] + tab.h2[t, j]) % b
        c[t] = np.bincount(z, weights=tab.s1[t, i] * tab.s2[t, j] * v, minlength=b)
    return c


def sketch_fft_sparse(A_csc, B_csr, tab: Tables) -> np.ndarray:
    """Fig. 1 on sparse inputs: only inner indices k with a nonzero a_k and b_k
    contribute (Sec. 2.2, time O(N + n2 b lg b) per repetition)."""
    A_csc = A_csc.tocsc()
    B_csr = B_csr.tocsr()
    n2 = A_csc.shape[1]
    b = tab.b
    c = np.zeros((tab.d, b), dtype=np.float64)
    for t in range(tab.d):
        p = np.zeros(b, dtype=np.complex128)
        for k in range(n2):
            a0, a1 = A_csc.indptr[k], A_csc.indptr[k + 1]
            b0, b1 = B_csr.indptr[k], B_csr.indptr[k + 1]
            if a0 == a1 or b0 == b1:
                continue
            ia = A_csc.indices[a0:a1]
            jb = B_csr.indices[b0:b1]
            pa = count_sketch(A_csc.data[a0:a1], tab.h1[t, ia], tab.s1[t, ia], b)
            pb = count_sketch(B_csr.data[b0:b1], tab.h2[t, jb], tab.s2[t, jb], b)
            p += np.fft.fft(pa) * np.fft.fft(pb)
        c[t] = np.fft.ifft(p).real
    return c


# --------------------------------------------------------------------------
# Covariance post-steps (Sec. 3.2, Fig. 2).  A linear sketch of Q gives one
# of Q~ (Q with its diagonal set to zero) by removing each diagonal entry's
# contribution from its bucket; the decoded estimates of Q~ are then
# thresholded into a short list of candidates for large entries.
# --------------------------------------------------------------------------
def product_diagonal(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """(AB)_ii = sum_k A_ik B_ki for i < min(n1, n3), in float64."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    m = min(A.shape[0], B.shape[1])
    return np.einsum("ik,ki->i", A[:m], B[:, :m])


def remove_diagonal(c: np.ndarray, diag: np.ndarray, tab: Tables) -> np.ndarray:
    """Sketch of AB without its diagonal: for every i and repetition t,
    s1_t(i) s2_t(i) diag_i leaves bucket (h1_t(i) + h2_t(i)) mod b (the
    entry (i, i) enters the sketch there with that sign, Sec. 2.2)."""
    out = np.array(c, dtype=np.float64, copy=True)
    i = np.arange(len(diag))
    for t in range(tab.d):
        z = (tab.h1[t, i] + tab.h2[t, i]) % tab.b
        np.subtract.at(out[t], z, tab.s1[t, i] * tab.s2[t, i] * np.asarray(diag, dtype=np.float64))
    return out


def candidates(c: np.ndarray, tab: Tables, n1: int, n3: int, tau: float,
               skip_diagonal: bool = True) -> np.ndarray:
    """Row-major (i, j) pairs whose estimate DECOMPRESS(i, j) exceeds tau in
    absolute value (Fig. 2: thresholding the approximation), shape (q, 2).

    The estimates decide set membership, so they are formed in float32, the
    precision of the sketch c: X_t = s1 s2 c_t[...] (sign changes are exact),
    the middle value for odd d, 0.5 (a + b) of the two middle values in
    float32 for even d; the comparison |estimate| > tau is made in float32.
    """
    c32 = np.asarray(c, dtype=np.float32)
    ii, jj = np.meshgrid(np.arange(n1), np.arange(n3), indexing="ij")
    ii = ii.ravel()
    jj = jj.ravel()
    X = np.empty((tab.d, len(ii)), dtype=np.float32)
    for t in range(tab.d):
        z = (tab.h1[t, ii] + tab.h2[t, jj]) % tab.b
        X[t] = c32[t][z] * (tab.s1[t, ii] * tab.s2[t, jj]).astype(np.float32)
    X.sort(axis=0)
    mid = tab.d // 2
    if tab.d % 2:
        est = X[mid]
    else:
        est = np.float32(0.5) * (X[mid - 1] + X[mid])
    keep = np.abs(est) > np.float32(tau)
    if skip_diagonal:
        keep &= ii != jj
    return np.stack([ii[keep], jj[keep]], axis=1).astype(np.int64)


# --------------------------------------------------------------------------
# Sec. 5.2: an upper bound on ||AB||_F / sqrt(b) from AMS sketches of AB.
# X = sum_ij s1(i) s2(j) (AB)_ij = (s1^T A)(B s2) (Sec. 2.1: the AMS sketch
# of AB is the sum of those of its outer products); with 4-wise independent
# s1, s2, X^2 is an unbiased estimate of ||AB||_F^2 with variance at most
# 8 E[X^2]^2, so 32 times the median of d values of X^2 bounds ||AB||_F^2
# from above with high probability.  The 4-wise independent signs are
# degree-3 polynomials over Z_p, p = 2^31 - 1, reduced mod 2 (the same
# mapping to {+1, -1} as the 2-wise signs; the paper names no family).
# --------------------------------------------------------------------------
def draw_sign4_coefficients(seed: int, d: int) -> np.ndarray:
    """Coefficients (a0, a1, a2, a3) of s1 and s2 for each repetition t, drawn
    with splitmix64 in the order t, function (s1, s2), a0..a3, each r mod p.
    Shape (d, 2, 4), int64."""
    out = np.zeros((d, 2, 4), dtype=np.int64)
    state = seed & _MASK64
    for t in range(d):
        for f in range(2):
            for q in range(4):
                state, r = splitmix64(state)
                out[t, f, q] = r % P31
    return out


def sign4(coef: np.ndarray, x: np.ndarray) -> np.ndarray:
    """1 - 2 (((a3 x^3 + a2 x^2 + a1 x + a0) mod p) mod 2) for 0-based x,
    with Python integers (exact)."""
    a0, a1, a2, a3 = (int(v) for v in coef)
    out = np.empty(len(x), dtype=np.int64)
    for q, xv in enumerate(np.asarray(x, dtype=np.int64).tolist()):
        v = (((a3 * xv + a2) * xv + a1) * xv + a0) % P31
        out[q] = 1 - 2 * (v % 2)
    return out


def ams_frobenius(A: np.ndarray, B: np.ndarray, seed: int, d: int) -> np.ndarray:
    """X_t = (s1_t^T A)(B s2_t) for t = 0..d-1, float64."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    coef = draw_sign4_coefficients(seed, d)
    X = np.empty(d, dtype=np.float64)
    for t in range(d):
        s1 = sign4(coef[t, 0], np.arange(A.shape[0]))
        s2 = sign4(coef[t, 1], np.arange(B.shape[1]))
        X[t] = (s1 @ A) @ (B @ s2)
    return X


def frobenius_bound(X: np.ndarray) -> float:
    """32 times the median of the X_t^2: a bound on ||AB||_F^2 (Sec. 5.2)."""
    return 32.0 * float(median(np.asarray(X, dtype=np.float64) ** 2))


# --------------------------------------------------------------------------
# Sec. 5.1: the doubling search for the number of nonzero entries of AB.
# Sketches of AB are taken with b = 2, 4, 8, ... until at most b/5 buckets
# are nonzero for every one of the d splitting functions; random diagonal
# scalings of A and B (Schwartz-Zippel) make a bucket zero only when every
# entry of AB hashed to it is zero, so the test is on the bucket pattern of
# the nonzero entries of AB.  The splitting functions of size b are those of
# Fig. 1 drawn from `seed` (the same (a, c) for every b).
# --------------------------------------------------------------------------
def nnz_doubling(rows: np.ndarray, cols: np.ndarray, seed: int, d: int, b_max: int) -> tuple[int, int]:
    """(b, distinct) for the nonzero entries (rows[q], cols[q]) of AB: the
    first b = 2^r <= b_max at which every repetition has at most b/5 distinct
    buckets (h1(i) + h2(j)) mod b, and the largest of those counts; (-1, 0)
    when b_max is reached first."""
    coef = draw_coefficients(seed, d)
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    b = 2
    while b <= b_max:
        worst = 0
        for t in range(d):
            z = (hash_bucket(coef[t, 0, 0], coef[t, 0, 1], rows, b) +
                 hash_bucket(coef[t, 2, 0], coef[t, 2, 1], cols, b)) % b
            worst = max(worst, len(np.unique(z)))
        if 5 * worst <= b:
            return b, worst
        b *= 2
    return -1, 0


# --------------------------------------------------------------------------
# Sec. 4, Fig. 3: FINDSIGNIFICANTENTRIES.  2 l sketches with the same hash
# functions of the masked products (I_{E_r} A) B (r < l) and A (B I_{E_r})
# (r >= l), where E : [n] -> {0, 1}^l is an error-correcting code; for every
# repetition t and bucket k the bits X_r > Delta/2 of X_r = |p^(t,r)[k]| are
# decoded into a position (i, j); positions inserted for at least d/2 of
# the (t, k) are returned.  The paper asks for an expander code and defines
# none; here E is a balanced repetition code: for each of the L bits of x
# (L = ceil(log2 max(n1, n3)), least significant first) rho copies of the
# bit and rho copies of its complement, l = 2 rho L.  DECODE takes a
# majority vote per bit (ties rejected) and rejects a string farther than
# l/4 from the decoded codeword (so the all-zero string of an empty bucket
# decodes to nothing).
# --------------------------------------------------------------------------
def code_length(n1: int, n3: int, rho: int) -> tuple[int, int]:
    """(L, l): bits per index and code length."""
    L = max(1, int(np.ceil(np.log2(max(n1, n3, 2)))))
    return L, 2 * rho * L


def code_bits(x: int, L: int, rho: int) -> np.ndarray:
    """E(x) as a 0/1 array of length 2 rho L."""
    out = np.zeros(2 * rho * L, dtype=np.int64)
    for q in range(L):
        bit = (int(x) >> q) & 1
        out[q * 2 * rho: q * 2 * rho + rho] = bit
        out[q * 2 * rho + rho: (q + 1) * 2 * rho] = 1 - bit
    return out


def decode_code(s: np.ndarray, L: int, rho: int) -> int:
    """x with E(x) closest to s by per-bit majority, or -1 (a tie, or the
    string farther than l/4 from E(x))."""
    s = np.asarray(s, dtype=np.int64)
    x = 0
    dist = 0
    for q in range(L):
        seg = s[q * 2 * rho: (q + 1) * 2 * rho]
        votes = int(seg[:rho].sum() + (rho - seg[rho:].sum()))
        if 2 * votes == 2 * rho:
            return -1
        bit = 1 if votes > rho else 0
        x |= bit << q
        dist += (2 * rho - votes) if bit else votes
    return x if 4 * dist <= 2 * rho * L else -1


def masked_sketches(A: np.ndarray, B: np.ndarray, tab: Tables, rho: int) -> np.ndarray:
    """The 2 l sketches of (3), shape (2 l, d, b), by the definition route."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    n1, n3 = A.shape[0], B.shape[1]
    L, ell = code_length(n1, n3, rho)
    Ei = np.stack([code_bits(i, L, rho) for i in range(n1)])      # (n1, l)
    Ej = np.stack([code_bits(j, L, rho) for j in range(n3)])      # (n3, l)
    out = np.empty((2 * ell, tab.d, tab.b))
    for r in range(ell):
        out[r] = sketch_definition(A * Ei[:, r:r + 1], B, tab)
        out[ell + r] = sketch_definition(A, B * Ej[:, r][None, :], tab)
    return out


def significant_from_sketches(P: np.ndarray, n1: int, n3: int, delta: float, rho: int) -> np.ndarray:
    """Fig. 3 on given sketches P (2 l, d, b): the positions inserted for at
    least d/2 of the (t, k), sorted, shape (q, 2).  The bits X_r > Delta/2
    are decided in float32 (the precision of the sketches)."""
    L, ell = code_length(n1, n3, rho)
    P32 = np.abs(np.asarray(P, dtype=np.float32))
    _, d, b = P32.shape
    counts: dict = {}
    for t in range(d):
        bits = (P32[:, t, :] > np.float32(delta) / np.float32(2)).astype(np.int64)   # (2 l, b)
        for k in np.nonzero(bits.any(axis=0))[0]:
            i = decode_code(bits[:ell, k], L, rho)
            j = decode_code(bits[ell:, k], L, rho)
            if 0 <= i < n1 and 0 <= j < n3:
                counts[(i, j)] = counts.get((i, j), 0) + 1
    keep = sorted(p for p, c in counts.items() if 2 * c >= d)
    return np.array(keep, dtype=np.int64).reshape(-1, 2)


def find_significant(A: np.ndarray, B: np.ndarray, tab: Tables, delta: float, rho: int) -> np.ndarray:
    """FINDSIGNIFICANTENTRIES(Delta) of Fig. 3 from the masked sketches."""
    A = np.asarray(A)
    B = np.asarray(B)
    return significant_from_sketches(masked_sketches(A, B, tab, rho), A.shape[0], B.shape[1], delta, rho)
