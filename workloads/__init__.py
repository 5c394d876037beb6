"""Seeded synthetic inputs for compressed matrix multiplication.

This module only draws data: it holds none of the method's arithmetic (no
hashing, sketching, FFT or decoding), so that both the FP64 oracle's tests and
the CUDA path's tests and benchmark can use it without sharing any code with
each other.  All draws use numpy's PCG64 generator, which gives the same
stream on x86-64 and AArch64.

Workload shapes follow the paper's uses of the method:

* dense i.i.d. N(0, 1) factors (Sec. 3.1, the Frobenius-norm guarantee);
* sample-covariance inputs (Sec. 3.2, Fig. 2): X is m samples x n variables,
  A = X^T and B = X, mostly independent variables plus planted correlated
  pairs (u, v) with X_v = rho X_u + sqrt(1 - rho^2) Z;
* sparse factors whose product is sparse (Sec. 3.3.1, Theorem 5): disjoint
  blocks, each joining a few inner indices to a set of rows of A and columns
  of B, integer values in [-8, 8] without 0;
* batches of covariance-shaped instances of uneven size, n log-uniform and
  rounded to a 5-smooth integer (2^a 3^b 5^c).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian(rows: int, cols: int, seed: int, dtype=np.float64) -> np.ndarray:
    """rows x cols i.i.d. N(0, 1), C (row-major) order."""
    return rng(seed).standard_normal((rows, cols)).astype(dtype, copy=False)


def uniform_pm1(rows: int, cols: int, seed: int, dtype=np.float64) -> np.ndarray:
    """rows x cols i.i.d. uniform on [-1, 1] (the Fig. 2 demonstration data)."""
    return rng(seed).uniform(-1.0, 1.0, (rows, cols)).astype(dtype, copy=False)


@dataclass
class Covariance:
    """X (m x n, row-major) and its planted correlated variable pairs."""
    X: np.ndarray
    pairs: np.ndarray          # (n_pairs, 2) int64: (u, v), u != v
    rho: float


def covariance(m: int, n: int, n_pairs: int, rho: float, seed: int,
               dtype=np.float32, chunk_rows: int = 4096) -> Covariance:
    """m samples of n variables, N(0, 1), with ``n_pairs`` disjoint planted pairs.

    The pairs are disjoint: a seeded permutation of the variables is cut into
    consecutive (u, v) couples.  Column v is replaced by
    rho * X_u + sqrt(1 - rho^2) * Z with fresh N(0, 1) noise Z, so corr = rho.
    Rows are drawn in chunks (each chunk its own derived stream) to bound the
    float64 temporaries for large m x n.
    """
    assert 2 * n_pairs <= n
    g = rng(seed)
    perm = g.permutation(n)
    pairs = perm[: 2 * n_pairs].reshape(n_pairs, 2).astype(np.int64)
    X = np.empty((m, n), dtype=dtype)
    s = math.sqrt(max(0.0, 1.0 - rho * rho))
    for r0 in range(0, m, chunk_rows):
        r1 = min(m, r0 + chunk_rows)
        gc = rng(seed * 1_000_003 + 7919 * (r0 // chunk_rows + 1))
        blk = gc.standard_normal((r1 - r0, n))
        if n_pairs:
            z = gc.standard_normal((r1 - r0, n_pairs))
            blk[:, pairs[:, 1]] = rho * blk[:, pairs[:, 0]] + s * z
        X[r0:r1] = blk.astype(dtype, copy=False)
    return Covariance(X=X, pairs=pairs, rho=rho)


@dataclass
class SparseBlocks:
    """Block-sparse A (n1 x n2, CSC) and B (n2 x n3, CSR) with sparse AB."""
    n: int
    a_colptr: np.ndarray       # int64 (n2 + 1)
    a_rowidx: np.ndarray       # int64
    a_val: np.ndarray          # float32 integer values
    b_rowptr: np.ndarray       # int64 (n2 + 1)
    b_colidx: np.ndarray       # int64
    b_val: np.ndarray          # float32 integer values
    blocks: list = field(default_factory=list)   # (inner, rows, cols) per block

    def scipy(self):
        import scipy.sparse as sp
        A = sp.csc_matrix((self.a_val.astype(np.float64), self.a_rowidx, self.a_colptr),
                          shape=(self.n, self.n))
        B = sp.csr_matrix((self.b_val.astype(np.float64), self.b_colidx, self.b_rowptr),
                          shape=(self.n, self.n))
        return A, B


def _nonzero_ints(g: np.random.Generator, size) -> np.ndarray:
    """Integers uniform on [-8, 8] without 0."""
    v = g.integers(1, 9, size=size)
    sgn = g.integers(0, 2, size=size) * 2 - 1
    return (v * sgn).astype(np.float32)


def sparse_blocks(n: int, n_blocks: int, inner: int, rows: int, cols: int,
                  seed: int) -> SparseBlocks:
    """Disjoint blocks: block q joins ``inner`` inner indices with ``rows``
    rows of A and ``cols`` columns of B (all index sets seeded and disjoint).

    A[rows_q, inner_q] and B[inner_q, cols_q] are dense with values in
    [-8, 8] \\ {0}, so AB has at most n_blocks * rows * cols nonzeros.
    """
    assert n_blocks * inner <= n and n_blocks * rows <= n and n_blocks * cols <= n
    g = rng(seed)
    ks = g.permutation(n)[: n_blocks * inner].reshape(n_blocks, inner)
    rs = g.permutation(n)[: n_blocks * rows].reshape(n_blocks, rows)
    cs = g.permutation(n)[: n_blocks * cols].reshape(n_blocks, cols)
    a_cols = {}
    b_rows = {}
    blocks = []
    for q in range(n_blocks):
        rows_q = np.sort(rs[q])
        cols_q = np.sort(cs[q])
        for k in ks[q]:
            a_cols[int(k)] = (rows_q, _nonzero_ints(g, rows))
            b_rows[int(k)] = (cols_q, _nonzero_ints(g, cols))
        blocks.append((np.sort(ks[q]), rows_q, cols_q))
    a_colptr = np.zeros(n + 1, dtype=np.int64)
    b_rowptr = np.zeros(n + 1, dtype=np.int64)
    for k, (r, _) in a_cols.items():
        a_colptr[k + 1] = len(r)
    for k, (c, _) in b_rows.items():
        b_rowptr[k + 1] = len(c)
    a_colptr = np.cumsum(a_colptr)
    b_rowptr = np.cumsum(b_rowptr)
    a_rowidx = np.zeros(a_colptr[-1], dtype=np.int64)
    a_val = np.zeros(a_colptr[-1], dtype=np.float32)
    b_colidx = np.zeros(b_rowptr[-1], dtype=np.int64)
    b_val = np.zeros(b_rowptr[-1], dtype=np.float32)
    for k, (r, v) in a_cols.items():
        a_rowidx[a_colptr[k]:a_colptr[k + 1]] = r
        a_val[a_colptr[k]:a_colptr[k + 1]] = v
    for k, (c, v) in b_rows.items():
        b_colidx[b_rowptr[k]:b_rowptr[k + 1]] = c
        b_val[b_rowptr[k]:b_rowptr[k + 1]] = v
    return SparseBlocks(n, a_colptr, a_rowidx, a_val, b_rowptr, b_colidx, b_val, blocks)


def five_smooth_near(x: float) -> int:
    """The 5-smooth integer (2^a 3^b 5^c) closest to x in log scale."""
    best, best_d = 1, float("inf")
    lx = math.log(x)
    for a in range(0, 40):
        for b3 in range(0, 26):
            for c5 in range(0, 18):
                v = (2 ** a) * (3 ** b3) * (5 ** c5)
                if v > 4 * x:
                    break
                dist = abs(math.log(v) - lx)
                if dist < best_d:
                    best, best_d = v, dist
    return best


@dataclass
class BatchSpec:
    n: int
    m: int
    dtype: str                 # "f32" or "bf16"
    seed: int
    n_pairs: int
    rho: float


def batched_specs(count: int, seed: int, n_lo: int = 512, n_hi: int = 8192,
                  rho: float = 0.5) -> list[BatchSpec]:
    """Uneven covariance-shaped instances: n log-uniform in [n_lo, n_hi],
    rounded to 5-smooth, m = 2n, floor(0.01 n) planted pairs, first half FP32
    and second half BF16 storage, instance q seeded with seed + q."""
    g = rng(seed)
    out = []
    for q in range(count):
        n = five_smooth_near(math.exp(g.uniform(math.log(n_lo), math.log(n_hi))))
        n = min(max(n, n_lo), n_hi)
        out.append(BatchSpec(n=n, m=2 * n, dtype="f32" if q < count // 2 else "bf16",
                             seed=seed + q, n_pairs=n // 100, rho=rho))
    return out


def sample_pairs(n1: int, n3: int, q: int, seed: int) -> np.ndarray:
    """q index pairs (i, j), uniform with replacement, shape (q, 2) int64."""
    g = rng(seed)
    return np.stack([g.integers(0, n1, q), g.integers(0, n3, q)], axis=1).astype(np.int64)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float32 holding the bf16 value exactly, and the raw uint16 bits."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)
    back = (r.astype(np.uint32) << 16).view(np.float32)
    return back, r
