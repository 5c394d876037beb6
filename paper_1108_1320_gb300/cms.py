"""Python binding of libcms (the C ABI in include/cms.h).

Argument marshalling only: every step of the compressed product runs in the
library's CUDA kernels.  PyTorch provides device memory and streams.  If
libcms.so is missing, every call raises: there is no fallback path.

Names mirror the C entry points without the ``cms_`` prefix.  Matrices are
torch tensors: A (n1 x n2) must be column-major (``A.stride(0) == 1``, e.g.
``X.T`` of a contiguous X), B (n2 x n3) row-major (``B.stride(1) == 1``), so
that column k of A and row k of B are contiguous (Sec. 2.2, single pass).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcms.so")

CMS_OK = 0
STATUS = {0: "CMS_OK", 1: "CMS_ERR_INVALID_ARG", 2: "CMS_ERR_UNSUPPORTED", 3: "CMS_ERR_CUDA",
          4: "CMS_ERR_WORKSPACE", 5: "CMS_ERR_TIMEOUT", 6: "CMS_ERR_DEVICE"}
CMS_F32, CMS_BF16, CMS_F64 = 0, 1, 2
_DTYPES = {torch.float32: CMS_F32, torch.bfloat16: CMS_BF16, torch.float64: CMS_F64}

# Every symbol the header declares, with (restype, argtypes).
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_U64 = ctypes.c_uint64
_SZ = ctypes.c_size_t
SIGNATURES = {
    "cms_make_hashes": (_I32, [_U64, _I64, _I64, _I32, ctypes.POINTER(_P)]),
    "cms_reseed_hashes": (_I32, [_P, _U64, _P]),
    "cms_make_hashes_from_tables": (_I32, [_I64, _I64, _I32, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "cms_free_hashes": (_I32, [_P]),
    "cms_hashes_info": (_I32, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I32),
                               ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "cms_hashes_coeffs": (_I32, [_P, _I32, _P]),
    "cms_hashes_tables": (_I32, [_P, _P, _P, _P, _P]),
    "cms_hashes_buckets": (_I32, [_P, _I32, _I32, _P, _P]),
    "cms_workspace_size": (_I32, [_P, _I64, _I64, _I64, _I32, ctypes.POINTER(_SZ)]),
    "cms_sketch_product": (_I32, [_P, _I64, _P, _I64, _I64, _I64, _I64, _I32, _P, _P, _P, _SZ, _P]),
    "cms_sketch_product_noalloc": (_I32, [_P, _I64, _P, _I64, _I64, _I64, _I64, _I32, _P, _P, _P]),
    "cms_sparse_workspace_size": (_I32, [_P, _I64, _I64, _I64, ctypes.POINTER(_SZ)]),
    "cms_sketch_product_csr": (_I32, [_P, _P, _P, _P, _P, _P, _I64, _I64, _I64, _I32, _P, _P, _P, _SZ,
                                      _P]),
    "cms_frobenius_workspace_size": (_I32, [_I64, _I64, _I64, _I32, ctypes.POINTER(_SZ)]),
    "cms_frobenius_estimate": (_I32, [_P, _I64, _P, _I64, _I64, _I64, _I64, _I32, ctypes.c_uint64, _I32, _P, _P,
                                      _P, _SZ, _P]),
    "cms_nnz_workspace_size": (_I32, [_I32, _I64, ctypes.POINTER(_SZ)]),
    "cms_nnz_estimate": (_I32, [_P, _P, _P, _P, _P, _P, _I64, _I64, _I64, _I32, ctypes.c_uint64, _I32, _I64,
                                ctypes.POINTER(_I64), ctypes.POINTER(_I64), _P, _SZ, _P]),
    "cms_significant_workspace_size": (_I32, [_P, _I64, _I64, _I64, _I32, _I32, ctypes.POINTER(_SZ)]),
    "cms_find_significant": (_I32, [_P, _I64, _P, _I64, _I64, _I64, _I64, _I32, _P, ctypes.c_float, _I32, _P, _I64,
                                    _P, _P, _SZ, _P]),
    "cms_significant_decode_workspace_size": (_I32, [_P, ctypes.POINTER(_SZ)]),
    "cms_decode_significant": (_I32, [_P, _P, _I64, _I64, ctypes.c_float, _I32, _P, _I64, _P, _P, _SZ, _P]),
    "cms_plan_kernel": (_I32, [_P, _I64, _P, _I64, _I64, _I64, _I64, _I32, _P, ctypes.POINTER(_I32)]),
    "cms_sketch_remove_diagonal": (_I32, [_P, _I64, _P, _I64, _I64, _I64, _I64, _I32, _P, _P, _P]),
    "cms_decode_threshold": (_I32, [_P, _P, _I64, _I64, ctypes.c_float, _I32, _P, _P, _I64, _P, _P, _SZ, _P]),
    "cms_sketch_product_csr_hybrid": (_I32, [_P, _P, _P, _P, _P, _P, _I64, _I64, _I64, _I32, _P, _I64, _P, _P,
                                             _SZ, _P]),
    "cms_batch_create": (_I32, [_P, _I32, _I32, ctypes.c_char_p, _P, ctypes.POINTER(_P)]),
    "cms_batch_run": (_I32, [_P, _P]),
    "cms_batch_run_graph": (_I32, [_P, _P]),
    "cms_batch_info": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                              ctypes.POINTER(_SZ), ctypes.POINTER(_I32)]),
    "cms_batch_free": (_I32, [_P]),
    "cms_plain_workspace_size": (_I32, [_P, _I64, _I64, _I64, ctypes.POINTER(_SZ)]),
    "cms_sketch_product_plain_f64": (_I32, [_P, _I64, _P, _I64, _I64, _I64, _I64, _P, _P, _P, _SZ,
                                            _P]),
    "cms_decode": (_I32, [_P, _P, _P, _I64, _P, _P]),
    "cms_decode_f64": (_I32, [_P, _P, _P, _I64, _P, _P]),
    "cms_decode_dense": (_I32, [_P, _P, _I64, _I64, _P, _I64, _P]),
    "cms_merge": (_I32, [_P, _I32, _I32, _I64, _P, _P]),
    "cms_check_async": (_I32, [_P]),
    "cms_selftest_wait": (_I32, [_P]),
    "cms_profile_enable": (_I32, [_I32]),
    "cms_profile_summary": (_I32, [_P, _SZ, ctypes.POINTER(_SZ)]),
    "cms_status_string": (ctypes.c_char_p, [_I32]),
    "cms_last_error": (ctypes.c_char_p, []),
}

_lib = None


class CmsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load libcms.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1108_1320_gb300.build` (no fallback exists)")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _check(status: int):
    if status != CMS_OK:
        raise CmsError(status, lib().cms_last_error().decode(errors="replace"))


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


class Hashes:
    """d repetitions of (h1, s1, h2, s2) over {0..n-1} into {0..b-1} (Fig. 1)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    @classmethod
    def make(cls, seed: int, n: int, b: int, d: int) -> "Hashes":
        out = ctypes.c_void_p()
        _check(lib().cms_make_hashes(seed & ((1 << 64) - 1), n, b, d, ctypes.byref(out)))
        return cls(out.value)

    @classmethod
    def from_tables(cls, h1, s1, h2, s2, b: int) -> "Hashes":
        h1 = np.ascontiguousarray(h1, dtype=np.uint32)
        h2 = np.ascontiguousarray(h2, dtype=np.uint32)
        s1 = np.ascontiguousarray(s1, dtype=np.int8)
        s2 = np.ascontiguousarray(s2, dtype=np.int8)
        d, n = h1.shape
        out = ctypes.c_void_p()
        _check(lib().cms_make_hashes_from_tables(n, b, d, h1.ctypes.data, s1.ctypes.data,
                                                 h2.ctypes.data, s2.ctypes.data, ctypes.byref(out)))
        return cls(out.value)

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise ValueError("hashes already freed")
        return self._h

    def reseed(self, seed: int, stream=None):
        _check(lib().cms_reseed_hashes(self.handle, seed & ((1 << 64) - 1), _stream(stream)))

    def info(self) -> dict:
        n, b, R, C = _I64(), _I64(), _I64(), _I64()
        d = _I32()
        _check(lib().cms_hashes_info(self.handle, ctypes.byref(n), ctypes.byref(b), ctypes.byref(d),
                                     ctypes.byref(R), ctypes.byref(C)))
        return {"n": n.value, "b": b.value, "d": d.value, "R": R.value, "C": C.value}

    def coeffs(self, t: int) -> np.ndarray:
        out = np.zeros(8, dtype=np.uint32)
        _check(lib().cms_hashes_coeffs(self.handle, t, out.ctypes.data))
        return out

    def tables(self):
        inf = self.info()
        d, n = inf["d"], inf["n"]
        h1 = np.zeros((d, n), np.uint32)
        h2 = np.zeros((d, n), np.uint32)
        s1 = np.zeros((d, n), np.int8)
        s2 = np.zeros((d, n), np.int8)
        _check(lib().cms_hashes_tables(self.handle, h1.ctypes.data, s1.ctypes.data, h2.ctypes.data,
                                       s2.ctypes.data))
        return h1, s1, h2, s2

    def buckets(self, t: int, side: int):
        """(perm uint32 [n], off uint32 [C + 1]): the indices of repetition t,
        side 0 (rows of A) or 1 (columns of B), stably sorted by bucket mod C."""
        inf = self.info()
        perm = np.zeros(inf["n"], np.uint32)
        off = np.zeros(max(inf["C"], 0) + 1, np.uint32)
        _check(lib().cms_hashes_buckets(self.handle, t, side, perm.ctypes.data, off.ctypes.data))
        return perm, off

    def free(self):
        if self._h:
            lib().cms_free_hashes(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def make_hashes(seed: int, n: int, b: int, d: int) -> Hashes:
    return Hashes.make(seed, n, b, d)


def _check_buf(t, name: str, device, dtype=None, numel: int = 0) -> None:
    """A caller-supplied device buffer: the library only sees its pointer, so
    its device, dtype, layout and size are checked here."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda or t.device != torch.device(device):
        raise ValueError(f"{name} must be a CUDA tensor on {device}")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, {numel} are needed")


def _sketch_out(c, h: "Hashes", device, dtype=torch.float32):
    inf = h.info()
    if c is None:
        return torch.empty((inf["d"], inf["b"]), dtype=dtype, device=device)
    _check_buf(c, "c", device, dtype, inf["d"] * inf["b"])
    return c


def _ab_args(A: torch.Tensor, B: torch.Tensor):
    if A.dim() != 2 or B.dim() != 2:
        raise ValueError("A and B must be 2-D")
    n1, n2 = A.shape
    n2b, n3 = B.shape
    if n2 != n2b:
        raise ValueError(f"inner dimensions differ: {n2} vs {n2b}")
    if A.dtype != B.dtype or A.dtype not in _DTYPES:
        raise ValueError("A and B must share a dtype in {float32, bfloat16, float64}")
    if not (A.is_cuda and B.is_cuda) or A.device != B.device:
        raise ValueError("A and B must be CUDA tensors on one device")
    if n1 > 1 and A.stride(0) != 1:
        raise ValueError("A must be column-major (A.stride(0) == 1), e.g. X.T")
    if n3 > 1 and B.stride(1) != 1:
        raise ValueError("B must be row-major (B.stride(1) == 1)")
    lda = A.stride(1) if n2 > 1 else max(n1, 1)
    ldb = B.stride(0) if n2 > 1 else max(n3, 1)
    return n1, n2, n3, lda, ldb


def workspace_size(h: Hashes, n1: int, n2: int, n3: int, dtype=torch.float32) -> int:
    out = _SZ()
    _check(lib().cms_workspace_size(h.handle, n1, n2, n3, _DTYPES[dtype], ctypes.byref(out)))
    return out.value


def alloc_workspace(nbytes: int, device=None) -> torch.Tensor:
    """A 256-byte aligned device buffer (torch's caching allocator aligns to 512)."""
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device or "cuda")


def sketch_product(A: torch.Tensor, B: torch.Tensor, h: Hashes, c: torch.Tensor | None = None,
                   ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """COMPRESSEDPRODUCT (Fig. 1): returns c, float32 of shape (d, b)."""
    n1, n2, n3, lda, ldb = _ab_args(A, B)
    c = _sketch_out(c, h, A.device)
    need = workspace_size(h, n1, n2, n3, A.dtype)
    if ws is None:
        ws = alloc_workspace(need, A.device)
    _check_buf(ws, "ws", A.device)
    _check(lib().cms_sketch_product(_ptr(A), lda, _ptr(B), ldb, n1, n2, n3, _DTYPES[A.dtype], h.handle,
                                    _ptr(c), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))
    return c


KERNEL_NAMES = {0: "shared_memory", 1: "lockstep", 2: "lockstep_tmem", 3: "warp_specialised", 4: "cluster"}


def plan_kernel(A: torch.Tensor, B: torch.Tensor, h: Hashes) -> str:
    """The fused kernel sketch_product(A, B, h) would run (see KERNEL_NAMES)."""
    n1, n2, n3, lda, ldb = _ab_args(A, B)
    out = _I32()
    _check(lib().cms_plan_kernel(_ptr(A), lda, _ptr(B), ldb, n1, n2, n3, _DTYPES[A.dtype], h.handle,
                                 ctypes.byref(out)))
    return KERNEL_NAMES[out.value]


def sketch_product_noalloc(A: torch.Tensor, B: torch.Tensor, h: Hashes,
                           c: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """COMPRESSEDPRODUCT without a workspace, for callers that cannot
    allocate device memory: the library's fixed 32 MiB scratch array is used
    (shared by all calls on the device; calls overlapping on the GPU race).
    Returns c, float32 (d, b)."""
    n1, n2, n3, lda, ldb = _ab_args(A, B)
    c = _sketch_out(c, h, A.device)
    _check(lib().cms_sketch_product_noalloc(_ptr(A), lda, _ptr(B), ldb, n1, n2, n3, _DTYPES[A.dtype],
                                            h.handle, _ptr(c), _stream(stream)))
    return c


def sparse_workspace_size(h: Hashes, n1: int, n2: int, n3: int) -> int:
    out = _SZ()
    _check(lib().cms_sparse_workspace_size(h.handle, n1, n2, n3, ctypes.byref(out)))
    return out.value


def sketch_product_csr(a_colptr: torch.Tensor, a_rowidx: torch.Tensor, a_val: torch.Tensor,
                       b_rowptr: torch.Tensor, b_colidx: torch.Tensor, b_val: torch.Tensor,
                       n1: int, n3: int, h: Hashes, c: torch.Tensor | None = None,
                       ws: torch.Tensor | None = None, stream=None,
                       direct_max_pairs: int | None = None) -> torch.Tensor:
    """COMPRESSEDPRODUCT of sparse A (CSC: colptr int64, rowidx int32) and B
    (CSR: rowptr int64, colidx int32); returns c float32 (d, b).

    ``direct_max_pairs`` selects the sparse-k hybrid (cms_sketch_product_csr_hybrid):
    inner indices with at most that many outer-product terms are sketched
    directly (-1: the library's default split); None keeps every inner index
    on the FFT route."""
    n2 = a_colptr.numel() - 1
    if b_rowptr.numel() - 1 != n2:
        raise ValueError("A and B disagree on the inner dimension")
    for t_, dt_ in ((a_colptr, torch.int64), (b_rowptr, torch.int64), (a_rowidx, torch.int32),
                    (b_colidx, torch.int32)):
        if t_.dtype != dt_ or not t_.is_cuda or not t_.is_contiguous():
            raise ValueError("pointer arrays must be contiguous CUDA int64, index arrays int32")
    if a_val.dtype != b_val.dtype or a_val.dtype not in _DTYPES:
        raise ValueError("values must share a dtype in {float32, bfloat16, float64}")
    dev = a_colptr.device
    for t_, nm in ((a_rowidx, "a_rowidx"), (b_rowptr, "b_rowptr"), (b_colidx, "b_colidx"), (a_val, "a_val"),
                   (b_val, "b_val")):
        _check_buf(t_, nm, dev)
    c = _sketch_out(c, h, dev)
    if ws is None:
        ws = alloc_workspace(sparse_workspace_size(h, n1, n2, n3), dev)
    _check_buf(ws, "ws", dev)
    if direct_max_pairs is None:
        _check(lib().cms_sketch_product_csr(_ptr(a_colptr), _ptr(a_rowidx), _ptr(a_val), _ptr(b_rowptr),
                                            _ptr(b_colidx), _ptr(b_val), n1, n2, n3, _DTYPES[a_val.dtype],
                                            h.handle, _ptr(c), _ptr(ws), ws.numel() * ws.element_size(),
                                            _stream(stream)))
    else:
        _check(lib().cms_sketch_product_csr_hybrid(_ptr(a_colptr), _ptr(a_rowidx), _ptr(a_val), _ptr(b_rowptr),
                                                   _ptr(b_colidx), _ptr(b_val), n1, n2, n3, _DTYPES[a_val.dtype],
                                                   h.handle, int(direct_max_pairs), _ptr(c), _ptr(ws),
                                                   ws.numel() * ws.element_size(), _stream(stream)))
    return c


class _Instance(ctypes.Structure):
    _fields_ = [("A", _P), ("lda", _I64), ("B", _P), ("ldb", _I64), ("n1", _I64), ("n2", _I64),
                ("n3", _I64), ("dt", _I32), ("reserved", _I32), ("h", _P), ("c", _P)]


class Batch:
    """Many products (A_q, B_q, hashes_q) -> c_q in one persistent launch.

    ``items`` is a list of (A, B, hashes) with A column-major and B row-major
    device tensors; outputs are allocated here (``self.c[q]``, float32 (d, b)).
    The tensors must stay alive and in place while the batch exists."""

    def __init__(self, items, autotune: bool = False, tune_cache: str | None = None, stream=None):
        self._keep = []
        self.c = []
        arr = (_Instance * len(items))()
        for q, (A, B, h) in enumerate(items):
            n1, n2, n3, lda, ldb = _ab_args(A, B)
            inf = h.info()
            c = torch.empty((inf["d"], inf["b"]), dtype=torch.float32, device=A.device)
            self.c.append(c)
            self._keep += [A, B, h]
            arr[q] = _Instance(_ptr(A), lda, _ptr(B), ldb, n1, n2, n3, _DTYPES[A.dtype], 0,
                               h.handle.value, _ptr(c))
        out = ctypes.c_void_p()
        _check(lib().cms_batch_create(arr, len(items), 1 if autotune else 0,
                                      tune_cache.encode() if tune_cache else None, _stream(stream),
                                      ctypes.byref(out)))
        self._b = out

    def run(self, stream=None):
        _check(lib().cms_batch_run(self._b, _stream(stream)))
        return self.c

    def run_graph(self, stream):
        _check(lib().cms_batch_run_graph(self._b, _stream(stream)))
        return self.c

    def info(self) -> dict:
        inst, tasks, launches, fast = _I32(), _I32(), _I32(), _I32()
        ws = _SZ()
        _check(lib().cms_batch_info(self._b, ctypes.byref(inst), ctypes.byref(tasks),
                                    ctypes.byref(launches), ctypes.byref(ws), ctypes.byref(fast)))
        return {"instances": inst.value, "tasks": tasks.value, "launches": launches.value,
                "ws_bytes": ws.value, "fast_instances": fast.value}

    def free(self):
        if self._b:
            lib().cms_batch_free(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def plain_workspace_size(h: Hashes, n1: int, n2: int, n3: int) -> int:
    out = _SZ()
    _check(lib().cms_plain_workspace_size(h.handle, n1, n2, n3, ctypes.byref(out)))
    return out.value


def sketch_product_plain_f64(A: torch.Tensor, B: torch.Tensor, h: Hashes,
                             c: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                             stream=None) -> torch.Tensor:
    """The plain FP64 form of the same sketch: returns c, float64 (d, b)."""
    n1, n2, n3, lda, ldb = _ab_args(A, B)
    if A.dtype != torch.float64:
        raise ValueError("the plain path takes float64 A and B")
    c = _sketch_out(c, h, A.device, torch.float64)
    if ws is None:
        ws = alloc_workspace(plain_workspace_size(h, n1, n2, n3), A.device)
    _check_buf(ws, "ws", A.device)
    _check(lib().cms_sketch_product_plain_f64(_ptr(A), lda, _ptr(B), ldb, n1, n2, n3, h.handle,
                                              _ptr(c), _ptr(ws), ws.numel() * ws.element_size(),
                                              _stream(stream)))
    return c


def decode(c: torch.Tensor, h: Hashes, ij: torch.Tensor, out: torch.Tensor | None = None,
           stream=None) -> torch.Tensor:
    """DECOMPRESS (Fig. 1) of q index pairs ij (int64, shape (q, 2))."""
    ij = ij.contiguous()
    if ij.dtype != torch.int64 or ij.dim() != 2 or ij.shape[1] != 2:
        raise ValueError("ij must be int64 of shape (q, 2)")
    q = ij.shape[0]
    c = c.contiguous()
    if c.dtype not in (torch.float32, torch.float64):
        raise ValueError("c must be float32 or float64")
    inf = h.info()
    _check_buf(c, "c", c.device, c.dtype, inf["d"] * inf["b"])
    _check_buf(ij, "ij", c.device)
    if out is None:
        out = torch.empty(q, dtype=c.dtype, device=c.device)
    _check_buf(out, "out", c.device, c.dtype, q)
    if c.dtype == torch.float64:
        _check(lib().cms_decode_f64(_ptr(c), h.handle, _ptr(ij), q, _ptr(out), _stream(stream)))
    elif c.dtype == torch.float32:
        _check(lib().cms_decode(_ptr(c), h.handle, _ptr(ij), q, _ptr(out), _stream(stream)))
    else:
        raise ValueError("c must be float32 or float64")
    return out


def decode_dense(c: torch.Tensor, h: Hashes, n1: int, n3: int, out: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """All n1 x n3 estimates, row-major float32."""
    c = c.contiguous()
    inf = h.info()
    _check_buf(c, "c", c.device, torch.float32, inf["d"] * inf["b"])
    if out is None:
        out = torch.empty((n1, n3), dtype=torch.float32, device=c.device)
    if (not isinstance(out, torch.Tensor) or not out.is_cuda or out.device != c.device
            or out.dtype != torch.float32 or out.dim() != 2 or tuple(out.shape) != (n1, n3)
            or (n3 > 1 and out.stride(1) != 1)):
        raise ValueError("out must be a float32 CUDA tensor of shape (n1, n3) with unit column stride, on c's device")
    _check(lib().cms_decode_dense(_ptr(c), h.handle, n1, n3, _ptr(out), out.stride(0) if n1 else n3,
                                  _stream(stream)))
    return out


def remove_diagonal(A: torch.Tensor, B: torch.Tensor, h: Hashes, c: torch.Tensor, stream=None) -> torch.Tensor:
    """Sec. 3.2: turn the sketch c of AB (in place) into the sketch of AB with
    its diagonal set to zero; A, B as for sketch_product."""
    n1, n2, n3, lda, ldb = _ab_args(A, B)
    inf = h.info()
    _check_buf(c, "c", A.device, torch.float32, inf["d"] * inf["b"])
    _check(lib().cms_sketch_remove_diagonal(_ptr(A), lda, _ptr(B), ldb, n1, n2, n3, _DTYPES[A.dtype], h.handle,
                                            _ptr(c), _stream(stream)))
    return c


def decode_threshold(c: torch.Tensor, h: Hashes, n1: int, n3: int, tau: float, skip_diagonal: bool = True,
                     capacity: int = 1 << 16, stream=None):
    """Fig. 2's thresholding: (ij int64 (q, 2), estimates float32 (q,), count)
    for every (i, j) with |estimate| > tau in row-major order; when count
    exceeds capacity only the first capacity hits are returned."""
    dev = c.device
    c = c.contiguous()
    inf = h.info()
    _check_buf(c, "c", dev, torch.float32, inf["d"] * inf["b"])
    ij = torch.empty((max(capacity, 1), 2), dtype=torch.int64, device=dev)
    val = torch.empty(max(capacity, 1), dtype=torch.float32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = torch.empty(n1 + 1, dtype=torch.int64, device=dev)
    _check(lib().cms_decode_threshold(_ptr(c), h.handle, n1, n3, float(tau), 1 if skip_diagonal else 0,
                                      _ptr(ij), _ptr(val), capacity, _ptr(cnt), _ptr(ws), ws.numel() * 8,
                                      _stream(stream)))
    q = int(cnt.item())
    k = min(q, capacity)
    return ij[:k], val[:k], q


def _sorted_positions(ij: torch.Tensor, count: torch.Tensor, capacity: int):
    q = int(count.item())
    out = ij[:min(q, capacity)]
    if out.shape[0] > 1:
        order = torch.argsort(out[:, 0] * (int(out[:, 1].max()) + 1) + out[:, 1])
        out = out[order]
    return out, q


def find_significant(A: torch.Tensor, B: torch.Tensor, h: Hashes, delta: float, rho: int = 1,
                     capacity: int = 1 << 16, stream=None):
    """FINDSIGNIFICANTENTRIES (Sec. 4, Fig. 3): positions (q, 2) int64, sorted
    row-major, and their count (which may exceed capacity)."""
    n1, n2, n3, lda, ldb = _ab_args(A, B)
    need = _SZ()
    _check(lib().cms_significant_workspace_size(h.handle, n1, n2, n3, _DTYPES[A.dtype], rho, ctypes.byref(need)))
    ws = alloc_workspace(need.value, A.device)
    ij = torch.empty((max(capacity, 1), 2), dtype=torch.int64, device=A.device)
    cnt = torch.zeros(1, dtype=torch.int64, device=A.device)
    _check(lib().cms_find_significant(_ptr(A), lda, _ptr(B), ldb, n1, n2, n3, _DTYPES[A.dtype], h.handle,
                                      float(delta), rho, _ptr(ij), capacity, _ptr(cnt), _ptr(ws),
                                      ws.numel() * ws.element_size(), _stream(stream)))
    return _sorted_positions(ij, cnt, capacity)


def decode_significant(sketches: torch.Tensor, h: Hashes, n1: int, n3: int, delta: float, rho: int = 1,
                       capacity: int = 1 << 16, stream=None):
    """Fig. 3's decode and vote on given sketches (float32 (2 l, d, b))."""
    sketches = sketches.contiguous()
    inf = h.info()
    if sketches.dim() != 3 or tuple(sketches.shape[1:]) != (inf["d"], inf["b"]) or sketches.shape[0] % 2:
        raise ValueError("sketches must have shape (2 l, d, b)")
    _check_buf(sketches, "sketches", sketches.device, torch.float32)
    need = _SZ()
    _check(lib().cms_significant_decode_workspace_size(h.handle, ctypes.byref(need)))
    ws = alloc_workspace(need.value, sketches.device)
    ij = torch.empty((max(capacity, 1), 2), dtype=torch.int64, device=sketches.device)
    cnt = torch.zeros(1, dtype=torch.int64, device=sketches.device)
    _check(lib().cms_decode_significant(_ptr(sketches), h.handle, n1, n3, float(delta), rho, _ptr(ij),
                                        capacity, _ptr(cnt), _ptr(ws), ws.numel() * ws.element_size(),
                                        _stream(stream)))
    return _sorted_positions(ij, cnt, capacity)


def nnz_estimate(a_colptr: torch.Tensor, a_rowidx: torch.Tensor, a_val: torch.Tensor,
                 b_rowptr: torch.Tensor, b_colidx: torch.Tensor, b_val: torch.Tensor, n1: int, n3: int,
                 seed: int, d: int, b_max: int = 1 << 24, stream=None):
    """Sec. 5.1 doubling search: (b, buckets) with b the first power of two at
    which every repetition has at most b/5 nonzero buckets (-1 if b_max was
    passed), buckets the largest such count."""
    n2 = a_colptr.numel() - 1
    need = _SZ()
    _check(lib().cms_nnz_workspace_size(d, b_max, ctypes.byref(need)))
    ws = alloc_workspace(need.value, a_colptr.device)
    b_out = _I64()
    k_out = _I64()
    _check(lib().cms_nnz_estimate(_ptr(a_colptr), _ptr(a_rowidx), _ptr(a_val), _ptr(b_rowptr), _ptr(b_colidx),
                                  _ptr(b_val), n1, n2, n3, _DTYPES[a_val.dtype], seed & ((1 << 64) - 1), d, b_max,
                                  ctypes.byref(b_out), ctypes.byref(k_out), _ptr(ws), ws.numel() * ws.element_size(),
                                  _stream(stream)))
    return b_out.value, k_out.value


def frobenius_estimate(A: torch.Tensor, B: torch.Tensor, seed: int, d: int, stream=None):
    """Sec. 5.2: (X float64 (d,), bound) with X_t the AMS sketches of AB under
    4-wise independent signs and bound = 32 median X_t^2 >= ||AB||_F^2 (whp)."""
    n1, n2, n3, lda, ldb = _ab_args(A, B)
    need = _SZ()
    _check(lib().cms_frobenius_workspace_size(n1, n2, n3, d, ctypes.byref(need)))
    ws = alloc_workspace(need.value, A.device)
    est = torch.empty(d, dtype=torch.float64, device=A.device)
    bound = torch.empty(1, dtype=torch.float64, device=A.device)
    _check(lib().cms_frobenius_estimate(_ptr(A), lda, _ptr(B), ldb, n1, n2, n3, _DTYPES[A.dtype],
                                        seed & ((1 << 64) - 1), d, _ptr(est), _ptr(bound), _ptr(ws),
                                        ws.numel() * ws.element_size(), _stream(stream)))
    return est, float(bound.item())


def merge(parts: list[torch.Tensor], out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Sum of partial sketches over disjoint inner-index ranges (linearity, eq. (1))."""
    if not parts:
        raise ValueError("parts is empty")
    d, b = parts[0].shape
    dev = parts[0].device
    for i, p_ in enumerate(parts):
        if p_.dim() != 2 or tuple(p_.shape) != (d, b):
            raise ValueError("parts must share one (d, b) shape")
        _check_buf(p_, f"parts[{i}]", dev, torch.float32, d * b)
    if out is None:
        out = torch.empty((d, b), dtype=torch.float32, device=dev)
    _check_buf(out, "out", dev, torch.float32, d * b)
    arr = (ctypes.c_void_p * len(parts))(*[p.data_ptr() for p in parts])
    _check(lib().cms_merge(arr, len(parts), d, b, _ptr(out), _stream(stream)))
    return out


def check_async(stream=None):
    _check(lib().cms_check_async(_stream(stream)))


def selftest_wait(stream=None):
    """Failure-detection self-test: the library's bounded wait on a phase that
    nothing completes.  Raises CmsError with status CMS_ERR_TIMEOUT (5) when
    the wait gave up, the designed outcome (about 2 s)."""
    _check(lib().cms_selftest_wait(_stream(stream)))


def profile_enable(on: bool = True):
    """Per-kernel CUDA-event timing of the library's launches (clears records)."""
    _check(lib().cms_profile_enable(1 if on else 0))


def profile_summary() -> dict:
    """{kernel: {"launches": L, "ms": total}} of the launches recorded so far."""
    import json
    need = _SZ()
    _check(lib().cms_profile_summary(None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value + 64)
    _check(lib().cms_profile_summary(buf, len(buf), None))
    return json.loads(buf.value.decode())


def status_string(s: int) -> str:
    return lib().cms_status_string(s).decode()

