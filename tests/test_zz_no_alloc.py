"""The allocation-free sketch entry point against the workspace one.

cms_sketch_product_noalloc serves callers that cannot allocate device
memory (it uses the library's fixed scratch array); here it must give the
same sketch as cms_sketch_product on two calls in a row, the second on new
data, so the shared array's leftover contents cannot leak into a result.
This file is collected last on purpose.
"""
import ctypes

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
    import paper_1108_1320_gb300.cms as m
    m.lib()
    return m


def _noalloc(cms, A, B, h, c):
    n1, n2, n3, lda, ldb = cms._ab_args(A, B)
    st = cms.lib().cms_sketch_product_noalloc(A.data_ptr(), lda, B.data_ptr(), ldb, n1, n2, n3,
                                              cms._DTYPES[A.dtype], h.handle, c.data_ptr(),
                                              torch.cuda.current_stream().cuda_stream)
    return st


def test_noalloc_matches_workspace_entry_point_twice(cms):
    dev = torch.device("cuda", torch.cuda.current_device())
    m, n, b, d = 512, 2048, 65536, 5
    h = cms.make_hashes(2, n, b, d)
    for call, seed in enumerate((41, 42)):
        X = torch.from_numpy(W.gaussian(m, n, seed).astype(np.float32)).to(dev)
        want = cms.sketch_product(X.T, X, h)
        got = torch.full_like(want, float("nan"))
        st = _noalloc(cms, X.T, X, h, got)
        assert st == 0, cms.lib().cms_last_error()
        torch.cuda.synchronize()
        cms.check_async()
        assert O.rel_l2(got.cpu().numpy(), want.cpu().numpy()) < TOL_F32, call
    h.free()


def test_noalloc_rejects_shapes_above_its_scratch(cms):
    dev = torch.device("cuda", torch.cuda.current_device())
    # b = 2^20 with many repetitions needs far more than 32 MiB of scratch
    h = cms.make_hashes(3, 1024, 1 << 20, 16)
    X = torch.zeros((64, 1024), device=dev)
    c = torch.empty((16, 1 << 20), device=dev)
    assert cms.workspace_size(h, 1024, 64, 1024) > (32 << 20)
    st = _noalloc(cms, X.T, X, h, c)
    assert st == 4
    assert b"32" in cms.lib().cms_last_error() or b"scratch" in cms.lib().cms_last_error()
    h.free()
