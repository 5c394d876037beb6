"""The allocation-free sketch entry point, checked against the FP64 oracle
and against the workspace entry point.

cms_sketch_product_noalloc serves callers that cannot allocate device
memory: code running inside a host application whose allocator owns the
device, or a path that must not call cudaMalloc/cudaFree.  It uses the
library's fixed scratch array instead of a caller workspace.  Here it must
give, on two calls in a row (the second on new data, so the shared array's
leftover contents cannot leak into a result), the sketch of the Sec. 2.2
definition within the tolerance of the parity tests, and the same sketch as
cms_sketch_product.  This file is collected last on purpose.
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


def test_noalloc_matches_oracle_and_workspace_entry_point_twice(cms):
    dev = torch.device("cuda", torch.cuda.current_device())
    m, n, b, d = 512, 2048, 65536, 5
    h = cms.make_hashes(2, n, b, d)
    tab = O.make_tables(2, n, b, d)
    for call, seed in enumerate((41, 42)):
        Xh = W.gaussian(m, n, seed).astype(np.float32)
        X = torch.from_numpy(Xh).to(dev)
        want = cms.sketch_product(X.T, X, h)
        got = torch.full_like(want, float("nan"))
        st = _noalloc(cms, X.T, X, h, got)
        assert st == 0, cms.lib().cms_last_error()
        torch.cuda.synchronize()
        cms.check_async()
        g = got.cpu().numpy().astype(np.float64)
        Xd = Xh.astype(np.float64)
        ref = O.sketch_definition(Xd.T, Xd, tab)
        errs = [O.rel_l2(g[t], ref[t]) for t in range(d)]
        assert max(errs) < TOL_F32, (call, errs)
        assert O.rel_l2(g, want.cpu().numpy()) < TOL_F32, call
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
