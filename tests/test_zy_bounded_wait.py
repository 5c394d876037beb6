"""Failure detection on the GPU without a fault: the bounded wait the sketch
kernels use gives up and reports CMS_ERR_TIMEOUT, and the device still
computes afterwards.

The wait runs on an mbarrier phase that nothing completes; its limit is 2 s of
%globaltimer, after which the kernel writes its status and returns (no trap,
no hang).  This file is collected after the parity files so that a failure
here cannot hide them from a run that stops at the first failure.
"""
import time

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


def test_bounded_wait_gives_up_and_the_device_stays_usable(cms):
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.time()
    with pytest.raises(cms.CmsError) as e:
        cms.selftest_wait()
    assert e.value.status == 5                  # CMS_ERR_TIMEOUT
    assert 1.0 < time.time() - t0 < 60
    cms.check_async()                           # no error word left behind
    n1, n2, n3, b, d = 64, 40, 48, 1024, 2
    A = W.gaussian(n1, n2, 3).astype(np.float32)
    B = W.gaussian(n2, n3, 4).astype(np.float32)
    h = cms.make_hashes(5, max(n1, n3), b, d)
    tab = O.make_tables(5, max(n1, n3), b, d)
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev).T
    Bd = torch.from_numpy(B).to(dev)
    c = cms.sketch_product(Ad, Bd, h).cpu().numpy().astype(np.float64)
    ref = O.sketch_definition(A.astype(np.float64), B.astype(np.float64), tab)
    assert max(O.rel_l2(c[t], ref[t]) for t in range(d)) < 1e-5
    h.free()
