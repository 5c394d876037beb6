"""GPU parity of the Sec. 5.2 estimator: the AMS sketches X_t of AB under
4-wise independent signs (FP64 sums; equal to the oracle's to 1e-9 of the
sum of |terms|) and the bound 32 median X_t^2."""
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


@pytest.mark.parametrize("n1,n2,n3,d,dtype,alias", [
    (2048, 512, 2048, 9, torch.float32, True),
    (700, 333, 500, 5, torch.float32, False),
    (1024, 128, 1024, 4, torch.bfloat16, True),
    (300, 77, 450, 3, torch.float64, False),
    (64, 1, 64, 1, torch.float32, True),
])
def test_frobenius_estimate_matches_oracle(cms, n1, n2, n3, d, dtype, alias):
    seed = 1000 + n1 + d
    if alias:
        X = W.gaussian(n2, n1, seed).astype(np.float32)
        Xr = W.bf16_round(X)[0] if dtype == torch.bfloat16 else X
        xt = torch.from_numpy(X).to(dev(), dtype)
        A, B = xt.T, xt
        Ad, Bd = Xr.T.astype(np.float64), Xr.astype(np.float64)
    else:
        Ah = W.gaussian(n1, n2, seed).astype(np.float32)
        Bh = W.gaussian(n2, n3, seed + 1).astype(np.float32)
        A = torch.from_numpy(np.ascontiguousarray(Ah.T)).to(dev(), dtype).T
        B = torch.from_numpy(Bh).to(dev(), dtype)
        Ad, Bd = Ah.astype(np.float64), Bh.astype(np.float64)
    est, bound = cms.frobenius_estimate(A, B, seed, d)
    cms.check_async()
    want = O.ams_frobenius(Ad, Bd, seed, d)
    scale = np.abs(Ad).sum(axis=0) @ np.abs(Bd).sum(axis=1)      # sum_k |a_k|_1 |b_k|_1
    np.testing.assert_allclose(est.cpu().numpy(), want, rtol=0, atol=1e-9 * scale)
    assert abs(bound - O.frobenius_bound(want)) <= 1e-9 * 32 * scale ** 2
    if d >= 5:
        assert bound >= np.sum((Ad @ Bd) ** 2)
