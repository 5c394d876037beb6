"""Seeded sweep of sketch products over shapes, storage types, aliasing and
alignment, each against the FP64 oracle's definition route, and each
kernel family reached at least once: the shared-memory kernel, the
lock-step register-FFT kernel (records in shared or tensor memory), the
warp-specialised kernel and the cluster kernel.  Tolerance: relative L2
1e-5 per repetition (BF16 against the BF16 values)."""
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


# (n1, n2, n3, b, d, dtype, alias, pad): pad > 0 gives A (or X) a leading
# dimension n1 + pad (rows not in whole 16-byte units when pad is odd)
CASES = [
    (512, 33, 512, 16384, 3, "f32", True, 0),
    (512, 33, 512, 16384, 3, "bf16", True, 0),
    (700, 21, 640, 12800, 2, "f32", False, 0),
    (701, 21, 643, 12800, 2, "f32", False, 3),
    (640, 9, 640, 10240, 4, "bf16", True, 1),
    (2048, 40, 2048, 65536, 5, "f32", True, 0),
    (1000, 30, 1000, 2000, 3, "f32", True, 0),
    (999, 17, 998, 27000, 1, "f64", False, 0),
    (300, 64, 300, 1 << 18, 2, "f32", True, 0),
    (1024, 12, 1024, 3 << 16, 3, "bf16", True, 0),
    (256, 256, 256, 1024, 1, "f32", True, 0),
    (96, 5, 80, 96, 2, "f32", False, 0),
    (1536, 8, 1536, 24576, 6, "f32", True, 0),
    (800, 25, 800, 4000, 7, "bf16", True, 0),
    (1024, 21, 960, 32768, 3, "f32", False, 0),   # warp-specialised: two operands, odd inner dimension
    (2048, 13, 2048, 65536, 2, "f32", True, 0),   # warp-specialised: aliased, odd inner dimension
]
DT = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}x{c[2]}-b{c[3]}-d{c[4]}-{c[5]}-{'alias' if c[6] else 'ab'}-pad{c[7]}"
                                             for c in CASES])
def test_sweep_matches_oracle(cms, case):
    n1, n2, n3, b, d, dts, alias, pad = case
    dt = DT[dts]
    seed = n1 * 7 + n2 * 11 + b
    n = max(n1, n3)
    h = cms.make_hashes(seed, n, b, d)
    tab = O.make_tables(seed, n, b, d)

    def stored(a):
        return W.bf16_round(a)[0] if dts == "bf16" else a

    if alias:
        X = W.gaussian(n2, n1, seed).astype(np.float32 if dts != "f64" else np.float64)
        buf = torch.zeros((n2, n1 + pad), dtype=dt, device=dev())
        buf[:, :n1] = torch.from_numpy(X).to(dev(), dt)
        xt = buf[:, :n1]
        A, B = xt.T, xt
        Xs = stored(X).astype(np.float64)
        Ad, Bd = Xs.T, Xs
    else:
        Ah = W.gaussian(n1, n2, seed).astype(np.float32 if dts != "f64" else np.float64)
        Bh = W.gaussian(n2, n3, seed + 1).astype(np.float32 if dts != "f64" else np.float64)
        abuf = torch.zeros((n2, n1 + pad), dtype=dt, device=dev())
        abuf[:, :n1] = torch.from_numpy(np.ascontiguousarray(Ah.T)).to(dev(), dt)
        A = abuf[:, :n1].T
        B = torch.from_numpy(Bh).to(dev(), dt)
        Ad, Bd = stored(Ah).astype(np.float64), stored(Bh).astype(np.float64)
    kernel = cms.plan_kernel(A, B, h)
    c = cms.sketch_product(A, B, h).cpu().numpy()
    cms.check_async()
    ref = O.sketch_definition(Ad, Bd, tab)
    err = max(O.rel_l2(c[t], ref[t]) for t in range(d))
    assert err < 1e-5, (kernel, err)
    h.free()


def test_sweep_reaches_every_kernel_family(cms):
    seen = set()
    for n1, n2, n3, b, d, dts, alias, pad in CASES:
        h = cms.make_hashes(1, max(n1, n3), b, d)
        dt = DT[dts]
        buf = torch.zeros((n2, n1 + pad), dtype=dt, device=dev())
        xt = buf[:, :n1]
        B = xt if alias else torch.zeros((n2, n3), dtype=dt, device=dev())
        seen.add(cms.plan_kernel(xt.T, B, h))
        h.free()
    # large hash domains reach the tensor-memory records
    h = cms.make_hashes(1, 6000, 96000, 2)
    x = torch.zeros((4, 6000), device=dev())
    seen.add(cms.plan_kernel(x.T, x, h))
    h.free()
    assert seen == {"shared_memory", "lockstep", "lockstep_tmem", "warp_specialised", "cluster"}, seen


def test_warp_specialised_cases_take_that_kernel(cms):
    # the two odd-inner-dimension cases above run the warp-specialised
    # kernel (its last group then holds one inner index)
    for n1, n2, n3, b, d, dts, alias, pad in CASES[-2:]:
        h = cms.make_hashes(1, max(n1, n3), b, d)
        xt = torch.zeros((n2, n1), dtype=DT[dts], device=dev())
        B = xt if alias else torch.zeros((n2, n3), dtype=DT[dts], device=dev())
        assert cms.plan_kernel(xt.T, B, h) == "warp_specialised", (n1, n2, n3)
        h.free()
