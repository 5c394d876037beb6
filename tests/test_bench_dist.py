"""The benchmark's multi-rank path on CPU: two gloo ranks, per-rank times
reduced with a max, whole-job throughput from the slowest rank; the
reference arm does no work on ranks other than 0."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    per_rank_ms = [120.0, 150.0][rank]
    mx = bench.reduce_max(per_rank_ms, dist, torch.device("cpu"))
    val = bench.job_value(world, 10, mx)
    dist.barrier()
    q.put((rank, mx, val))
    dist.destroy_process_group()


def test_two_rank_max_and_job_value():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, mx, val in res:
        assert mx == 150.0                       # the slowest rank's time
        assert abs(val - 2 * 10 / 0.150) < 1e-9  # all ranks' products over that time


def test_single_process_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, None, torch.device("cpu")) == 3.5
    assert bench.job_value(1, 200, 1000.0) == 200.0


def test_reference_arm_idles_on_other_ranks(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        gpus, steps, warmup = 2, 1, 3
    bench.reference_arm(A())
    assert capsys.readouterr().out == ""


def test_roofline_bookkeeping():
    # the algorithmic flop count of the fused step, Sec. 2.2: per repetition
    # and inner index one packed complex length-b FFT (5 b log2 b) and the
    # spectral multiply-accumulate (8 flops x b/2 bins), plus one inverse
    # (2.5 b log2 b) per repetition; covariance shape: 1.127e11 per launch
    sys.path.insert(0, ROOT)
    import bench
    d, K, b = 5, 4096, 65536
    assert bench.sketch_flops(d, K, b) == d * K * (5 * b * 16 + 4 * b)
    assert abs(bench.sketch_flops(d, K, b) - 1.1274e11) / 1.1274e11 < 1e-3
    assert bench.total_flops(d, K, b) == bench.sketch_flops(d, K, b) + d * 2.5 * b * 16
    assert bench.sketch_flops(3, 1, 1) == 3 * 4          # log2 1 = 0: the MAC term alone


def test_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    # the DRAM traffic figure is reported only for the kernel source it was
    # captured on: any change to a kernel file makes it null
    sys.path.insert(0, ROOT)
    import json
    import bench
    rec = {"source_sha": bench.kernel_source_hash(), "dram_bytes_per_launch_full": 123}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.load_traffic() == 123
    f.write_text(json.dumps(dict(rec, source_sha="0" * 16)))
    assert bench.load_traffic() is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "absent.json"))
    assert bench.load_traffic() is None


def test_shard_ranges_cover_the_inner_indices_in_order():
    sys.path.insert(0, ROOT)
    import bench
    for total in (0, 1, 5, 4096, 4097):
        for world in (1, 2, 3, 8):
            rs = bench.shard_ranges(total, world)
            assert len(rs) == world
            assert rs[0][0] == 0 and rs[-1][1] == total
            for (a0, a1), (b0, b1) in zip(rs, rs[1:]):
                assert a1 == b0                       # contiguous, disjoint, in rank order
            sizes = [k1 - k0 for k0, k1 in rs]
            assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1


def _kshard_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np

    import bench
    import workloads as W
    from oracle import cms_oracle as O
    m, n, b, d = 37, 24, 64, 3
    X = W.gaussian(m, n, 11)
    tab = O.make_tables(5, n, b, d)
    k0, k1 = bench.shard_ranges(m, world)[rank]
    Xr = X[k0:k1]
    part = torch.from_numpy(O.sketch_fft(Xr.T, Xr, tab))      # this rank's partial sketch
    parts = bench.gather_in_rank_order(part, dist)
    merged = parts[0].clone()
    for p_ in parts[1:]:
        merged += p_                                           # fixed rank order
    q.put((rank, merged.numpy()))
    dist.destroy_process_group()


def test_k_split_over_two_ranks_gives_the_whole_sketch():
    # eq. (1): the sketch of AB is the sum over k of the outer products'
    # sketches, so two ranks sketching the two halves of the inner indices
    # and merging their partials in rank order give the whole product's
    # sketch, the same on both ranks
    import numpy as np

    sys.path.insert(0, ROOT)
    import workloads as W
    from oracle import cms_oracle as O
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_kshard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    X = W.gaussian(37, 24, 11)
    whole = O.sketch_fft(X.T, X, O.make_tables(5, 24, 64, 3))
    for _, merged in res:
        assert O.rel_l2(merged, whole) < 1e-12
    np.testing.assert_array_equal(res[0][1], res[1][1])
