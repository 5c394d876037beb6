#!/usr/bin/env python
"""Throughput of the compressed matrix product (COMPRESSEDPRODUCT + DECOMPRESS,
Fig. 1 of Pagh, arXiv 1108.1320) on the sample-covariance workload.

Workload (Sec. 3.2 use): X = 4096 samples x 2048 variables, FP32, i.i.d.
N(0, 1) with 32 disjoint planted pairs of correlation 0.5; A = X^T, B = X;
b = 65536, d = 5.  One step = one product: redraw the hash functions on the
device (new seed), sketch (hash -> FFT -> spectral product summed over k ->
inverse FFT), and decode all 2048 x 2048 estimates (median of 5).

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead
(on a bounded sample of the same workload, scaled to products/s).
"""
from __future__ import annotations

import argparse
import datetime as _dt
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "A,B GB/s as % of HBM roofline; products/s fused FP32 vs plain FP64, same error"
WORKLOAD = dict(name="covariance", m=4096, n=2048, pairs=32, rho=0.5, b=65536, d=5, seed=2)
FLUSH_BYTES = 256 << 20            # > 129 MB L2: written between timed steps
FP32_LANES_PER_SM = 128            # Blackwell SM: 4 partitions x 32 FP32 lanes
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_sketch_ws_covariance.json")
# the fused sketch kernels' profiling names: warp-specialised, lock-step,
# shared-memory (generic)
SKETCH_KERNEL_NAMES = ("k_sketch_ws", "k_sketch_fast", "k_sketch_fused")
# the sources of the dominant kernel's code and launch: the kernel itself,
# its helpers, the planner that shapes its launch and the table builder whose
# records it reads (a change to any of them voids the kept DRAM counters)
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1108_1320_gb300", "csrc", f)
                  for f in ("k_sketch.cu", "k_sketch_ws.cu", "k_tables.cu", "warp_fft.cuh",
                            "cms_common.cuh")]


def workload_label(w=WORKLOAD) -> str:
    return (f"covariance X {w['m']}x{w['n']} fp32, {w['pairs']} planted pairs rho={w['rho']}, "
            f"A=X^T B=X, b={w['b']}, d={w['d']}")


def sketch_flops(d: int, K: int, b: int) -> float:
    """Algorithmic flops of the fused kernel: per repetition and inner index,
    two real length-b FFTs packed as one complex FFT (5 b log2 b) plus the
    spectral complex multiply-accumulate (8 flops x b/2 bins)."""
    return d * K * (5.0 * b * math.log2(b) + 4.0 * b)


def total_flops(d: int, K: int, b: int) -> float:
    return sketch_flops(d, K, b) + d * 2.5 * b * math.log2(b)


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def load_traffic():
    """DRAM bytes per launch of the fused kernel from the committed ncu
    summary, or None when absent or taken on a different kernel source."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_sha") != kernel_source_hash():
        return None
    return rec.get("dram_bytes_per_launch_full")


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.6)      # let nvidia-smi attach before the timed region

    def mark_begin(self):
        self.t0 = _dt.datetime.now()

    def mark_end(self):
        self.t1 = _dt.datetime.now()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = []
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = _dt.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                continue
            rows.append((ts, parts))
        inside = [p for ts, p in rows if self.t0 and self.t1 and self.t0 <= ts <= self.t1]
        used = inside if inside else [p for _, p in rows]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[1]) for p in used if num(p[1]) is not None]
        mx = [num(p[2]) for p in used if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for p in used for k in range(4) if p[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons,
                "samples": len(inside),
                "samples_total": len(rows),
                "power_w_max": max((num(p[3]) or 0.0) for p in used) if used else None}


# ------------------------------------------------------ multi-rank timing --
def reduce_max(x: float, dist, device) -> float:
    """Max of a per-rank time over all ranks (identity without a process group)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, units_per_rank: int, max_ms: float) -> float:
    """Whole-job throughput: units processed by all ranks over the slowest rank's time."""
    return world * units_per_rank / (max_ms / 1e3)


def shard_ranges(total: int, world: int) -> list:
    """The inner indices 0..total-1 cut into `world` contiguous, disjoint
    ranges in rank order (sizes differ by at most one): rank r sketches the
    rows X[k0:k1] of its range (eq. (1): the sketch of AB is the sum over k)."""
    q, r = divmod(total, world)
    out, k0 = [], 0
    for i in range(world):
        k1 = k0 + q + (1 if i < r else 0)
        out.append((k0, k1))
        k0 = k1
    return out


def gather_in_rank_order(part, dist) -> list:
    """Every rank's partial sketch, in rank order (one all-gather of d b
    floats per rank); summed in that fixed order the result is the same on
    every rank and in every run."""
    import torch
    parts = [torch.empty_like(part) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, part.contiguous())
    return parts


# --------------------------------------------------------- CPU oracle leg --
def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_warm(_):
    from oracle import cms_oracle  # noqa: F401
    return os.getpid()


def _route_f_chunk(job):
    """Pool worker: Route F (Fig. 1) of the oracle over one contiguous range of
    inner indices (rows of X), FP64."""
    Xs, seed, n, b, d = job
    from oracle import cms_oracle as O
    X64 = np.asarray(Xs, dtype=np.float64)
    return O.sketch_fft(X64.T, X64, O.make_tables(seed, n, b, d))


class OraclePool:
    """The FP64 oracle's Route F on every host core: the inner indices are cut
    into one contiguous range per process and the partial sketches summed
    (the sketch is linear in the sum over k, eq. (1)).  The processes are
    started with 'spawn' (the parent holds a CUDA context) and import the
    oracle before anything is timed."""

    def __init__(self, cores: int):
        import multiprocessing as mp
        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores)
        self.pool.map(_oracle_warm, range(cores))

    def sketch(self, X: np.ndarray, seed: int, w: dict, k_count: int) -> np.ndarray:
        ranges = [r for r in np.array_split(np.arange(k_count), self.cores) if len(r)]
        jobs = [(X[r[0]:r[-1] + 1], seed, w["n"], w["b"], w["d"]) for r in ranges]
        return np.sum(self.pool.map(_route_f_chunk, jobs), axis=0)

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_sample(pool: OraclePool, X: np.ndarray, w: dict, k_count: int, seed: int, rows: int = 16):
    """Time the oracle (Route F over the first k_count inner indices on all
    host cores, then DECOMPRESS of `rows` rows of the dense decode on one);
    returns (c of the sample, sketch seconds, decode seconds, extrapolated
    seconds per full product)."""
    from oracle import cms_oracle as O
    n, b, d = w["n"], w["b"], w["d"]
    t0 = time.perf_counter()
    c = pool.sketch(X, seed, w, k_count)
    t1 = time.perf_counter()
    O.decompress_dense(c, O.make_tables(seed, n, b, d), rows, n)
    t2 = time.perf_counter()
    per_product = (t1 - t0) * (w["m"] / k_count) + (t2 - t1) * (n / rows)
    return c, t1 - t0, t2 - t1, per_product


def sample_size(pool: OraclePool, X: np.ndarray, w: dict, budget_s: float) -> int:
    """Inner indices the pool sketches (plus the decode rows) in about
    budget_s seconds: at least one per core, at most the whole product."""
    oracle_sample(pool, X, w, pool.cores, 1)          # first calls: FFT plans, tables
    k = 4 * pool.cores
    _, t_sketch, t_decode, _ = oracle_sample(pool, X, w, k, 1)
    per_k = t_sketch / k
    return int(max(pool.cores, min(w["m"], (budget_s - t_decode) / max(per_k, 1e-9))))


def cpu_baseline(X: np.ndarray, w: dict, budget_s: float = 12.0, gpu_sketch=None) -> dict:
    """The oracle as it stands on every host core, on a bounded sample of the
    workload (the whole product when the budget allows).  With gpu_sketch
    (seed, k_count) -> c, the library's sketch of the same sample is compared
    with the oracle's, bucket by bucket: the rounding error of the FP32 path
    against FP64."""
    cores = host_cores()
    pool = OraclePool(cores)
    try:
        k_count = sample_size(pool, X, w, budget_s)
        seed = 2
        c_ref, t_sketch, t_decode, per = oracle_sample(pool, X, w, k_count, seed)
        took = t_sketch + t_decode
    finally:
        pool.close()
    out = {"value": 1.0 / per, "unit": "products/s", "cores": cores, "kind": "oracle",
           "sample": f"Route F (per-k numpy FFT, FP64) over {k_count} of {w['m']} inner indices on "
                     f"{cores} processes, and 16 of {w['n']} decode rows, scaled to one product; "
                     f"{took:.1f} s wall"}
    if gpu_sketch is not None:
        c_gpu = np.asarray(gpu_sketch(seed, k_count), dtype=np.float64)
        per_rep = [float(np.linalg.norm(c_gpu[t] - c_ref[t]) / np.linalg.norm(c_ref[t]))
                   for t in range(w["d"])]
        out["c_rel_l2_gpu_vs_oracle"] = max(per_rep)
        out["c_rel_l2_per_rep"] = per_rep
        out["compared"] = f"all {w['d']} x {w['b']} buckets of the sketch of X[:{k_count}] (seed {seed})"
        out["k_count"] = k_count
    return out


def reference_arm(args):
    """--impl reference: the oracle on the host cores, rank 0 only.  Every
    step sketches a bounded sample of the covariance workload (the first
    k_count inner indices) on all host cores; ms_per_step is that sample's
    wall time, value the throughput scaled to whole products."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import workloads as W
    w = WORKLOAD
    cov = W.covariance(w["m"], w["n"], w["pairs"], w["rho"], w["seed"], dtype=np.float32)
    cores = host_cores()
    pool = OraclePool(cores)
    try:
        per_step_s = max(0.25, min(3.0, 60.0 / max(args.steps + args.warmup, 1)))
        k_count = sample_size(pool, cov.X, w, per_step_s)
        walls, pers = [], []
        for i in range(args.warmup + args.steps):
            _, t_sketch, t_decode, per = oracle_sample(pool, cov.X, w, k_count, 100 + i)
            took = t_sketch + t_decode
            if i >= args.warmup:
                walls.append(took)
                pers.append(per)
    finally:
        pool.close()
    value = 1.0 / statistics.mean(pers)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "products/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(walls) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_label(), "m": w["m"], "n": w["n"], "b": w["b"], "d": w["d"],
                   "pairs": w["pairs"], "rho": w["rho"], "l2": "host run"},
        "cpu_baseline": {"value": value, "unit": "products/s", "cores": cores, "kind": "oracle",
                         "sample": f"each step: Route F over {k_count} of {w['m']} inner indices on "
                                   f"{cores} processes + 16 decode rows; ms_per_step is that sample's "
                                   f"wall time, value scaled to whole products"},
        "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------- GPU arm -----
def gpu_arm(args):
    import torch
    import torch.distributed as dist

    import workloads as W
    from paper_1108_1320_gb300 import build as B
    B.build()
    import paper_1108_1320_gb300 as cms

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOAD
    m, n, b, d = w["m"], w["n"], w["b"], w["d"]

    cov = W.covariance(m, n, w["pairs"], w["rho"], w["seed"], dtype=np.float32)
    X_host = torch.from_numpy(cov.X).pin_memory()
    X = X_host.to(dev)
    h = cms.make_hashes(w["seed"], n, b, d)
    ws = cms.alloc_workspace(cms.workspace_size(h, n, m, n, torch.float32), dev)
    c = torch.empty((d, b), dtype=torch.float32, device=dev)
    est = torch.empty((n, n), dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    seed_base = 1000 * (rank + 1)

    def step(i):
        h.reseed(seed_base + i, stream)
        cms.sketch_product(X.T, X, h, c=c, ws=ws, stream=stream)
        cms.decode_dense(c, h, n, n, out=est, stream=stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    cms.check_async()

    uuid = str(torch.cuda.get_device_properties(dev).uuid)
    sampler = ClockSampler(uuid if uuid.startswith("GPU-") else f"GPU-{uuid}")
    sampler.start()
    cms.profile_enable(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.mark_begin()
    for i in range(args.steps):
        flush.zero_()                                  # evict X and c from L2
        starts[i].record(stream)
        step(args.warmup + i)
        stops[i].record(stream)
    torch.cuda.synchronize()
    sampler.mark_end()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    prof = cms.profile_summary()
    cms.profile_enable(False)
    cms.check_async()
    step_ms = [a.elapsed_time(z) for a, z in zip(starts, stops)]
    total_ms = reduce_max(sum(step_ms), dist if world > 1 else None, dev)
    value = job_value(world, args.steps, total_ms)
    launches = int(sum(v["launches"] for v in prof.values()))

    # ---- roofline of the dominant kernel (the fused sketch kernel) --------
    # the fused sketch kernel this plan ran (each kernel has its own record)
    fused_name = next((k for k in SKETCH_KERNEL_NAMES if prof.get(k, {}).get("launches", 0) > 0),
                      "k_sketch_ws")
    fused = prof.get(fused_name, {"launches": 0, "ms": float("nan")})
    fused_ms = fused["ms"] / max(fused["launches"], 1)
    props = torch.cuda.get_device_properties(dev)
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    alg_flops = sketch_flops(d, m, b)
    achieved = alg_flops / (fused_ms * 1e-3) / 1e12
    traffic = load_traffic()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic,
                "kernel": fused_name, "kernel_ms": fused_ms,
                "alg_flops_per_launch": alg_flops,
                "peak_source": f"derived: {props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 "
                               f"lanes x 2 flop/FMA x {max_mhz:.0f} MHz (FP32 FMA pipe, not tensor)"}
    ms_step = total_ms / args.steps
    ab_bytes = 2 * m * n * 4                       # A and B each read once (same bytes here)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    ab_gbs = ab_bytes / (ms_step * 1e-3) / 1e9
    extra = {
        "ab_gbs": ab_gbs, "ab_hbm_frac": ab_gbs / hbm,
        "hbm_peak_gbs": hbm, "hbm_peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
        "roofline_time_ms": max(ab_bytes / (hbm * 1e9), total_flops(d, m, b) / (peak_tflops * 1e12)) * 1e3,
        "kernel_ms": {k: v["ms"] / max(v["launches"], 1) for k, v in prof.items()},
    }
    extra["step_frac_of_roofline"] = extra["roofline_time_ms"] / ms_step
    sketch_kernels = ("k_twiddle_table", "k_frontend_twiddles", *SKETCH_KERNEL_NAMES, "k_rows_inverse",
                      "k_cols_inverse")
    extra["sketch_only_ms"] = sum(prof[k]["ms"] for k in sketch_kernels if k in prof) / args.steps

    # ---- end to end through the public API with host buffers --------------
    c_host = torch.empty((d, b), dtype=torch.float32).pin_memory()
    pairs = torch.from_numpy(cov.pairs).to(dev)
    pair_host = torch.empty(len(cov.pairs), dtype=torch.float32).pin_memory()
    pair_est = torch.empty(len(cov.pairs), dtype=torch.float32, device=dev)
    e2e_steps = max(3, min(args.steps, 50))
    # the input of step i is copied into buffer i % 2 on a copy stream while
    # step i - 1 computes (double buffering, as a caller of the asynchronous
    # API would); every step's copy lies inside the timed region
    copy_stream = torch.cuda.Stream(device=dev)
    Xe = [torch.empty_like(X), torch.empty_like(X)]
    x_ready = [torch.cuda.Event(), torch.cuda.Event()]
    x_free = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_copy(i):
        s2 = i % 2
        copy_stream.wait_event(x_free[s2])        # step i - 2 is done reading it
        with torch.cuda.stream(copy_stream):
            Xe[s2].copy_(X_host, non_blocking=True)
        x_ready[s2].record(copy_stream)

    def e2e_step(i, prefetch):
        s2 = i % 2
        stream.wait_event(x_ready[s2])
        if prefetch:
            e2e_copy(i + 1)
        h.reseed(seed_base + 50000 + i, stream)
        cms.sketch_product(Xe[s2].T, Xe[s2], h, c=c, ws=ws, stream=stream)
        x_free[s2].record(stream)
        cms.decode_dense(c, h, n, n, out=est, stream=stream)
        cms.decode(c, h, pairs, out=pair_est, stream=stream)
        c_host.copy_(c, non_blocking=True)
        pair_host.copy_(pair_est, non_blocking=True)

    e2e_copy(0)
    e2e_step(0, False)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    copy_stream.wait_event(e0)
    e2e_copy(1)
    for i in range(e2e_steps):
        e2e_step(1 + i, i + 1 < e2e_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(e0.elapsed_time(e1), dist if world > 1 else None, dev)
    e2e = {"value": job_value(world, e2e_steps, e2e_ms), "unit": "products/s",
           "h2d_bytes_per_step": m * n * 4,
           "d2h_bytes_per_step": d * b * 4 + len(cov.pairs) * 4,
           "steps": e2e_steps}

    line = {
        "metric": METRIC, "value": value, "unit": "products/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_label(), "m": m, "n": n, "b": b, "d": d,
                   "pairs": w["pairs"], "rho": w["rho"],
                   "l2": f"flushed between steps ({FLUSH_BYTES >> 20} MiB write, outside the step events)",
                   "parallelism": f"independent products per GPU x{world}"},
        "roofline": roofline, "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
    }
    line.update(extra)

    if rank == 0 and not args.no_context:
        line["context"] = context_numbers(cms, torch, X, h, c, cov, w, dev, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        def gpu_sketch(seed, k_count):
            Xk = X[:k_count]
            hk = cms.make_hashes(seed, n, b, d)
            ck = cms.sketch_product(Xk.T, Xk, hk, stream=stream).cpu().numpy()
            hk.free()
            return ck
        cb = cpu_baseline(cov.X, w, budget_s=args.cpu_budget, gpu_sketch=gpu_sketch)
        line["cpu_baseline"] = cb
        Xk = X[: cb["k_count"]].double()
        line["rounding_error"] = {
            "c_rel_l2_vs_fp64_oracle": cb.get("c_rel_l2_gpu_vs_oracle"),
            "compared": cb.get("compared"),
            "sketch_std_of_compared": float(torch.linalg.norm(Xk.T @ Xk)) / math.sqrt(b),
            "note": "the FP32 path's c against the oracle's Route F (FP64) over the same inner indices "
                    "and hash draw; the sketch's own standard deviation ||AB||_F / sqrt(b) beside it"}
        del Xk
    if rank == 0:
        print(json.dumps(line))
    h.free()
    if world > 1:
        dist.destroy_process_group()


def gpu_arm_kshard(args):
    """--shard k: one product shared by all ranks (Sec. 2.2 / eq. (1): the
    sketch is linear in the sum over k).  Rank r sketches X[k0:k1] of its
    range with the hash draw every rank makes from the same seed; the d b
    partial sketches are all-gathered and merged in rank order (cms_merge),
    then decoded.  One step = one product; value = products/s over the
    slowest rank's time (strong scaling: the work per product is fixed)."""
    import torch
    import torch.distributed as dist

    import workloads as W
    from paper_1108_1320_gb300 import build as B
    B.build()
    import paper_1108_1320_gb300 as cms

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOAD
    m, n, b, d = w["m"], w["n"], w["b"], w["d"]
    k0, k1 = shard_ranges(m, world)[rank]
    cov = W.covariance(m, n, w["pairs"], w["rho"], w["seed"], dtype=np.float32)
    X_host = torch.from_numpy(np.ascontiguousarray(cov.X[k0:k1])).pin_memory()
    Xr = X_host.to(dev)
    h = cms.make_hashes(w["seed"], n, b, d)
    ws = cms.alloc_workspace(cms.workspace_size(h, n, k1 - k0, n, torch.float32), dev)
    c_part = torch.empty((d, b), dtype=torch.float32, device=dev)
    c = torch.empty((d, b), dtype=torch.float32, device=dev)
    est = torch.empty((n, n), dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(i):
        h.reseed(7000 + i, stream)            # the same draw on every rank
        cms.sketch_product(Xr.T, Xr, h, c=c_part, ws=ws, stream=stream)
        parts = gather_in_rank_order(c_part, dist) if world > 1 else [c_part]
        cms.merge(parts, out=c, stream=stream)
        cms.decode_dense(c, h, n, n, out=est, stream=stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    cms.check_async()
    uuid = str(torch.cuda.get_device_properties(dev).uuid)
    sampler = ClockSampler(uuid if uuid.startswith("GPU-") else f"GPU-{uuid}")
    sampler.start()
    cms.profile_enable(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.mark_begin()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        step(args.warmup + i)
        stops[i].record(stream)
    torch.cuda.synchronize()
    sampler.mark_end()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    prof = cms.profile_summary()
    cms.profile_enable(False)
    cms.check_async()
    total_ms = reduce_max(sum(a.elapsed_time(z) for a, z in zip(starts, stops)), dist if world > 1 else None,
                          dev)
    value = args.steps / (total_ms / 1e3)
    fused_name = next((k for k in SKETCH_KERNEL_NAMES if prof.get(k, {}).get("launches", 0) > 0),
                      "k_sketch_ws")
    fused = prof.get(fused_name, {"launches": 0, "ms": float("nan")})
    fused_ms = fused["ms"] / max(fused["launches"], 1)
    props = torch.cuda.get_device_properties(dev)
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    achieved = sketch_flops(d, k1 - k0, b) / (fused_ms * 1e-3) / 1e12
    # end to end: each rank's rows of X copied from pinned host memory, the
    # merged sketch read back, inside the timed region
    c_host = torch.empty((d, b), dtype=torch.float32).pin_memory()
    Xe = torch.empty_like(Xr)
    e2e_steps = max(3, min(args.steps, 50))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(e2e_steps):
        Xe.copy_(X_host, non_blocking=True)
        h.reseed(9000 + i, stream)
        cms.sketch_product(Xe.T, Xe, h, c=c_part, ws=ws, stream=stream)
        parts = gather_in_rank_order(c_part, dist) if world > 1 else [c_part]
        cms.merge(parts, out=c, stream=stream)
        c_host.copy_(c, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(e0.elapsed_time(e1), dist if world > 1 else None, dev)
    line = {
        "metric": METRIC, "value": value, "unit": "products/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_label(), "m": m, "n": n, "b": b, "d": d, "pairs": w["pairs"],
                   "rho": w["rho"],
                   "l2": f"flushed between steps ({FLUSH_BYTES >> 20} MiB write, outside the step events)",
                   "parallelism": f"one product over {world} GPUs: inner indices split in contiguous ranges, "
                                  f"partial sketches all-gathered and merged in rank order"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": fused_name, "kernel_ms": fused_ms,
                     "note": "this rank's share of the inner indices"},
        "clocks": clocks,
        "e2e": {"value": e2e_steps / (e2e_ms / 1e3), "unit": "products/s",
                "h2d_bytes_per_step": (k1 - k0) * n * 4, "d2h_bytes_per_step": d * b * 4, "steps": e2e_steps},
        "gpu_launches": int(sum(v["launches"] for v in prof.values())),
        "rank_inner_range": [k0, k1],
    }
    if rank == 0:
        print(json.dumps(line))
    h.free()
    if world > 1:
        dist.destroy_process_group()


def context_numbers(cms, torch, X, h, c, cov, w, dev, stream):
    """Plain FP64 form (same product, same seed) and cuBLAS SGEMM for context,
    plus the 'same error' comparison of the two forms."""
    m, n, b, d = w["m"], w["n"], w["b"], w["d"]
    out = {}
    h.reseed(w["seed"], stream)
    c32 = cms.sketch_product(X.T, X, h, stream=stream)
    Xd = X.double()
    wsp = cms.alloc_workspace(cms.plain_workspace_size(h, n, m, n), dev)
    c64 = torch.empty((d, b), dtype=torch.float64, device=dev)
    cms.sketch_product_plain_f64(Xd.T, Xd, h, c=c64, ws=wsp, stream=stream)   # warm-up
    torch.cuda.synchronize()
    reps = 2
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        cms.sketch_product_plain_f64(Xd.T, Xd, h, c=c64, ws=wsp, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / reps
    out["plain_f64"] = {"value": 1e3 / plain_ms, "unit": "products/s", "ms_per_product": plain_ms,
                        "note": "sketch only (no decode), FP64, unfused passes, one instance per call"}
    # same error: decoded estimates of both forms against the exact product
    AB = Xd.T @ Xd
    fro = float(torch.linalg.norm(AB))
    idx = torch.from_numpy(np.stack(np.meshgrid(np.arange(0, n, 7), np.arange(0, n, 5),
                                                indexing="ij"), -1).reshape(-1, 2)).to(dev)
    e32 = cms.decode(c32, h, idx).double()
    e64 = cms.decode(c64, h, idx)
    ref = AB[idx[:, 0], idx[:, 1]]
    rms = lambda v: float(torch.sqrt(torch.mean(v * v)))          # noqa: E731
    out["same_error"] = {
        "sketch_std": fro / math.sqrt(b),
        "fused_rms_err_vs_AB": rms(e32 - ref), "plain_rms_err_vs_AB": rms(e64 - ref),
        "c_rel_l2_fused_vs_plain": float(torch.max(torch.linalg.norm(c32.double() - c64, dim=1) /
                                                    torch.linalg.norm(c64, dim=1))),
        "pairs_sampled": int(idx.shape[0])}
    planted = torch.from_numpy(cov.pairs).to(dev)
    pe = cms.decode(c32, h, planted)
    out["planted_pairs"] = {"count": int(planted.shape[0]), "median_estimate": float(pe.median()),
                            "expected": w["rho"] * m,
                            "recovered_above_half": int((pe > 0.5 * w["rho"] * m).sum())}
    # covariance post-steps (Sec. 3.2, Fig. 2): the diagonal's contribution
    # removed from the sketch, then the estimates thresholded at rho m / 2
    cq = c32.clone()
    e0.record(stream)
    cms.remove_diagonal(X.T, X, h, cq, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    rd_ms = e0.elapsed_time(e1)
    tau = 0.5 * w["rho"] * m
    cms.decode_threshold(cq, h, n, n, tau, capacity=1 << 20, stream=stream)      # warm-up
    torch.cuda.synchronize()
    e0.record(stream)
    ij, _, count = cms.decode_threshold(cq, h, n, n, tau, capacity=1 << 20, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    th_ms = e0.elapsed_time(e1)
    hits = set(map(tuple, ij.cpu().numpy().tolist()))
    pl = [(int(u), int(v)) for u, v in cov.pairs] + [(int(v), int(u)) for u, v in cov.pairs]
    found = sum(p in hits for p in pl)
    pe2 = cms.decode(cq, h, planted)
    out["post_steps"] = {"remove_diagonal_ms": rd_ms, "threshold_ms": th_ms, "threshold": tau,
                         "candidates": count, "planted_entries_found": found, "planted_entries": len(pl),
                         "other_candidates": count - found,
                         "planted_median_estimate_without_diagonal": float(pe2.median()),
                         "note": "thresholded decode without a dense n x n output; the threshold timing "
                                 "includes the host read of the count"}
    # cuBLAS SGEMM of the same shapes (A^T A), context only
    torch.matmul(X.T, X)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(5):
        torch.matmul(X.T, X)
    e1.record(stream)
    torch.cuda.synchronize()
    sg = e0.elapsed_time(e1) / 5
    out["sgemm"] = {"ms": sg, "tflops": 2.0 * n * n * m / (sg * 1e-3) / 1e12,
                    "note": "torch.matmul fp32 (cuBLAS, TF32 off by default) of X^T X"}
    del Xd, wsp, c64, AB
    torch.cuda.empty_cache()
    out["plain_method"] = plain_method_context(cms, torch, dev)
    out["sparse_exact"] = sparse_context(cms, torch, dev)
    out["batched"] = batched_context(cms, torch, dev)
    out["large"] = large_context(cms, torch, dev)
    return out


def plain_method_context(cms, torch, dev):
    """The plain-method shape: A, B 256 x 256 FP64 with i.i.d. N(0, 1)
    entries, b = 1024, d = 1; the fused path (FP64 storage read as such) and
    the plain FP64 form, per product, with a new hash draw per call."""
    import workloads as W
    n, b = 256, 1024
    A = torch.from_numpy(np.ascontiguousarray(W.gaussian(n, n, 1).T)).to(dev).T
    B = torch.from_numpy(W.gaussian(n, n, 2)).to(dev)
    h = cms.make_hashes(1, n, b, 1)
    ws = cms.alloc_workspace(cms.workspace_size(h, n, n, n, torch.float64), dev)
    wsp = cms.alloc_workspace(cms.plain_workspace_size(h, n, n, n), dev)
    c = torch.empty((1, b), dtype=torch.float32, device=dev)
    c64 = torch.empty((1, b), dtype=torch.float64, device=dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 50
    res = {}
    for name, run in (("fused", lambda i: cms.sketch_product(A, B, h, c=c, ws=ws)),
                      ("plain_f64", lambda i: cms.sketch_product_plain_f64(A, B, h, c=c64, ws=wsp))):
        for i in range(3):
            h.reseed(1 + i)
            run(i)
        torch.cuda.synchronize()
        e0.record()
        for i in range(reps):
            h.reseed(100 + i)
            run(i)
        e1.record()
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / reps
    h.reseed(1)
    cms.sketch_product(A, B, h, c=c, ws=ws)
    cms.sketch_product_plain_f64(A, B, h, c=c64, ws=wsp)
    rel = float(torch.linalg.norm(c.double() - c64) / torch.linalg.norm(c64))
    h.free()
    return {"workload": "plain method A, B 256x256 FP64 N(0,1), b=1024, d=1",
            "fused_ms_per_product": res["fused"], "plain_f64_ms_per_product": res["plain_f64"],
            "c_rel_l2_fused_vs_plain": rel,
            "note": "hash draw included in each call's time; launch-bound at this size"}


def sparse_context(cms, torch, dev):
    """Exact sparse product: n = 2^20, 256 blocks (8 inner indices, 32 rows of
    A, 32 columns of B), integer values, b = 2^20, d = 3; A CSC, B CSR."""
    import workloads as W
    n, b, d = 1 << 20, 1 << 20, 3
    sb = W.sparse_blocks(n, n_blocks=256, inner=8, rows=32, cols=32, seed=3)
    T = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)   # noqa: E731
    args = (T(sb.a_colptr, torch.int64), T(sb.a_rowidx, torch.int32), T(sb.a_val, torch.float32),
            T(sb.b_rowptr, torch.int64), T(sb.b_colidx, torch.int32), T(sb.b_val, torch.float32))
    h = cms.make_hashes(3, n, b, d)
    ws = cms.alloc_workspace(cms.sparse_workspace_size(h, n, n, n), dev)
    c = torch.empty((d, b), dtype=torch.float32, device=dev)
    cms.sketch_product_csr(*args, n, n, h, c=c, ws=ws)
    torch.cuda.synchronize()
    reps = 5
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    for _ in range(reps):
        cms.sketch_product_csr(*args, n, n, h, c=c, ws=ws)   # no host wait inside the call
    e1.record()
    host_ms = (time.perf_counter() - t0) * 1e3 / reps
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    K = 256 * 8
    flops = d * K * (5.0 * b * math.log2(b) + 4.0 * b) + d * 2.5 * b * math.log2(b)
    # sparse-k hybrid (default split): every outer product here has 1024
    # terms, so all 2048 inner indices are sketched directly
    ch = torch.empty_like(c)
    cms.sketch_product_csr(*args, n, n, h, c=ch, ws=ws, direct_max_pairs=-1)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        cms.sketch_product_csr(*args, n, n, h, c=ch, ws=ws, direct_max_pairs=-1)
    e1.record()
    torch.cuda.synchronize()
    ms_h = e0.elapsed_time(e1) / reps
    same = bool(torch.equal(torch.round(c), torch.round(ch)))
    # the direct route sums exact FP64 products of the integer values, so its
    # c is the exact sketch: the FFT route's rounding error against it
    err = torch.linalg.norm((c.double() - ch.double()), dim=1) / torch.linalg.norm(ch.double(), dim=1)
    h.free()
    return {"workload": "exact sparse n=2^20, 256 blocks x (8 inner, 32 rows, 32 cols), b=2^20, d=3",
            "ms_per_product": ms, "products_per_s": 1e3 / ms, "nonempty_k": K,
            "alg_tflops": flops / (ms * 1e-3) / 1e12, "host_ms_per_call": host_ms,
            "c_rel_l2_vs_exact": float(err.max()),
            "c_max_abs_err_vs_exact": float((c.double() - ch.double()).abs().max()),
            "note": "FFT route, CUDA events (the call does not wait for the device); error against the "
                    "direct route's exact sketch of the integer product",
            "hybrid": {"ms_per_product": ms_h, "products_per_s": 1e3 / ms_h,
                       "direct_terms": d * K * 32 * 32, "rounded_c_equal_to_fft_route": same,
                       "note": "sparse-k hybrid, default split (all inner indices direct, FP64 scatter); "
                               "not an FFT-route roofline number"}}


def large_context(cms, torch, dev):
    """Large covariance product at full size: X 16384 x 32768 stored as BF16
    (N(0, 1), 4096 planted pairs of correlation 0.3), A = X^T, B = X,
    b = 2^20, d = 7.  Runs the cluster kernel (rows of 2^16 bins)."""
    m, n, b, d, npairs, rho = 16384, 32768, 1 << 20, 7, 4096, 0.3
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    X = torch.randn((m, n), generator=gen, device=dev, dtype=torch.float32)
    perm = torch.randperm(n, generator=gen, device=dev)[: 2 * npairs].view(-1, 2)
    z = torch.randn((m, npairs), generator=gen, device=dev)
    X[:, perm[:, 1]] = rho * X[:, perm[:, 0]] + math.sqrt(1 - rho ** 2) * z
    Xb = X.to(torch.bfloat16)
    del X, z
    torch.cuda.empty_cache()
    h = cms.make_hashes(5, n, b, d)
    ws = cms.alloc_workspace(cms.workspace_size(h, n, m, n, torch.bfloat16), dev)
    c = torch.empty((d, b), dtype=torch.float32, device=dev)
    cms.profile_enable(True)
    cms.sketch_product(Xb.T, Xb, h, c=c, ws=ws)          # warm-up, and the kernel list
    torch.cuda.synchronize()
    kernels = cms.profile_summary()
    cms.profile_enable(False)
    reps = 2
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        cms.sketch_product(Xb.T, Xb, h, c=c, ws=ws)
    e1.record()
    torch.cuda.synchronize()
    cms.check_async()
    ms = e0.elapsed_time(e1) / reps
    flops = total_flops(d, m, b)
    pe = cms.decode(c, h, perm.to(torch.int64))
    out = {"workload": "large covariance X 16384x32768 BF16, 4096 pairs rho=0.3, b=2^20, d=7",
           "ms_per_product": ms, "products_per_s": 1e3 / ms, "alg_tflops": flops / (ms * 1e-3) / 1e12,
           "kernels": sorted(kernels),
           "planted_pairs": {"count": npairs, "median_estimate": float(pe.median()), "expected": rho * m}}
    # the plain FP64 form on the first ks inner indices (cost linear in them),
    # and the fused path's rounding error against it on the same sample
    ks = 2048
    Xs = Xb[:ks]
    Xd = Xs.double()
    c32 = cms.sketch_product(Xs.T, Xs, h)
    wsp = cms.alloc_workspace(cms.plain_workspace_size(h, n, ks, n), dev)
    c64 = cms.sketch_product_plain_f64(Xd.T, Xd, h, ws=wsp)
    torch.cuda.synchronize()
    e0.record()
    cms.sketch_product_plain_f64(Xd.T, Xd, h, c=c64, ws=wsp)
    e1.record()
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) * (m / ks)
    rel = torch.linalg.norm(c32.double() - c64, dim=1) / torch.linalg.norm(c64, dim=1)
    out["plain_f64"] = {"ms_per_product": plain_ms, "products_per_s": 1e3 / plain_ms,
                        "note": f"timed on the first {ks} of {m} inner indices, scaled (the cost is linear in them)"}
    out["rounding_error"] = {"c_rel_l2_vs_plain_f64": float(rel.max()),
                             "compared": f"all {d} x {b} buckets of the sketch of X[:{ks}] (BF16 values)"}
    del Xd, wsp, c64, c32
    # sketch standard deviation ||AB||_F / sqrt(b) of the full product, and
    # cuBLAS SGEMM of the same shapes for context
    X32 = Xb.float()
    G = torch.matmul(X32.T, X32)
    torch.cuda.synchronize()
    e0.record()
    torch.matmul(X32.T, X32, out=G)
    e1.record()
    torch.cuda.synchronize()
    sg = e0.elapsed_time(e1)
    out["sketch_std"] = float(torch.linalg.norm(G)) / math.sqrt(b)
    out["sgemm"] = {"ms": sg, "tflops": 2.0 * n * n * m / (sg * 1e-3) / 1e12,
                    "note": "torch.matmul fp32 (cuBLAS) of X^T X, X the BF16 values widened"}
    h.free()
    del Xb, ws, c, X32, G
    torch.cuda.empty_cache()
    return out


def batched_context(cms, torch, dev, n_hi: int = 8192):
    """64 covariance-shaped instances of uneven n (log-uniform in [512, n_hi],
    5-smooth), m = 2n, half FP32 / half BF16 storage, b = 16 n, d = 3: one
    batch through a CUDA graph vs one plain FP64 launch per instance."""
    import workloads as W
    specs = W.batched_specs(64, seed=4, n_lo=512, n_hi=n_hi)
    gen = torch.Generator(device=dev)
    items, xs = [], []
    for q, sp in enumerate(specs):
        gen.manual_seed(sp.seed)
        X = torch.randn((sp.m, sp.n), generator=gen, device=dev, dtype=torch.float32)
        if sp.n_pairs:
            perm = torch.randperm(sp.n, generator=gen, device=dev)[: 2 * sp.n_pairs].view(-1, 2)
            z = torch.randn((sp.m, sp.n_pairs), generator=gen, device=dev)
            X[:, perm[:, 1]] = sp.rho * X[:, perm[:, 0]] + math.sqrt(1 - sp.rho ** 2) * z
        Xs = X.to(torch.bfloat16) if sp.dtype == "bf16" else X
        h = cms.make_hashes(1000 + q, sp.n, 16 * sp.n, 3)
        items.append((Xs.T, Xs, h))
        xs.append(X)
    batch = cms.Batch(items)
    info = batch.info()
    s = torch.cuda.Stream()
    batch.run_graph(s)                 # capture + first replay
    s.synchronize()
    reps = 5
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        batch.run_graph(s)
    e1.record(s)
    s.synchronize()
    graph_ms = e0.elapsed_time(e1) / reps
    # plain FP64 form: one call per instance
    plain_ms = 0.0
    errs = []
    for q, ((A, B, h), X) in enumerate(zip(items, xs)):
        # the plain form of the values the batch read (BF16 instances widened)
        Xd = B.double()
        ws = cms.alloc_workspace(cms.plain_workspace_size(h, X.shape[1], X.shape[0], X.shape[1]), dev)
        c64 = cms.sketch_product_plain_f64(Xd.T, Xd, h, ws=ws)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        a.record()
        cms.sketch_product_plain_f64(Xd.T, Xd, h, c=c64, ws=ws)
        z.record()
        torch.cuda.synchronize()
        plain_ms += a.elapsed_time(z)
        cq = batch.c[q].double()
        errs.append(float((torch.linalg.norm(cq - c64, dim=1) / torch.linalg.norm(c64, dim=1)).max()))
        del Xd, ws, c64
    flops = sum(3 * sp.m * (5.0 * 16 * sp.n * math.log2(16 * sp.n) + 4.0 * 16 * sp.n) for sp in specs)
    batch.free()
    for _, _, h in items:
        h.free()
    torch.cuda.empty_cache()
    return {"workload": f"64 covariance instances, n log-uniform [512, {n_hi}] 5-smooth, m=2n, 32 FP32 + 32 BF16, "
                        "b=16n, d=3", "instances": info["instances"], "tasks": info["tasks"],
            "kernel_launches_per_run": info["launches"], "fast_kernel_instances": info["fast_instances"],
            "graph_ms_per_batch": graph_ms, "products_per_s": 64 * 1e3 / graph_ms,
            "alg_tflops": flops / (graph_ms * 1e-3) / 1e12,
            "plain_f64_ms_per_batch": plain_ms, "plain_f64_products_per_s": 64 * 1e3 / plain_ms,
            "rounding_error": {"c_rel_l2_vs_plain_f64_max": max(errs), "c_rel_l2_vs_plain_f64_median":
                               statistics.median(errs),
                               "note": "per instance, the batch's c against the plain FP64 form of the same "
                                       "stored values (max over the repetitions)"}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["cms", "reference"], default="cms")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-context", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--shard", choices=["products", "k"], default="products",
                    help="products: every GPU computes whole, independent products (weak scaling); "
                         "k: the GPUs share one product, each sketching its range of inner indices, "
                         "the partial sketches merged in rank order (strong scaling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    elif args.shard == "k":
        gpu_arm_kshard(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
