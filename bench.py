#!/usr/bin/env python3
"""Throughput benchmark of the IMDP abstraction build on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the 5-D room-temperature system (x+ = A x + B u + 1.8 + w, A = 0.85 I
+ 0.03 ring, [17,23]^5 on an 11^5 grid, 9 inputs, sigma 0.2, cutoff 1e-8),
FP32-sound bounds with FP64 row terms. One step is one whole build through
the C ABI: the count pass (per-row counts, sink, truncated mass, row checks),
the row-pointer scan and the emit pass (col/lo/up). Inputs are synthetic and
seeded; the output (~33 GB) is far larger than L2, and L2 is also flushed
between timed steps.

The JSON line reports pairs/s (value), the emit kernel against the measured
HBM copy bandwidth (roofline), the end-to-end rate with the CSR read back to
pinned host memory (e2e), the FP64-plain GPU path on the same workload, and
the CPU oracle timed on a bounded sample of rows (cpu_baseline).

With N > 1 (torchrun, one process per GPU) every rank builds its own copy of
the workload: the rows of independent builds need no exchange, so the run
scales weakly and `value` is the pairs of all ranks over the slowest rank's
time. `--impl reference` times the CPU oracle instead (rank 0 only).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IMDP lo/up bound pairs/sec, FP32-sound vs FP64 plain; served p50/p99 latency"
UNIT = "pairs/s"


def workload_name(cells=11):
    return ("5-D room temperature: A=0.85I+0.03 ring, B on rooms 1,3,5 / 2,4, c=1.8, "
            f"[17,23]^5 on {cells}^5 cells, inputs {{0,0.5,1}}^2, sigma 0.2, cutoff 1e-8, "
            "FP32-sound")


WORKLOAD = workload_name()
# kernels one count + emit step launches: setup, prep, tree count, three scan
# stages, tree emit
LAUNCHES_PER_STEP = 7
L2_FLUSH_BYTES = 512 << 20


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64-plain comparison")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--cpu-rows", type=int, default=0, help="oracle sample size (0: auto)")
    p.add_argument("--cells", type=int, default=11,
                   help="cells per dimension (11 = the benchmark workload; smaller values "
                        "give the reduced case used for detailed kernel profiles)")
    return p.parse_args(argv)


# --------------------------------------------------------------------------
# distributed plumbing (one process per GPU; no data-path collective)
# --------------------------------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init_dist(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over all ranks (the slowest rank's time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device=None) -> float:
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------------------
# clocks sampled while the timed region runs
# --------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# measured peaks
# --------------------------------------------------------------------------

def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def emit_traffic(alg_bytes):
    """DRAM bytes of one emit launch, from the committed ncu summary.

    The summary records the DRAM traffic per algorithmic byte of the emit
    kernel and the hash of the source it was captured on; the figure is used
    only while that source is unchanged (None otherwise)."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "room5d_fp32_tree_kernels_ncu.txt")
    src = os.path.join(ROOT, "paper_2401_03555_gb300", "csrc", "tree_fp32.cu")
    try:
        text = open(prof).read()
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    want, ratio = None, None
    for line in text.splitlines():
        if "sha256 prefix" in line:
            want = line.split("sha256 prefix")[1].strip().rstrip(".").split()[0]
        if line.strip().startswith("traffic_bytes_per_algorithmic_byte:"):
            ratio = float(line.split(":")[1])
    if want is None or ratio is None or not digest.startswith(want):
        return None
    return int(ratio * alg_bytes)


# --------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# --------------------------------------------------------------------------

def cpu_oracle_sample(prob, rows_target: int, seed: int = 0):
    """Time the CPU oracle on a seeded sample of rows; returns a dict."""
    import oracle
    orc = oracle.default()
    threads = orc.max_threads()
    rows = np.sort(np.random.default_rng(seed).choice(prob.rows, size=rows_target, replace=False))
    t0 = time.perf_counter()
    res = orc.build_rows(prob, rows)
    dt = time.perf_counter() - t0
    return {"value": res.nnz / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{len(rows)} seeded random rows of the {prob.rows} (dense scan of "
                      f"{prob.total_cells} targets per row), {res.nnz} pairs in {dt:.2f} s",
            "rows_per_s": len(rows) / dt, "seconds": dt}


def auto_cpu_rows(prob):
    """About 10-30 s of oracle work on this host (each row is a dense scan)."""
    import oracle
    threads = max(1, oracle.default().max_threads())
    per_row_s = 0.17 * prob.total_cells / 161051.0 * prob.n / 5.0
    return int(max(threads, min(4096, 15.0 * threads / max(per_row_s, 1e-6))))


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2401_03555_gb300 import impact, workloads as W
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    init_dist(world, "nccl")
    prob = W.room_5d(cells_per_dim=args.cells)
    rows = prob.rows

    # exact sizes from one build, then caller-owned buffers reused every step
    first = impact.build(prob, "fp32")
    nnz = first.nnz
    del first
    torch.cuda.empty_cache()
    rbuf = impact.alloc_rows(rows, dev)
    pbuf = impact.alloc_pairs(nnz, "fp32", dev)
    wbuf = impact.alloc_workspace(prob, "fp32", dev)
    args_c = impact._Args(prob)
    lib = impact.load()
    import ctypes
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sh = ctypes.c_void_p(int(stream.cuda_stream))

    def step():
        c = impact._csr_struct(rbuf, pbuf, capacity=nnz, workspace=wbuf)
        s = lib.impact_count(ctypes.byref(args_c.sys), ctypes.byref(args_c.grid),
                             ctypes.byref(args_c.inp), args_c.sigma_ptr, args_c.cutoff,
                             impact.FP32_SOUND, ctypes.byref(c), sh)
        impact._check(s)
        mid.record(stream)
        c.nnz = nnz
        impact._check(lib.impact_emit(ctypes.byref(args_c.sys), ctypes.byref(args_c.grid),
                                      ctypes.byref(args_c.inp), args_c.sigma_ptr, args_c.cutoff,
                                      impact.FP32_SOUND, ctypes.byref(c), sh))
        return int(c.nnz)

    for _ in range(args.warmup):
        mid = torch.cuda.Event(enable_timing=True)
        step()
    torch.cuda.synchronize(dev)

    step_ms, emit_ms = [], []
    barrier(world)
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter()
    with ClockSampler(local_rank) as clocks:
        for _ in range(args.steps):
            flush.fill_(1.0)                      # evict L2 between steps
            s = torch.cuda.Event(enable_timing=True)
            mid = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record(stream)
            got = step()
            e.record(stream)
            e.synchronize()
            assert got == nnz
            step_ms.append(s.elapsed_time(e))
            emit_ms.append(mid.elapsed_time(e))
        torch.cuda.synchronize(dev)
    barrier(world)
    wall_s = time.perf_counter() - t_wall
    ms_local = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms_local, world, dev)
    total_pairs = sum_over_ranks(float(nnz), world, dev)
    value = total_pairs / (ms / 1e3)

    # roofline of the emit kernel: algorithmic bytes = 12 B per pair written
    # (int32 col + f32 lo + f32 up) + 16 B per row read (two row pointers)
    peak, peak_kind = hbm_peak()
    emit_avg = sum(emit_ms) / len(emit_ms)
    alg_bytes = nnz * 12 + rows * 16
    achieved = alg_bytes / (emit_avg / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": emit_traffic(alg_bytes),
                "kernel": "tree_fp32<emit>", "peak_source": peak_kind,
                "traffic_source": "ncu dram__bytes_read+write of the emit kernel on the 7^5-cell "
                                  "case, scaled per algorithmic byte "
                                  "(profiles/room5d_fp32_tree_kernels_ncu.txt)",
                "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": round(emit_avg, 3)}
    clk = clocks.summary()

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": workload_name(args.cells), "rows": rows, "pairs_per_step": nnz,
                      "parallelism": f"replicas{world}" if world > 1 else "single",
                      "l2": f"flushed between steps (512 MiB write); output {nnz * 12 / 1e9:.1f} GB"},
           "roofline": roofline, "clocks": clk,
           "gpu_launches": LAUNCHES_PER_STEP * args.steps, "wall_s": round(wall_s, 3)}
    del pbuf, flush, wbuf
    torch.cuda.empty_cache()

    # FP64-plain GPU path on the same workload (one build, rank-local)
    if not args.no_fp64 and rank == 0:
        torch.cuda.synchronize(dev)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        c64 = impact.build(prob, "fp64")
        e.record(stream)
        e.synchronize()
        ms64 = s.elapsed_time(e)
        out["fp64_plain"] = {"value": c64.nnz / (ms64 / 1e3), "unit": UNIT, "ms": ms64,
                             "pairs": c64.nnz, "fp32_over_fp64": value / world / (c64.nnz / (ms64 / 1e3))}
        del c64
        torch.cuda.empty_cache()

    # end to end through the public API with the CSR read back to pinned host memory
    if not args.no_e2e:
        out["e2e"] = run_e2e(prob, nnz, dev, stream, world, steps=max(1, min(args.steps, 3)))

    if rank == 0 and not args.no_cpu:
        try:
            n_rows = args.cpu_rows or auto_cpu_rows(prob)
            out["cpu_baseline"] = cpu_oracle_sample(prob, n_rows)
        except Exception as exc:  # the oracle is a baseline, not the product
            out["cpu_baseline"] = {"value": None, "error": str(exc)[:200]}
    return out


def run_e2e(prob, nnz, dev, stream, world, steps=3):
    import torch
    from paper_2401_03555_gb300 import impact
    b = impact.Builder(prob, "fp32", capacity=nnz)
    rb, pb = b.rows_buf, b.pairs_buf
    host = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in
            list(rb.items()) + list(pb.items())}
    d2h = sum(v.numel() * v.element_size() for v in host.values())
    h2d = impact_blob_bytes(prob)
    times = []
    for it in range(steps + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        got = b.run(stream)
        for k, v in list(rb.items()) + list(pb.items()):
            host[k].copy_(v, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
        dt = time.perf_counter() - t0
        if it > 0:
            times.append(dt)
    t = max_over_ranks(sum(times) / len(times), world, dev)
    total = sum_over_ranks(float(got), world, dev)
    return {"value": total / t, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": t * 1e3,
            "path": "impact_build (C ABI) + cudaMemcpy of row_ptr/col/lo/up/sink/trunc/flags "
                    "into pinned host buffers, synchronized"}


def impact_blob_bytes(prob):
    """Bytes the planner uploads per build (descriptor + tables), from impact_plan."""
    from paper_2401_03555_gb300 import impact
    rows, bound, nbytes = impact.plan(prob, "fp32")
    per_pair = 12
    return int(nbytes - bound * per_pair - (rows + 1) * 8 - rows * 28)


# --------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# --------------------------------------------------------------------------

def run_reference(args, rank, world):
    from paper_2401_03555_gb300 import workloads as W
    if rank != 0:
        return None
    prob = W.room_5d()
    n_rows = args.cpu_rows or max(16, auto_cpu_rows(prob) // max(1, args.steps + args.warmup))
    for w in range(args.warmup):
        cpu_oracle_sample(prob, n_rows, seed=1000 + w)
    samples = [cpu_oracle_sample(prob, n_rows, seed=s) for s in range(args.steps)]
    pairs = sum(float(s["value"]) * s["seconds"] for s in samples)
    secs = sum(s["seconds"] for s in samples)
    value = pairs / secs
    cb = dict(samples[0])
    cb["value"] = value
    cb["sample"] = f"{args.steps} steps of {n_rows} seeded random rows each"
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD.replace("FP32-sound", "FP64 CPU oracle")},
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}


def main(argv=None):
    args = parse_args(argv)
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
