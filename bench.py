#!/usr/bin/env python3
"""Throughput benchmark of the IMDP abstraction build on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the 5-D room-temperature system (x+ = A x + B u + 1.8 + w, A = 0.85 I
+ 0.03 ring, [17,23]^5 on an 11^5 grid, 9 inputs, sigma 0.2, cutoff 1e-8),
FP32-sound bounds with FP64 row terms. One step is one whole build replayed
from a CUDA graph made through the C ABI: the setup pass (per-row records,
sink bounds, mass outside the window box), the count pass (per-row counts,
truncated mass, row checks), the row-pointer scan and the emit pass
(col/lo/up). Inputs are synthetic and seeded; the output (~33 GB) is far
larger than L2, and L2 is also flushed between timed steps.

The JSON line reports pairs/s (value), the emit kernel (the step's largest)
against the measured HBM copy bandwidth (roofline, with the whole step's
fraction as step_frac), the end-to-end rate with the CSR read back to pinned
host memory (e2e), the FP64-plain GPU path on the same workload, and the CPU
oracle timed on a bounded sample of rows (cpu_baseline).

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
# kernels one step launches: setup, count walk, three scan kernels, emit walk
# (the graph's resets are memset nodes, not kernels)
LAUNCHES_PER_STEP = 6
# FP64 rate of the GB300 FMA pipe, measured with a dependent-chain DFMA
# probe (2 flops per DFMA): the bound of the FP64-plain path
FP64_PEAK_GFLOPS = 1200.0
L2_FLUSH_BYTES = 512 << 20


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64-plain comparison")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    p.add_argument("--e2e-mode", choices=["copy", "direct"], default="copy",
                   help="read-back of the end-to-end measurement: device build + copies, or "
                        "pairs written by the kernel straight into pinned host memory")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-serve", action="store_true",
                   help="skip the served stream (Poisson arrivals, continuous batching)")
    p.add_argument("--no-synth", action="store_true",
                   help="skip the controller-synthesis measurement (interval iteration)")
    p.add_argument("--no-batched", action="store_true",
                   help="skip the batched workload (256 seeded systems, graphs, autotuner)")
    p.add_argument("--cpu-rows", type=int, default=0, help="oracle sample size (0: auto)")
    p.add_argument("--case", choices=["synth", "regions", "mc", "walk", "fp64", "batched"],
                   default=None,
                   help="run one small invocation of that leg and exit (a target for "
                        "profilers; prints no JSON line)")
    p.add_argument("--systems", type=int, default=16,
                   help="--case batched: the first this many systems of the batched workload")
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


def profile_figure(profile, source, key):
    """A figure recorded in a committed ncu summary (a "key: value" line), or
    None. The summary records the sha256 prefix of the kernel source it was
    captured on; the figure is used only while that source is unchanged."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", profile)
    src = os.path.join(ROOT, "paper_2401_03555_gb300", "csrc", source)
    try:
        text = open(prof).read()
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    want, val = None, None
    for line in text.splitlines():
        if "sha256 prefix" in line:
            want = line.split("sha256 prefix")[1].strip().rstrip(".").split()[0]
        if line.strip().startswith(key + ":"):
            val = float(line.split(":")[1])
    if want is None or val is None or not digest.startswith(want):
        return None
    return val


def walk_traffic(alg_bytes):
    """DRAM bytes of one launch of the emit kernel: the traffic per algorithmic
    byte from the committed ncu summary, scaled to this launch."""
    r = profile_figure("room5d_fp32_walk_ncu.txt", "walk_fp32.cu",
                       "traffic_bytes_per_algorithmic_byte")
    return None if r is None else int(r * alg_bytes)


def fp64_roofline(pairs, ms):
    """The FP64-plain build against the FP64 pipe: its FP64 flops per pair
    (2 per DFMA + DADD + DMUL, counted by ncu over both passes on the 7^5 room)
    times the pairs, over the build's time."""
    f = profile_figure("room5d_fp64_rows_ncu.txt", "kernels.cu", "fp64_flops_per_pair")
    out = {"bound": "fp64", "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
           "peak_source": "measured (dependent-chain DFMA probe on GB300)",
           "flops_per_pair": f}
    if f is None:
        out.update({"achieved": None, "frac": None})
    else:
        ach = f * pairs / (ms / 1e3) / 1e9
        out.update({"achieved": round(ach, 1), "frac": round(ach / FP64_PEAK_GFLOPS, 4)})
    return out


def run_two_pass(prob, nnz, rbuf, pbuf, wbuf, flush, stream, dev, reps=3):
    """impact_count then impact_emit (the two-call path for callers that size
    their arrays from the count), each pass timed with CUDA events."""
    import ctypes
    import torch
    from paper_2401_03555_gb300 import impact
    a = impact._Args(prob)
    lib = impact.load()
    sh = ctypes.c_void_p(int(stream.cuda_stream))
    cms, ems = [], []
    for it in range(reps + 1):
        flush.fill_(1.0)
        s, m, e = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        c = impact._csr_struct(rbuf, pbuf, capacity=nnz, workspace=wbuf)
        s.record(stream)
        impact._check(lib.impact_count(ctypes.byref(a.sys), ctypes.byref(a.grid),
                                       ctypes.byref(a.inp), a.sigma_ptr, a.cutoff,
                                       impact.FP32_SOUND, ctypes.byref(c), sh))
        m.record(stream)
        c.nnz = nnz
        impact._check(lib.impact_emit(ctypes.byref(a.sys), ctypes.byref(a.grid),
                                      ctypes.byref(a.inp), a.sigma_ptr, a.cutoff,
                                      impact.FP32_SOUND, ctypes.byref(c), sh))
        e.record(stream)
        e.synchronize()
        if it > 0:
            cms.append(s.elapsed_time(m))
            ems.append(m.elapsed_time(e))
    peak, _ = hbm_peak()
    cm, em = sum(cms) / len(cms), sum(ems) / len(ems)
    emit_bytes = nnz * 12 + prob.rows * 16
    return {"count_ms": round(cm, 3), "emit_ms": round(em, 3), "step_ms": round(cm + em, 3),
            "value": nnz / ((cm + em) / 1e3), "unit": UNIT,
            "emit_frac": round(emit_bytes / (em / 1e3) / 1e9 / peak, 4),
            "path": "impact_count (setup, walk COUNT: per-row counts and row terms, scan) + "
                    "impact_emit (walk EMIT at those row pointers), each synchronized"}


def oracle_sample_rows(prob, rows_target: int, seed: int = 0):
    """The seeded row sample the oracle baseline times."""
    return np.sort(np.random.default_rng(seed).choice(prob.rows, size=rows_target, replace=False))


def fetch_rows(rbuf, pbuf, rows):
    """The GPU CSR of the given rows, copied to the host."""
    rp = rbuf["row_ptr"].cpu().numpy()
    out = {"row_ptr": rp, "rows": rows}
    spans = [(int(rp[r]), int(rp[r + 1])) for r in rows]
    for k in ("col", "lo", "up"):
        out[k] = [pbuf[k][a:b].cpu().numpy() for a, b in spans]
    for k in ("sink_lo", "sink_up", "trunc"):
        out[k] = rbuf[k].cpu().numpy()[rows]
    return out


def sample_parity(prob, gpu, ref):
    """The GPU rows against the oracle's on the same rows: largest
    differences and the FP32-sound bracketing (the parity test's rules)."""
    dlo = dup = 0.0
    bracket = True
    missing = 0
    for k in range(len(gpu["rows"])):
        oc, olo, oup = ref.row(k)
        gc = gpu["col"][k]
        _, gi, oi = np.intersect1d(gc, oc, return_indices=True)
        missing += len(oc) - len(oi)
        lo = gpu["lo"][k].astype(np.float64)[gi]
        up = gpu["up"][k].astype(np.float64)[gi]
        if len(gi):
            dlo = max(dlo, float(np.max(np.abs(lo - olo[oi]))))
            dup = max(dup, float(np.max(np.abs(up - oup[oi]))))
            bracket &= bool(np.all(lo <= olo[oi]) and np.all(up >= oup[oi]))
        extra = np.setdiff1d(np.arange(len(gc)), gi)
        bracket &= bool(np.all(gpu["up"][k][extra] >= prob.cutoff))
    dsl = float(np.max(np.abs(gpu["sink_lo"] - ref.sink_lo)))
    dsu = float(np.max(np.abs(gpu["sink_up"] - ref.sink_up)))
    dtr = float(np.max(np.abs(gpu["trunc"] - ref.trunc)))
    bracket &= bool(np.all(gpu["sink_lo"] <= ref.sink_lo) and np.all(gpu["sink_up"] >= ref.sink_up))
    ok = bracket and missing == 0 and max(dlo, dup, dsl, dsu, dtr) <= 2e-6
    return {"rows": len(gpu["rows"]), "max_dlo": dlo, "max_dup": dup,
            "max_dsink": max(dsl, dsu), "max_dtrunc": dtr, "missing_pairs": int(missing),
            "bracketing": bracket, "within_2e-6": ok}


# --------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# --------------------------------------------------------------------------

def cpu_oracle_sample(prob, rows_target: int, seed: int = 0, threads: int = 0, keep=False):
    """Time the CPU oracle on a seeded sample of rows (all OpenMP threads, or
    `threads` of them); returns a dict (and the oracle's rows with keep)."""
    import oracle
    orc = oracle.default()
    threads = threads or orc.max_threads()
    rows = oracle_sample_rows(prob, rows_target, seed)
    t0 = time.perf_counter()
    res = orc.build_rows(prob, rows, threads=threads)
    dt = time.perf_counter() - t0
    out = {"value": res.nnz / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{len(rows)} seeded random rows of the {prob.rows} (dense scan of "
                     f"{prob.total_cells} targets per row), {res.nnz} pairs in {dt:.2f} s",
           "rows_per_s": len(rows) / dt, "seconds": dt,
           "full_build_s_extrapolated": round(prob.rows / (len(rows) / dt), 1)}
    return (out, res) if keep else out


def auto_cpu_rows(prob):
    """About 10-30 s of oracle work on this host (each row is a dense scan).
    The thread count is the one OpenMP will use, read without loading the
    oracle: loading it starts the OpenMP runtime, after which the end-to-end
    leg's pinned host buffers measured half the copy bandwidth."""
    threads = int(os.environ.get("OMP_NUM_THREADS", "0") or 0) or len(os.sched_getaffinity(0))
    threads = max(1, threads)
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
    nnz = impact.build(prob, "fp32").nnz
    torch.cuda.empty_cache()
    rbuf = impact.alloc_rows(rows, dev)
    pbuf = impact.alloc_pairs(nnz, "fp32", dev)
    wbuf = impact.alloc_workspace(prob, "fp32", dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # one step = the whole build replayed from a CUDA graph: the setup kernel
    # (every row's record, sink bounds, outside-window mass), the count walk,
    # the scan of the counts into row pointers and the emit walk, with the
    # resets of the status and row-counter words as memset nodes
    graph = impact.Batch([prob], "fp32").graph(rbuf, pbuf, nnz, wbuf, stream)

    def step():
        graph.launch(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    assert graph.result() == nnz

    step_ms = []
    barrier(world)
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter()
    with ClockSampler(local_rank) as clocks:
        for _ in range(args.steps):
            flush.fill_(1.0)                      # evict L2 between steps
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record(stream)
            step()
            e.record(stream)
            e.synchronize()
            step_ms.append(s.elapsed_time(e))
        torch.cuda.synchronize(dev)
    barrier(world)
    wall_s = time.perf_counter() - t_wall
    assert graph.result() == nnz
    ms_local = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms_local, world, dev)
    total_pairs = sum_over_ranks(float(nnz), world, dev)
    value = total_pairs / (ms / 1e3)

    clk = clocks.summary()

    # the two-call path (impact_count, then impact_emit at its row pointers):
    # each pass timed on its own with CUDA events on the launching stream; the
    # emit pass is the step's largest kernel (its share of the launch list is
    # in profiles/room5d_fp32_launch_list.txt)
    two = run_two_pass(prob, nnz, rbuf, pbuf, wbuf, flush, stream, dev)

    # roofline of the emit kernel: algorithmic bytes = 12 B per pair written
    # (int32 col + f32 lo + f32 up) + 16 B per row (row_ptr read, two 8-byte
    # words); step_frac: the whole step's algorithmic bytes, 12 B per pair +
    # 36 B per row written (row_ptr, sink_lo, sink_up, trunc: 8 each;
    # row_flags 4), over ms_per_step
    peak, peak_kind = hbm_peak()
    emit_bytes = nnz * 12 + rows * 16
    achieved = emit_bytes / (two["emit_ms"] / 1e3) / 1e9
    step_bytes = nnz * 12 + rows * 36
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": walk_traffic(emit_bytes),
                "kernel": "walk_fp32<EMIT>", "peak_source": peak_kind,
                "traffic_source": "ncu dram__bytes_read+write of the emit kernel per algorithmic "
                                  "byte on the 7^5 room, scaled to this launch "
                                  "(profiles/room5d_fp32_walk_ncu.txt)",
                "algorithmic_bytes_per_launch": emit_bytes, "launch_ms": two["emit_ms"],
                "bytes_model": "12 B/pair written + 16 B/row read",
                "step_frac": round(step_bytes / (ms_local / 1e3) / 1e9 / peak, 4),
                "step_bytes_model": "12 B/pair + 36 B/row written, over ms_per_step",
                # every erf/erfc evaluation of the build is in setup_fp32, which
                # runs inside impact_count: the count call's time bounds it
                "erfc_term": {"kernel": "setup_fp32 (within impact_count)",
                              "ms_upper_bound": two["count_ms"],
                              "hbm_term_ms": round(emit_bytes / peak / 1e6, 3)}}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": workload_name(args.cells), "rows": rows, "pairs_per_step": nnz,
                      "sink_pairs_per_step": rows,
                      "parallelism": f"replicas{world}" if world > 1 else "single",
                      "l2": f"flushed between steps (512 MiB write); output {nnz * 12 / 1e9:.1f} GB"},
           "roofline": roofline, "clocks": clk,
           "gpu_launches": LAUNCHES_PER_STEP * args.steps, "wall_s": round(wall_s, 3)}

    out["two_pass"] = two

    # rows the oracle baseline will sample: their GPU values, kept for the
    # parity check after the oracle has run
    sample_rows = None
    if rank == 0 and not args.no_cpu:
        n_rows = args.cpu_rows or auto_cpu_rows(prob)
        sample_rows = oracle_sample_rows(prob, n_rows, seed=0)
        gpu_rows = fetch_rows(rbuf, pbuf, sample_rows)
    graph.close()
    del pbuf, flush, wbuf, rbuf
    torch.cuda.empty_cache()

    # end to end through the public API with the CSR read back to pinned host
    # memory (right after the device-timed steps, before the long legs below)
    if not args.no_e2e:
        out["e2e"] = run_e2e(prob, nnz, dev, stream, world, steps=max(1, min(args.steps, 3)),
                             mode=args.e2e_mode)
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
                             "pairs": c64.nnz, "fp32_over_fp64": value / world / (c64.nnz / (ms64 / 1e3)),
                             "roofline": fp64_roofline(c64.nnz, ms64)}
        del c64
        torch.cuda.empty_cache()

    if not args.no_batched and rank == 0:
        try:
            out["batched"] = run_batched(dev, stream)
        except Exception as exc:
            out["batched"] = {"value": None, "error": str(exc)[:300]}
        torch.cuda.empty_cache()

    if not args.no_synth and rank == 0:
        try:
            out["synthesis"] = run_synthesis()
        except Exception as exc:
            out["synthesis"] = {"value": None, "error": str(exc)[:300]}
        torch.cuda.empty_cache()
        try:
            out["regions"] = run_regions()
        except Exception as exc:
            out["regions"] = {"value": None, "error": str(exc)[:300]}
        torch.cuda.empty_cache()
        try:
            out["sampled_noise"] = run_mc()
        except Exception as exc:
            out["sampled_noise"] = {"value": None, "error": str(exc)[:300]}
        torch.cuda.empty_cache()

    if not args.no_serve and rank == 0:
        try:
            out["served"] = run_serving()
        except Exception as exc:
            out["served"] = {"value": None, "error": str(exc)[:300]}
        torch.cuda.empty_cache()

    if rank == 0 and not args.no_cpu:
        try:
            out["cpu_baseline"], ref = cpu_oracle_sample(prob, n_rows, keep=True)
            # the same rows of the timed build against the oracle
            out["cpu_baseline"]["parity"] = sample_parity(prob, gpu_rows, ref)
        except Exception as exc:  # the oracle is a baseline, not the product
            out["cpu_baseline"] = {"value": None, "error": str(exc)[:200]}
        try:   # the same oracle on one core, on a proportionally smaller sample
            cores = int(out["cpu_baseline"].get("cores") or 1)
            one = cpu_oracle_sample(prob, max(1, n_rows // max(cores, 1)), seed=1, threads=1)
            out["cpu_baseline"]["single_core"] = {k: one[k] for k in
                                                  ("value", "unit", "cores", "sample", "seconds")}
        except Exception as exc:
            out["cpu_baseline"]["single_core"] = {"value": None, "error": str(exc)[:200]}
    return out


BATCHED_WORKLOAD = ("256 seeded linear systems x+ = A x + B u + w (seeds 0..255): n in 2..5, "
                    "A = 0.9 Q D Q^T, B ~ N(0, 0.3^2), 1e3..1e5 cells log-uniform on [-1,1]^n, "
                    "2-3 input dims x 2-3 points, sigma 0.1..1 cell widths, cutoff 1e-8, "
                    "FP32-sound")


def run_batched(dev, stream, reps=2, cap_pairs=8_000_000_000):
    """The batched workload: all 256 systems counted in one batch, then built
    as groups of consecutive systems that fit `cap_pairs` of output, each group
    one persistent launch per kernel replayed from a captured CUDA graph, with
    launch shapes from the autotuner (timed against the default shapes)."""
    import torch
    from paper_2401_03555_gb300 import impact, workloads as W
    probs = W.batched_family(256)
    full = impact.Batch(probs, "fp32")
    rb = impact.alloc_rows(full.rows, dev)
    ws = full.alloc_workspace(dev)
    t0 = time.perf_counter()
    total = full.count(rb, ws, stream)
    count_all_s = time.perf_counter() - t0
    offs = torch.as_tensor(full.row_offsets, device=dev)
    rp = rb["row_ptr"]
    per = (rp[offs[1:]] - rp[offs[:-1]]).cpu().numpy()
    del ws, rb, rp
    torch.cuda.empty_cache()
    groups, cur, acc = [], [], 0
    for q, k in enumerate(per):
        if cur and acc + k > cap_pairs:
            groups.append(cur)
            cur, acc = [], 0
        cur.append(q)
        acc += int(k)
    groups.append(cur)
    gnnz = [int(sum(per[q] for q in g)) for g in groups]
    grows = [sum(probs[q].rows for q in g) for g in groups]
    pb = impact.alloc_pairs(max(gnnz), "fp32", dev)
    rbuf = impact.alloc_rows(max(grows), dev)

    def make_graphs(tune):
        batches = [impact.Batch([probs[q] for q in g], "fp32", tune=tune) for g in groups]
        wss = [b.alloc_workspace(dev) for b in batches]
        return [b.graph(rbuf, pb, k, w, stream) for b, k, w in zip(batches, gnnz, wss)], wss

    def timed(graphs):
        for g in graphs:                       # warm-up pass
            g.launch(stream)
        torch.cuda.synchronize(dev)
        ms = []
        for _ in range(reps):
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record(stream)
            for g in graphs:
                g.launch(stream)
            e.record(stream)
            e.synchronize()
            ms.append(s.elapsed_time(e))
        for g, k in zip(graphs, gnnz):         # every group built completely
            assert g.result() == k
        return min(ms)

    graphs, wss = make_graphs(None)
    ms_default = timed(graphs)
    for g in graphs:
        g.close()
    del graphs, wss
    torch.cuda.empty_cache()
    g0 = impact.Batch([probs[q] for q in groups[0]], "fp32")
    t0 = time.perf_counter()
    best, _ = g0.tune(rbuf, pb, gnnz[0], reps=2, stream=stream)
    tune_s = time.perf_counter() - t0
    graphs, wss = make_graphs(best)
    ms_tuned = timed(graphs)
    for g in graphs:
        g.close()
    del graphs, wss, pb, rbuf
    torch.cuda.empty_cache()
    peak, peak_kind = hbm_peak()
    alg_bytes = int(total) * 12 + int(full.rows) * 36
    achieved = alg_bytes / (ms_tuned / 1e3) / 1e9
    out = {"workload": BATCHED_WORKLOAD, "systems": len(probs), "rows": int(full.rows),
           "pairs": int(total), "groups": len(groups), "group_sizes": [len(g) for g in groups],
           "value": total / (ms_tuned / 1e3), "unit": UNIT, "ms_per_pass": ms_tuned,
           "ms_per_pass_default_shapes": ms_default, "tuning": best.as_dict(),
           "tune_s": round(tune_s, 2), "count_all_s": round(count_all_s, 3),
           "gpu_launches_per_pass": LAUNCHES_PER_STEP * len(groups),
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                        "unit": "GB/s", "frac": round(achieved / peak, 4),
                        "peak_source": peak_kind, "algorithmic_bytes_per_pass": alg_bytes,
                        "bytes_model": "12 B/pair + 36 B/row written",
                        "time": "every group's graph replay, back to back"},
           "path": "impact_graph_launch per group (setup, count, scan and emit, each one "
                   "persistent launch over every system of the group)"}
    out["fp64_plain"] = batched_fp64_sample(probs, dev)
    return out


def batched_fp64_sample(probs, dev, pairs_target=150_000_000):
    """FP32-sound against FP64 plain on the first systems of the batched
    workload (about `pairs_target` pairs: the FP64 plain kernel evaluates erfc
    in FP64 per pair and dimension, so the whole workload would take minutes)."""
    import torch
    from paper_2401_03555_gb300 import impact
    take, acc = [], 0
    for p in probs:
        take.append(p)
        acc += impact.plan(p, "fp32")[1]
        if acc >= pairs_target * 2:   # the plan's bound is about twice the pairs
            break
    res = {}
    for prec in ("fp32", "fp64"):
        b = impact.Batch(take, prec)
        b.build()                                 # warm-up (and sizes)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        r = b.build()
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        res[prec] = (r.csr.nnz, dt)
        del r
        torch.cuda.empty_cache()
    (n32, t32), (n64, t64) = res["fp32"], res["fp64"]
    return {"systems": len(take), "pairs_fp32": n32, "pairs_fp64": n64,
            "fp32_value": n32 / t32, "fp64_value": n64 / t64,
            "fp32_over_fp64": (n32 / t32) / (n64 / t64), "unit": UNIT,
            "path": "impact_batch_count + impact_batch_emit (library-sized arrays), "
                    "wall time of each precision"}


SYNTH_WORKLOAD = ("reach-avoid controller for the 2-D robot (21^2 cells, 9 inputs, dense "
                  "FP64 IMDP, 1.75e6 pairs): target [3,7]^2, avoid [-7,-3]^2 and the "
                  "out-of-domain sink; interval iteration to eps 1e-6, both phases")


def run_synthesis(eps=1e-6, oracle_iters=2):
    """impact_synthesize on the robot abstraction; the oracle's interval
    iteration timed on the same IMDP for a bounded number of iterations."""
    import torch
    from paper_2401_03555_gb300 import impact, workloads as W
    prob = W.robot_2d()
    target, avoid = [([3, 3], [7, 7])], [([-7, -7], [-3, -3])]
    labels = impact.label_cells(prob, target, avoid)
    csr = impact.build(prob, "fp64")
    impact.synthesize(csr, prob, labels, eps=eps)          # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = impact.synthesize(csr, prob, labels, eps=eps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    its = sum(g.iterations)
    # one iteration = both vectors' Bellman update over every row
    row_lps = 2 * prob.rows * its
    out = {"workload": SYNTH_WORKLOAD, "iterations": list(g.iterations), "ms": dt * 1e3,
           "ms_per_iteration": dt * 1e3 / its, "value": row_lps / dt, "unit": "row LPs/s",
           "p_min_max": float(g.p_min.max().item()),
           "path": "impact_synthesize (sorting-method LP by warp bisection, one warp per row, "
                   "then one thread per cell)"}
    # the same controller with the region vectors (one box relaxation per region)
    rv = impact.region_vectors(prob, target, avoid, "box", "fp64")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gr = impact.synthesize(csr, prob, labels, eps=eps, regions=rv)
    torch.cuda.synchronize()
    out["with_region_boxes"] = {"iterations": list(gr.iterations),
                                "ms": (time.perf_counter() - t0) * 1e3,
                                "p_min_gain_max": float((gr.p_min - g.p_min).max().item())}
    try:
        import oracle
        from oracle import synthesis as SY
        ocsr = oracle.build_rows(prob)
        olab = labels.cpu().numpy()
        t0 = time.perf_counter()
        SY.interval_iteration(ocsr, olab, prob.n_inputs, SY.REACH_AVOID, eps=eps,
                              max_iters=oracle_iters)
        odt = time.perf_counter() - t0
        # the oracle runs both phases for `oracle_iters` iterations each
        out["cpu_baseline"] = {"value": 2 * prob.rows * 2 * oracle_iters / odt,
                               "unit": "row LPs/s", "cores": 1, "kind": "oracle",
                               "sample": f"{oracle_iters} iterations of each phase"}
    except Exception as exc:
        out["cpu_baseline"] = {"value": None, "error": str(exc)[:200]}
    return out


MC_WORKLOAD = ("5-D room (11^5 cells x 9 inputs = 1,449,459 rows) with correlated noise: "
               "covariance 0.2^2 (0.7 I + 0.3 J), 1024 seeded draws passed in, cutoff 2e-3 "
               "(>= 2 draws); sampled-noise bounds in FP32")


def run_mc(draws=1024, oracle_rows=4):
    """impact_build_mc on the 5-D room with correlated noise; the oracle's
    sampled-noise rows on a few sampled rows."""
    import torch
    from paper_2401_03555_gb300 import impact, workloads as W
    prob = W.room_5d(cutoff=2e-3)
    rng = np.random.default_rng(12)
    C = 0.2 ** 2 * (0.7 * np.eye(5) + 0.3 * np.ones((5, 5)))
    w = rng.normal(size=(draws, 5)) @ np.linalg.cholesky(C).T
    impact.build_mc(prob, w, "fp32")                       # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = impact.build_mc(prob, w, "fp32")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out = {"workload": MC_WORKLOAD, "rows": int(prob.rows), "pairs": int(g.nnz), "ms": dt * 1e3,
           "value": g.nnz / dt, "unit": "pairs/s", "row_draws_per_s": prob.rows * draws / dt,
           "path": "impact_build_mc (one block per row: shared-memory histograms of the cells "
                   "each moved image box meets / lies in; count, scan, emit)"}
    del g
    try:
        import oracle
        rows = W.sample_rows(prob, oracle_rows, seed=6, include_boundary=False)
        t0 = time.perf_counter()
        ref = oracle.build_rows_mc(prob, w, rows)
        odt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": ref.nnz / odt, "unit": "pairs/s",
                               "rows_per_s": len(rows) / odt, "cores": oracle.max_threads(),
                               "kind": "oracle", "sample": f"{len(rows)} sampled rows"}
    except Exception as exc:
        out["cpu_baseline"] = {"value": None, "error": str(exc)[:200]}
    return out


REGION_WORKLOAD = ("target / avoid vectors R and A of the 5-D room (11^5 cells x 9 inputs = "
                   "1,449,459 rows): target [19,21]^5, avoid x1 in [17,17.6]; box relaxation "
                   "and the paper's per-cell sums, FP32-sound evaluation")


def run_regions(reps=5, oracle_rows=16):
    """impact_region_vectors over every row of the 5-D room, both modes; the
    oracle (dense per-cell sums) on a few sampled rows."""
    import torch
    from paper_2401_03555_gb300 import impact, workloads as W
    prob = W.room_5d()
    target = [([19.0] * 5, [21.0] * 5)]
    avoid = [([17.0] * 5, [17.6, 23, 23, 23, 23])]
    out = {"workload": REGION_WORKLOAD, "rows": int(prob.rows), "unit": "rows/s"}
    for mode in ("box", "cells"):
        impact.region_vectors(prob, target, avoid, mode, "fp32")       # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            impact.region_vectors(prob, target, avoid, mode, "fp32")
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / reps
        out[mode] = {"ms": ms, "value": prob.rows / (ms * 1e-3),
                     "path": "impact_region_vectors (plan upload + one thread per row)"}
    try:
        import oracle
        rows = W.sample_rows(prob, oracle_rows, seed=5, include_boundary=False)
        t0 = time.perf_counter()
        oracle.region_vectors(prob, rows, target, avoid, "cells")
        odt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": len(rows) / odt, "unit": "rows/s",
                               "cores": oracle.max_threads(), "kind": "oracle",
                               "sample": f"{len(rows)} sampled rows, dense per-cell sums"}
    except Exception as exc:
        out["cpu_baseline"] = {"value": None, "error": str(exc)[:200]}
    return out


SERVED_WORKLOAD = ("Poisson stream of 500 requests (seed 1): 7-D building (6^7 cells, inputs "
                   "{0,1}^2, sigma 0.15, cutoff 1e-8) with probability 1/8, else a seeded "
                   "linear system of the batched workload; arrivals at 70% of the measured "
                   "service rate; FP32-sound, results kept on device until the client "
                   "releases them")


def served_requests(count=500, seed=1):
    from paper_2401_03555_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        if rng.random() < 0.125:
            out.append(W.building_7d())
        else:
            out.append(W.random_linear(int(rng.integers(256))))
    return out


def serve_stream(srv, probs, gaps):
    """Submit probs after the given gaps (seconds) from a client thread while a
    collector waits for each in order and releases it; returns latencies (ms),
    pairs and the wall time from the first submission to the last completion."""
    import threading
    tickets = [None] * len(probs)
    ready = [threading.Event() for _ in probs]
    lat = [None] * len(probs)
    parts = [None] * len(probs)
    t_start = time.perf_counter()

    def client():
        t = time.perf_counter()
        for i, (p, g) in enumerate(zip(probs, gaps)):
            t += g
            d = t - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets[i] = srv.submit(p)
            ready[i].set()

    th = threading.Thread(target=client)
    th.start()
    for i in range(len(probs)):
        ready[i].wait()
        _, lat[i] = srv.poll(tickets[i], wait=True)
        parts[i] = srv.timing(tickets[i])
        srv.release(tickets[i])
    th.join()
    wall = time.perf_counter() - t_start
    serve_stream.parts = parts
    return np.array(lat), wall


def latency_breakdown(lat, parts):
    """Where latency went: each phase's p50 / p99 over the requests, and the
    mean of each phase over the slowest 1% of the requests."""
    keys = ("queue", "count", "emit_wait", "emit")
    arr = {k: np.array([p[k] for p in parts]) for k in keys}
    slow = np.argsort(lat)[-max(1, len(lat) // 100):]
    return {"p50_ms": {k: float(np.percentile(arr[k], 50)) for k in keys},
            "p99_ms": {k: float(np.percentile(arr[k], 99)) for k in keys},
            "slowest_1pct_mean_ms": {k: float(arr[k][slow].mean()) for k in keys}}


def run_serving(count=500, seed=1, load=0.7):
    from paper_2401_03555_gb300 import impact
    probs = served_requests(count, seed)
    with impact.Server("fp32", timeout_s=120.0) as srv:
        # service rate: the same requests submitted at once (closed burst)
        lat_b, wall_b = serve_stream(srv, probs, [0.0] * len(probs))
        st = srv.stats()
        pairs = st["pairs"]
        service_s = wall_b / len(probs)
        rate = load / service_s
        gaps = np.random.default_rng(seed + 1000).exponential(1.0 / rate, size=len(probs))
        gaps[0] = 0.0
        lat, wall = serve_stream(srv, probs, gaps.tolist())
        parts = serve_stream.parts
        st2 = srv.stats()
    pairs_stream = st2["pairs"] - pairs
    return {"workload": SERVED_WORKLOAD, "requests": len(probs),
            "building_requests": int(sum(1 for p in probs if p.n == 7)),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "value": pairs_stream / wall, "unit": UNIT, "wall_s": round(wall, 3),
            "arrival_rate_per_s": round(rate, 2),
            "burst": {"pairs_per_s": pairs / wall_b, "wall_s": round(wall_b, 3),
                      "p50_ms": float(np.percentile(lat_b, 50)),
                      "p99_ms": float(np.percentile(lat_b, 99))},
            "groups": st2["groups"], "budget_bytes": st2["budget"],
            "breakdown": latency_breakdown(lat, parts),
            "path": "impact_server_submit / impact_server_poll / impact_server_release "
                    "(continuous batching, admission by device-memory footprint)"}


def run_e2e(prob, nnz, dev, stream, world, steps=3, mode="copy", copy_streams=4,
            chunk_bytes=256 << 20):
    """impact_build through the C ABI, results read back into pinned host
    memory inside the timed region. mode "copy": pairs built in device memory,
    then copied device -> host in chunks over several streams; mode "direct":
    col/lo/up are pinned host arrays that the emit kernel writes straight into
    over the host link. Row arrays are copied device -> host in both."""
    import torch
    from paper_2401_03555_gb300 import impact
    direct = mode == "direct"
    b = impact.Builder(prob, "fp32", capacity=nnz, pairs_on_host=direct)
    rb, pb = b.rows_buf, b.pairs_buf
    arrays = list(rb.items()) + ([] if direct else [(k, v[:nnz]) for k, v in pb.items()])
    host = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in arrays}
    chunks = []
    for k, v in arrays:
        step = max(1, chunk_bytes // v.element_size())
        for a0 in range(0, v.numel(), step):
            chunks.append((v[a0:a0 + step], host[k][a0:a0 + step]))
    cs = [torch.cuda.Stream(dev) for _ in range(copy_streams)]
    d2h = sum(v.numel() * v.element_size() for v in rb.values()) + \
        sum(v[:nnz].numel() * v.element_size() for v in pb.values())
    h2d = impact_blob_bytes(prob)
    times = []
    for it in range(steps + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        got = b.run(stream)                   # synchronizes its stream at the end
        for i, (src, dst) in enumerate(chunks):
            with torch.cuda.stream(cs[i % copy_streams]):
                dst.copy_(src, non_blocking=True)
        for c in cs:
            c.synchronize()
        dt = time.perf_counter() - t0
        if it > 0:
            times.append(dt)
    t = max_over_ranks(sum(times) / len(times), world, dev)
    total = sum_over_ranks(float(got), world, dev)
    how = ("col/lo/up in pinned host memory written by the emit kernel over the host link, "
           "then row_ptr/sink/trunc/flags copied device -> pinned host") if direct else \
          (f"every output array copied device -> pinned host in {chunk_bytes >> 20} MiB "
           f"chunks over {copy_streams} streams")
    return {"value": total / t, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": t * 1e3, "mode": mode,
            "path": f"impact_build (C ABI, tables uploaded per call); {how}; synchronized"}


def impact_blob_bytes(prob):
    """Bytes one build copies host -> device (descriptor and tables)."""
    from paper_2401_03555_gb300 import impact
    return int(impact.Batch([prob], "fp32").upload_bytes)


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


def run_case(which, cells=7, systems=16):
    """One small invocation of a leg, for a profiler to capture: synthesis on
    the 21^2 robot (3 iterations per phase), region vectors and sampled noise
    (1024 draws) on the 7^5-cell room; the FP32-sound build (count, then emit)
    and the FP64-plain build of the room on `cells`^5 cells; one group of the
    first `systems` systems of the batched workload built into caller arrays."""
    import torch
    from paper_2401_03555_gb300 import impact, workloads as W
    if which == "walk":
        prob = W.room_5d(cells_per_dim=cells)
        b = impact.Batch([prob], "fp32")
        rb = impact.alloc_rows(b.rows)
        ws = b.alloc_workspace()
        nnz = b.count(rb, ws)
        pb = impact.alloc_pairs(max(nnz, 1), "fp32")
        b.emit(rb, pb, max(nnz, 1), ws)
        torch.cuda.synchronize()
        print("pairs", nnz)
    elif which == "fp64":
        c = impact.build(W.room_5d(cells_per_dim=cells), "fp64")
        torch.cuda.synchronize()
        print("pairs", c.nnz)
    elif which == "batched":
        b = impact.Batch(W.batched_family(systems), "fp32")
        rb = impact.alloc_rows(b.rows)
        ws = b.alloc_workspace()
        nnz = b.count(rb, ws)
        pb = impact.alloc_pairs(max(nnz, 1), "fp32")
        b.build_into(rb, pb, max(nnz, 1), ws)
        torch.cuda.synchronize()
        print("pairs", nnz)
    elif which == "synth":
        prob = W.robot_2d()
        lab = impact.label_cells(prob, [([3, 3], [7, 7])], [([-7, -7], [-3, -3])])
        g = impact.synthesize(impact.build(prob, "fp64"), prob, lab, eps=1e-6, max_iters=3)
        print("synthesis iterations", g.iterations)
    elif which == "regions":
        prob = W.room_5d(cells_per_dim=7)
        v = impact.region_vectors(prob, [([19.0] * 5, [21.0] * 5)],
                                  [([17.0] * 5, [17.6, 23, 23, 23, 23])], "box", "fp32")
        torch.cuda.synchronize()
        print("region vectors, max R_max", float(v.r_up.max()))
    else:
        rng = np.random.default_rng(12)
        C = 0.2 ** 2 * (0.7 * np.eye(5) + 0.3 * np.ones((5, 5)))
        prob = W.room_5d(cells_per_dim=7, cutoff=2e-3)
        w = rng.normal(size=(1024, 5)) @ np.linalg.cholesky(C).T
        print("sampled-noise pairs", impact.build_mc(prob, w, "fp32").nnz)


def main(argv=None):
    args = parse_args(argv)
    if args.case:
        run_case(args.case, args.cells, args.systems)
        return
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
