"""Python binding of the C ABI in ``include/impact.h`` (argument marshalling only).

Every step of the abstraction runs in ``libimpact.so`` (hand-written sm_103a
CUDA). PyTorch supplies device memory and the current stream. There is no CPU
fallback: if the library is missing or no CUDA device is present, the calls
raise.

    from paper_2401_03555_gb300 import impact, workloads
    csr = impact.build(workloads.room_5d(), precision="fp32")
"""

from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import build as _build

IMPACT_OK, IMPACT_ERR_ARG, IMPACT_ERR_OOM, IMPACT_ERR_CAPACITY = 0, 1, 2, 3
IMPACT_ERR_CUDA, IMPACT_ERR_TIMEOUT, IMPACT_ERR_UNSOUND, IMPACT_ERR_CANCELLED = 4, 5, 6, 7
FP64_PLAIN, FP32_SOUND = 0, 1
_PREC = {"fp64": FP64_PLAIN, "fp32": FP32_SOUND, FP64_PLAIN: FP64_PLAIN, FP32_SOUND: FP32_SOUND}

ENTRY_POINTS = ("impact_plan", "impact_workspace_bytes", "impact_build", "impact_count",
                "impact_emit", "impact_free", "impact_last_error", "impact_version",
                "impact_scan_rows_static", "impact_batch_plan", "impact_batch_count",
                "impact_batch_emit", "impact_batch_build", "impact_graph_create",
                "impact_graph_launch", "impact_graph_result", "impact_graph_destroy",
                "impact_batch_tune", "impact_server_create", "impact_server_submit",
                "impact_server_poll", "impact_server_release", "impact_server_stats",
                "impact_server_destroy", "impact_synthesize", "impact_label_cells",
                "impact_region_vectors", "impact_synthesize_ex", "impact_build_mc",
                "impact_debug_fail_alloc", "impact_debug_live_bytes", "impact_server_timing",
                "impact_server_cancel")


class ImpactError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"impact status {status}: {message}")
        self.status = status


class _System(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("m", ctypes.c_int),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("c", ctypes.c_void_p),
                ("params", ctypes.c_void_p), ("dev_images", ctypes.c_void_p)]


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p),
                ("cells", ctypes.c_void_p)]


class _Inputs(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("m", ctypes.c_int), ("points", ctypes.c_void_p)]


class _CSR(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("lo", ctypes.c_void_p), ("up", ctypes.c_void_p),
                ("sink_lo", ctypes.c_void_p), ("sink_up", ctypes.c_void_p),
                ("trunc", ctypes.c_void_p), ("row_flags", ctypes.c_void_p),
                ("owned", ctypes.c_int), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_int64)]


class _Request(ctypes.Structure):
    _fields_ = [("sys", ctypes.c_void_p), ("grid", ctypes.c_void_p), ("inputs", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("cutoff", ctypes.c_double)]


class _Tuning(ctypes.Structure):
    _fields_ = [("count_warps", ctypes.c_int), ("emit_warps", ctypes.c_int),
                ("spin_limit", ctypes.c_int), ("one_pass", ctypes.c_int),
                ("stall_row", ctypes.c_int64), ("fault_row", ctypes.c_int64),
                ("guard_row", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class _Regions(ctypes.Structure):
    _fields_ = [("n_target", ctypes.c_int), ("n_avoid", ctypes.c_int),
                ("target_lo", ctypes.c_void_p), ("target_hi", ctypes.c_void_p),
                ("avoid_lo", ctypes.c_void_p), ("avoid_hi", ctypes.c_void_p)]


class _SynthOptions(ctypes.Structure):
    _fields_ = [("spec", ctypes.c_int), ("optimistic", ctypes.c_int), ("horizon", ctypes.c_int),
                ("n_disturb", ctypes.c_int), ("eps", ctypes.c_double),
                ("max_iters", ctypes.c_int), ("r_lo", ctypes.c_void_p), ("r_up", ctypes.c_void_p),
                ("a_lo", ctypes.c_void_p), ("a_up", ctypes.c_void_p)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_int64), ("max_batch", ctypes.c_int),
                ("max_group_rows", ctypes.c_int64), ("streams", ctypes.c_int),
                ("precision", ctypes.c_int)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("groups", ctypes.c_int64), ("waiting", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_int64), ("budget", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libimpact.so (building it first when the sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run paper_2401_03555_gb300.build)")
        lib = ctypes.CDLL(path)
        common = [ctypes.POINTER(_System), ctypes.POINTER(_Grid), ctypes.POINTER(_Inputs),
                  ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
        lib.impact_plan.restype = ctypes.c_int
        lib.impact_plan.argtypes = common + [ctypes.POINTER(ctypes.c_int64)] * 3
        lib.impact_workspace_bytes.restype = ctypes.c_int
        lib.impact_workspace_bytes.argtypes = common + [ctypes.POINTER(ctypes.c_int64)]
        for name in ("impact_build", "impact_count", "impact_emit"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = common + [ctypes.POINTER(_CSR), ctypes.c_void_p]
        lib.impact_free.restype = ctypes.c_int
        lib.impact_free.argtypes = [ctypes.POINTER(_CSR)]
        lib.impact_last_error.restype = ctypes.c_char_p
        lib.impact_last_error.argtypes = []
        lib.impact_version.restype = ctypes.c_int
        lib.impact_version.argtypes = []
        lib.impact_scan_rows_static.restype = ctypes.c_int
        lib.impact_scan_rows_static.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        lib.impact_debug_fail_alloc.restype = ctypes.c_int
        lib.impact_debug_fail_alloc.argtypes = [ctypes.c_int64]
        lib.impact_debug_live_bytes.restype = ctypes.c_int
        lib.impact_debug_live_bytes.argtypes = [ctypes.POINTER(ctypes.c_int64)] * 2
        breq = [ctypes.POINTER(_Request), ctypes.c_int, ctypes.c_int, ctypes.POINTER(_Tuning)]
        lib.impact_batch_plan.restype = ctypes.c_int
        lib.impact_batch_plan.argtypes = breq + [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int64)] * 3
        for name in ("impact_batch_count", "impact_batch_emit", "impact_batch_build"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = breq + [ctypes.POINTER(_CSR), ctypes.c_void_p]
        lib.impact_graph_create.restype = ctypes.c_int
        lib.impact_graph_create.argtypes = breq + [ctypes.POINTER(_CSR), ctypes.c_void_p,
                                                   ctypes.POINTER(ctypes.c_void_p)]
        lib.impact_graph_launch.restype = ctypes.c_int
        lib.impact_graph_launch.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        lib.impact_graph_result.restype = ctypes.c_int
        lib.impact_graph_result.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
        lib.impact_graph_destroy.restype = ctypes.c_int
        lib.impact_graph_destroy.argtypes = [ctypes.c_void_p]
        lib.impact_batch_tune.restype = ctypes.c_int
        lib.impact_batch_tune.argtypes = [ctypes.POINTER(_Request), ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(_CSR), ctypes.c_int, ctypes.c_void_p,
                                          ctypes.POINTER(_Tuning),
                                          ctypes.POINTER(ctypes.c_double)]
        lib.impact_server_create.restype = ctypes.c_int
        lib.impact_server_create.argtypes = [ctypes.POINTER(_ServerConfig),
                                             ctypes.POINTER(ctypes.c_void_p)]
        lib.impact_server_submit.restype = ctypes.c_int
        lib.impact_server_submit.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Request),
                                             ctypes.POINTER(ctypes.c_int64)]
        lib.impact_server_poll.restype = ctypes.c_int
        lib.impact_server_poll.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_CSR),
                                           ctypes.POINTER(ctypes.c_double)]
        lib.impact_server_release.restype = ctypes.c_int
        lib.impact_server_release.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        lib.impact_server_cancel.restype = ctypes.c_int
        lib.impact_server_cancel.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        lib.impact_server_timing.restype = ctypes.c_int
        lib.impact_server_timing.argtypes = [ctypes.c_void_p, ctypes.c_int64] + \
            [ctypes.POINTER(ctypes.c_double)] * 4
        lib.impact_server_stats.restype = ctypes.c_int
        lib.impact_server_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(_ServerStats)]
        lib.impact_server_destroy.restype = ctypes.c_int
        lib.impact_server_destroy.argtypes = [ctypes.c_void_p]
        lib.impact_synthesize.restype = ctypes.c_int
        lib.impact_synthesize.argtypes = [ctypes.POINTER(_CSR), ctypes.c_int, ctypes.c_int64,
                                          ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]
        lib.impact_build_mc.restype = ctypes.c_int
        lib.impact_build_mc.argtypes = [ctypes.POINTER(_System), ctypes.POINTER(_Grid),
                                        ctypes.POINTER(_Inputs), ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_double, ctypes.c_int, ctypes.POINTER(_CSR),
                                        ctypes.c_void_p]
        lib.impact_label_cells.restype = ctypes.c_int
        lib.impact_label_cells.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Regions),
                                           ctypes.c_void_p, ctypes.c_void_p]
        lib.impact_region_vectors.restype = ctypes.c_int
        lib.impact_region_vectors.argtypes = [ctypes.POINTER(_System), ctypes.POINTER(_Grid),
                                              ctypes.POINTER(_Inputs), ctypes.c_void_p,
                                              ctypes.POINTER(_Regions), ctypes.c_int, ctypes.c_int,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p]
        lib.impact_synthesize_ex.restype = ctypes.c_int
        lib.impact_synthesize_ex.argtypes = [ctypes.POINTER(_CSR), ctypes.c_int, ctypes.c_int64,
                                             ctypes.c_int, ctypes.c_void_p,
                                             ctypes.POINTER(_SynthOptions), ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]
        _lib = lib
        return lib


def _check(status: int):
    if status != IMPACT_OK:
        raise ImpactError(status, load().impact_last_error().decode())


class _Args:
    """ctypes structs for one problem; holds the numpy buffers they point into."""

    def __init__(self, prob, images: Optional[torch.Tensor] = None, need_images: bool = True):
        f64 = lambda x: None if x is None else np.ascontiguousarray(np.asarray(x, np.float64))
        self.lo, self.hi = f64(prob.lo), f64(prob.hi)
        self.cells = np.ascontiguousarray(np.asarray(prob.cells, np.int32))
        self.sigma = f64(prob.sigma)
        n = int(self.lo.shape[0])
        inputs = np.asarray(prob.inputs, np.float64)
        if inputs.ndim == 1:
            inputs = inputs.reshape(-1, 1)
        self.inputs = np.ascontiguousarray(inputs)
        m = int(self.inputs.shape[1])
        self.A, self.B, self.c = f64(prob.A), f64(prob.B), f64(prob.c)
        if self.B is not None and self.B.size == 0:
            self.B = None
        self.images = images
        if prob.kind == 2 and images is None and need_images:
            if prob.images is None:
                raise ValueError("an IMAGES problem needs images")
            self.images = torch.as_tensor(np.asarray(prob.images, np.float64)).cuda().contiguous()
        ptr = lambda a: None if a is None else a.ctypes.data
        self.sys = _System(int(prob.kind), n, m, ptr(self.A), ptr(self.B), ptr(self.c), None,
                           None if self.images is None else self.images.data_ptr())
        self.grid = _Grid(n, ptr(self.lo), ptr(self.hi), ptr(self.cells))
        self.inp = _Inputs(int(self.inputs.shape[0]), m, ptr(self.inputs) if m > 0 else None)
        self.sigma_ptr = ptr(self.sigma)
        self.cutoff = float(prob.cutoff)


@dataclass
class CSR:
    """Device-resident result of one build (torch tensors on the GPU)."""
    precision: str
    row_ptr: torch.Tensor    # int64 [rows+1]
    col: torch.Tensor        # int32 [nnz]
    lo: torch.Tensor         # float32/float64 [nnz]
    up: torch.Tensor
    sink_lo: torch.Tensor    # float64 [rows]
    sink_up: torch.Tensor
    trunc: torch.Tensor
    row_flags: torch.Tensor  # int32 view of uint32 [rows]

    @property
    def rows(self) -> int:
        return int(self.row_ptr.shape[0]) - 1

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def nbytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in
                   (self.row_ptr, self.col, self.lo, self.up, self.sink_lo, self.sink_up,
                    self.trunc, self.row_flags))


def _stream_handle(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def plan(prob, precision="fp32"):
    """(rows, nnz upper bound, device bytes upper bound) without touching the GPU."""
    a = _Args(prob, need_images=False)
    if prob.kind == 2:
        a.sys.dev_images = 1  # the planner only checks that images are given
    rows, nnz, nbytes = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().impact_plan(ctypes.byref(a.sys), ctypes.byref(a.grid), ctypes.byref(a.inp),
                              a.sigma_ptr, a.cutoff, _PREC[precision], ctypes.byref(rows),
                              ctypes.byref(nnz), ctypes.byref(nbytes)))
    return rows.value, nnz.value, nbytes.value


def workspace_bytes(prob, precision="fp32") -> int:
    """Device scratch bytes of one build (descriptor, tables, scan, offset words)."""
    a = _Args(prob, need_images=False)
    if prob.kind == 2:
        a.sys.dev_images = 1
    b = ctypes.c_int64()
    _check(load().impact_workspace_bytes(ctypes.byref(a.sys), ctypes.byref(a.grid),
                                         ctypes.byref(a.inp), a.sigma_ptr, a.cutoff,
                                         _PREC[precision], ctypes.byref(b)))
    return b.value


def alloc_workspace(prob, precision="fp32", device=None) -> torch.Tensor:
    dev = device or torch.device("cuda")
    return torch.empty(max(workspace_bytes(prob, precision), 256), dtype=torch.uint8, device=dev)


def alloc_rows(rows: int, device=None):
    dev = device or torch.device("cuda")
    return dict(row_ptr=torch.empty(rows + 1, dtype=torch.int64, device=dev),
                sink_lo=torch.empty(rows, dtype=torch.float64, device=dev),
                sink_up=torch.empty(rows, dtype=torch.float64, device=dev),
                trunc=torch.empty(rows, dtype=torch.float64, device=dev),
                row_flags=torch.empty(rows, dtype=torch.int32, device=dev))


def alloc_pairs(nnz: int, precision="fp32", device=None, host: bool = False):
    """col/lo/up buffers for `nnz` pairs: device memory, or (host=True) pinned
    host memory that the emit kernel writes directly."""
    vt = torch.float32 if _PREC[precision] == FP32_SOUND else torch.float64
    k = max(int(nnz), 1)
    if host:
        mk = lambda dt: torch.empty(k, dtype=dt, pin_memory=True)
    else:
        dev = device or torch.device("cuda")
        mk = lambda dt: torch.empty(k, dtype=dt, device=dev)
    return dict(col=mk(torch.int32), lo=mk(vt), up=mk(vt))


def _csr_struct(rows_buf, pairs_buf=None, capacity=0, workspace=None):
    p = lambda t: t.data_ptr()
    c = _CSR()
    if workspace is not None:
        c.workspace = workspace.data_ptr()
        c.workspace_bytes = workspace.numel()
    c.rows = 0
    c.nnz = capacity
    c.row_ptr = p(rows_buf["row_ptr"])
    c.sink_lo = p(rows_buf["sink_lo"])
    c.sink_up = p(rows_buf["sink_up"])
    c.trunc = p(rows_buf["trunc"])
    c.row_flags = p(rows_buf["row_flags"]) if rows_buf.get("row_flags") is not None else None
    if pairs_buf is not None:
        c.col, c.lo, c.up = p(pairs_buf["col"]), p(pairs_buf["lo"]), p(pairs_buf["up"])
    return c


def build(prob, precision="fp32", stream=None, check_unsound: bool = True) -> CSR:
    """Full build with exactly sized torch buffers: count (C ABI impact_count),
    allocate, emit (impact_emit). Returns the device CSR."""
    lib = load()
    a = _Args(prob)
    prec = _PREC[precision]
    rows = prob.rows
    rb = alloc_rows(rows)
    ws = alloc_workspace(prob, precision)
    c = _csr_struct(rb, workspace=ws)
    st = _stream_handle(stream)
    status = lib.impact_count(ctypes.byref(a.sys), ctypes.byref(a.grid), ctypes.byref(a.inp),
                              a.sigma_ptr, a.cutoff, prec, ctypes.byref(c), ctypes.c_void_p(st))
    if status != IMPACT_OK and not (status == IMPACT_ERR_UNSOUND and not check_unsound):
        _check(status)
    nnz = int(c.nnz)
    pb = alloc_pairs(nnz, precision)
    c2 = _csr_struct(rb, pb, capacity=nnz, workspace=ws)
    _check(lib.impact_emit(ctypes.byref(a.sys), ctypes.byref(a.grid), ctypes.byref(a.inp),
                           a.sigma_ptr, a.cutoff, prec, ctypes.byref(c2), ctypes.c_void_p(st)))
    return CSR("fp32" if prec == FP32_SOUND else "fp64", rb["row_ptr"], pb["col"][:nnz],
               pb["lo"][:nnz], pb["up"][:nnz], rb["sink_lo"], rb["sink_up"], rb["trunc"],
               rb["row_flags"])


def build_mc(prob, samples, precision="fp64", cutoff=None, stream=None) -> CSR:
    """impact_build_mc: the IMDP for a noise given by draws (an (S, n) array
    of samples, e.g. L z for a full covariance L L^T); library-owned result."""
    a = _Args(prob)
    W = torch.as_tensor(np.asarray(samples, np.float64).reshape(-1, a.lo.shape[0]).T.copy())
    W = W.cuda().contiguous()
    S = int(W.shape[1])
    c = _CSR()
    cut = float(prob.cutoff if cutoff is None else cutoff)
    _check(load().impact_build_mc(ctypes.byref(a.sys), ctypes.byref(a.grid), ctypes.byref(a.inp),
                                  W.data_ptr(), S, cut, _PREC[precision], ctypes.byref(c),
                                  ctypes.c_void_p(_stream_handle(stream))))
    torch.cuda.synchronize()
    rows, nnz = int(c.rows), int(c.nnz)
    vt = torch.float32 if _PREC[precision] == FP32_SOUND else torch.float64
    try:   # copies into torch tensors, then the library's arrays are freed
        out = CSR(precision, _view(c.row_ptr, rows + 1, torch.int64).clone(),
                  _view(c.col, nnz, torch.int32).clone(), _view(c.lo, nnz, vt).clone(),
                  _view(c.up, nnz, vt).clone(), _view(c.sink_lo, rows, torch.float64).clone(),
                  _view(c.sink_up, rows, torch.float64).clone(),
                  _view(c.trunc, rows, torch.float64).clone(),
                  _view(c.row_flags, rows, torch.int32).clone())
        torch.cuda.synchronize()
    finally:
        _check(load().impact_free(ctypes.byref(c)))
    return out


class Builder:
    """Repeated builds of one problem into preallocated device buffers through
    the single-call entry point impact_build (caller-owned arrays)."""

    def __init__(self, prob, precision="fp32", capacity: Optional[int] = None, images=None,
                 pairs_on_host: bool = False):
        self.prob = prob
        self.precision = precision
        self.prec = _PREC[precision]
        self.args = _Args(prob, images=images)
        self.rows_buf = alloc_rows(prob.rows)
        if capacity is None:
            capacity = build(prob, precision).nnz
        self.capacity = int(capacity)
        self.pairs_buf = alloc_pairs(self.capacity, precision, host=pairs_on_host)
        self.workspace = alloc_workspace(prob, precision)
        self.nnz = 0

    def run(self, stream=None) -> int:
        lib = load()
        a = self.args
        c = _csr_struct(self.rows_buf, self.pairs_buf, capacity=self.capacity,
                        workspace=self.workspace)
        _check(lib.impact_build(ctypes.byref(a.sys), ctypes.byref(a.grid), ctypes.byref(a.inp),
                                a.sigma_ptr, a.cutoff, self.prec, ctypes.byref(c),
                                ctypes.c_void_p(_stream_handle(stream))))
        self.nnz = int(c.nnz)
        return self.nnz

    def result(self) -> CSR:
        k = self.nnz
        rb, pb = self.rows_buf, self.pairs_buf
        return CSR(self.precision, rb["row_ptr"], pb["col"][:k], pb["lo"][:k], pb["up"][:k],
                   rb["sink_lo"], rb["sink_up"], rb["trunc"], rb["row_flags"])


def build_library_owned(prob, precision="fp32", stream=None):
    """impact_build with library-owned output (col == NULL on entry); returns
    (rows, nnz) and frees the result again. Exercises the ownership path."""
    lib = load()
    a = _Args(prob)
    c = _CSR()
    _check(lib.impact_build(ctypes.byref(a.sys), ctypes.byref(a.grid), ctypes.byref(a.inp),
                            a.sigma_ptr, a.cutoff, _PREC[precision], ctypes.byref(c),
                            ctypes.c_void_p(_stream_handle(stream))))
    rows, nnz, owned = int(c.rows), int(c.nnz), int(c.owned)
    _check(lib.impact_free(ctypes.byref(c)))
    return rows, nnz, owned


def scan_rows_static(row_ptr: torch.Tensor, rows: int, stream=None) -> None:
    """In-place exclusive scan of per-row counts (row_ptr[0..rows)) into CSR
    row pointers with the allocation-free entry point impact_scan_rows_static."""
    if (row_ptr.dtype != torch.int64 or not row_ptr.is_cuda or row_ptr.numel() < rows + 1
            or not row_ptr.is_contiguous()):
        raise ValueError("row_ptr must be a contiguous CUDA int64 tensor of rows+1 entries")
    _check(load().impact_scan_rows_static(ctypes.c_void_p(row_ptr.data_ptr()), int(rows),
                                          ctypes.c_void_p(_stream_handle(stream))))


def version() -> int:
    return int(load().impact_version())


def fail_alloc(n: int) -> None:
    """impact_debug_fail_alloc: the n-th allocation the library makes from now
    on fails as out of memory (0: off)."""
    _check(load().impact_debug_fail_alloc(ctypes.c_int64(int(n))))


def live_bytes():
    """impact_debug_live_bytes: (device, pinned host) bytes the library holds."""
    d, h = ctypes.c_int64(), ctypes.c_int64()
    _check(load().impact_debug_live_bytes(ctypes.byref(d), ctypes.byref(h)))
    return int(d.value), int(h.value)


# --------------------------------------------------------------------------
# batches: several builds per launch (impact_batch_*), CUDA graphs, autotuner
# --------------------------------------------------------------------------

def tuning(count_warps=0, emit_warps=0, spin_limit=0, stall_row=None, fault_row=None,
           one_pass=False, guard_row=None):
    """An impact_tuning (zero fields take the library defaults). `stall_row`,
    `fault_row` and `guard_row` are fault injection for the failure-path
    tests: row r never publishes its pair count (one_pass: the rows after it
    time out), row r's row check sees an impossible lower-bound sum
    (IMPACT_ERR_UNSOUND), or row r's walk starts with its step guard spent
    (IMPACT_ERR_CUDA, internal)."""
    opt = lambda r: 0 if r is None else int(r) + 1
    return _Tuning(count_warps, emit_warps, spin_limit, int(bool(one_pass)),
                   opt(stall_row), opt(fault_row), opt(guard_row))


@dataclass
class BatchCSR:
    """Device result of a batch: one CSR over the concatenated rows."""
    csr: CSR
    row_offsets: np.ndarray   # int64 [count+1], host

    @property
    def count(self) -> int:
        return int(self.row_offsets.shape[0]) - 1

    def part(self, q: int) -> CSR:
        """Build q as its own CSR (views; row_ptr rebased to start at 0)."""
        r0, r1 = int(self.row_offsets[q]), int(self.row_offsets[q + 1])
        c = self.csr
        rp = c.row_ptr[r0:r1 + 1]
        base = int(rp[0].item())
        end = int(rp[-1].item())
        return CSR(c.precision, rp - base, c.col[base:end], c.lo[base:end], c.up[base:end],
                   c.sink_lo[r0:r1], c.sink_up[r0:r1], c.trunc[r0:r1], c.row_flags[r0:r1])


class Batch:
    """Several builds handled by one launch of each kernel (impact_batch_*).

    Holds the marshalled arguments of every problem; `plan`, `count`, `emit`,
    `build`, `tune` and `graph` call the C ABI."""

    def __init__(self, problems, precision="fp32", tune=None):
        self.problems = list(problems)
        self.precision = precision
        self.prec = _PREC[precision]
        self.args = [_Args(p) for p in self.problems]
        n = len(self.args)
        self.reqs = (_Request * n)()
        for q, a in enumerate(self.args):
            self.reqs[q] = _Request(ctypes.addressof(a.sys), ctypes.addressof(a.grid),
                                    ctypes.addressof(a.inp), a.sigma_ptr, a.cutoff)
        self.tuning = tune
        self.row_offsets, self.nnz_bound, self.ws_bytes, self.upload_bytes = self.plan()
        self.rows = int(self.row_offsets[-1])

    def _tp(self):
        return None if self.tuning is None else ctypes.byref(self.tuning)

    def plan(self):
        n = len(self.args)
        offs = np.zeros(n + 1, dtype=np.int64)
        nnz, ws, up = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().impact_batch_plan(self.reqs, n, self.prec, self._tp(), offs.ctypes.data,
                                        ctypes.byref(nnz), ctypes.byref(ws), ctypes.byref(up)))
        return offs, nnz.value, ws.value, up.value

    def alloc_workspace(self, device=None):
        dev = device or torch.device("cuda")
        return torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)

    def count(self, rows_buf, workspace=None, stream=None, check_unsound=True) -> int:
        c = _csr_struct(rows_buf, workspace=workspace)
        st = load().impact_batch_count(self.reqs, len(self.args), self.prec, self._tp(),
                                       ctypes.byref(c), ctypes.c_void_p(_stream_handle(stream)))
        if st != IMPACT_OK and not (st == IMPACT_ERR_UNSOUND and not check_unsound):
            _check(st)
        return int(c.nnz)

    def emit(self, rows_buf, pairs_buf, capacity, workspace=None, stream=None):
        c = _csr_struct(rows_buf, pairs_buf, capacity=capacity, workspace=workspace)
        _check(load().impact_batch_emit(self.reqs, len(self.args), self.prec, self._tp(),
                                        ctypes.byref(c), ctypes.c_void_p(_stream_handle(stream))))

    def build(self, stream=None) -> BatchCSR:
        """count, allocate exactly, emit (shared workspace)."""
        rb = alloc_rows(self.rows)
        ws = self.alloc_workspace()
        nnz = self.count(rb, ws, stream)
        pb = alloc_pairs(nnz, self.precision)
        self.emit(rb, pb, nnz, ws, stream)
        csr = CSR("fp32" if self.prec == FP32_SOUND else "fp64", rb["row_ptr"], pb["col"][:nnz],
                  pb["lo"][:nnz], pb["up"][:nnz], rb["sink_lo"], rb["sink_up"], rb["trunc"],
                  rb["row_flags"])
        return BatchCSR(csr, self.row_offsets.copy())

    def build_into(self, rows_buf, pairs_buf, capacity, workspace=None, stream=None) -> int:
        """impact_batch_build into caller buffers; returns nnz."""
        c = _csr_struct(rows_buf, pairs_buf, capacity=capacity, workspace=workspace)
        _check(load().impact_batch_build(self.reqs, len(self.args), self.prec, self._tp(),
                                         ctypes.byref(c), ctypes.c_void_p(_stream_handle(stream))))
        return int(c.nnz)

    def tune(self, rows_buf, pairs_buf=None, capacity=0, reps=3, stream=None):
        """Run the autotuner; stores and returns (tuning, count+emit ms)."""
        c = _csr_struct(rows_buf, pairs_buf, capacity=capacity)
        best = _Tuning()
        ms = ctypes.c_double()
        _check(load().impact_batch_tune(self.reqs, len(self.args), self.prec, ctypes.byref(c),
                                        int(reps), ctypes.c_void_p(_stream_handle(stream)),
                                        ctypes.byref(best), ctypes.byref(ms)))
        self.tuning = best
        return best, ms.value

    def graph(self, rows_buf, pairs_buf, capacity, workspace=None, stream=None) -> "Graph":
        return Graph(self, rows_buf, pairs_buf, capacity, workspace, stream)


class Graph:
    """A captured CUDA graph of one batch's whole pipeline (impact_graph_*)."""

    def __init__(self, batch: Batch, rows_buf, pairs_buf, capacity, workspace=None, stream=None):
        self.batch = batch
        self.bufs = (rows_buf, pairs_buf, workspace)   # kept alive with the graph
        c = _csr_struct(rows_buf, pairs_buf, capacity=capacity, workspace=workspace)
        h = ctypes.c_void_p()
        _check(load().impact_graph_create(batch.reqs, len(batch.args), batch.prec, batch._tp(),
                                          ctypes.byref(c), ctypes.c_void_p(_stream_handle(stream)),
                                          ctypes.byref(h)))
        self.handle = h

    def launch(self, stream=None):
        _check(load().impact_graph_launch(self.handle, ctypes.c_void_p(_stream_handle(stream))))

    def result(self) -> int:
        """Status and nnz of the last launch (synchronize its stream first)."""
        nnz = ctypes.c_int64()
        _check(load().impact_graph_result(self.handle, ctypes.byref(nnz)))
        return int(nnz.value)

    def close(self):
        if self.handle:
            load().impact_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# serving (impact_server_*)
# --------------------------------------------------------------------------

class _DeviceArray:
    """A zero-copy view of server-owned device memory (CUDA array interface)."""

    def __init__(self, ptr, count, typestr):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr,
                                         "data": (int(ptr) if count else 0, False),
                                         "version": 3, "strides": None}


def _view(ptr, count, dtype):
    typestr = {torch.int64: "<i8", torch.int32: "<i4", torch.float32: "<f4",
               torch.float64: "<f8"}[dtype]
    if count == 0:
        return torch.empty(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, count, typestr), device="cuda")


class Server:
    """Continuous-batching request loop (impact_server_*): submit builds as
    they arrive, poll for their device results, release them when done."""

    def __init__(self, precision="fp32", memory_budget=0, max_batch=0, streams=0,
                 max_group_rows=0, timeout_s=600.0):
        self.precision = precision
        self.prec = _PREC[precision]
        self.timeout_ms = int(timeout_s * 1000)
        cfg = _ServerConfig(int(memory_budget), int(max_batch), int(max_group_rows), int(streams),
                            self.prec)
        h = ctypes.c_void_p()
        _check(load().impact_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self._args = {}

    def submit(self, prob) -> int:
        a = _Args(prob)
        req = _Request(ctypes.addressof(a.sys), ctypes.addressof(a.grid), ctypes.addressof(a.inp),
                       a.sigma_ptr, a.cutoff)
        t = ctypes.c_int64()
        _check(load().impact_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        if prob.kind == 2:
            self._args[t.value] = a   # device images must outlive the request
        return int(t.value)

    def poll(self, ticket: int, wait: bool = False):
        """(done, latency_ms); raises if the request failed, TimeoutError if
        `wait` and it did not finish within the server's timeout."""
        done = ctypes.c_int()
        lat = ctypes.c_double()
        _check(load().impact_server_poll(self.handle, int(ticket),
                                         self.timeout_ms if wait else 0, ctypes.byref(done),
                                         None, ctypes.byref(lat)))
        if wait and not done.value:
            raise TimeoutError(f"request {ticket} still in flight after {self.timeout_ms} ms")
        return bool(done.value), (lat.value if done.value else None)

    def result(self, ticket: int) -> CSR:
        """Zero-copy views of a finished request's device result (row_ptr
        rebased to 0 as a new tensor); valid until release(ticket)."""
        done = ctypes.c_int()
        c = _CSR()
        _check(load().impact_server_poll(self.handle, int(ticket), self.timeout_ms,
                                         ctypes.byref(done), ctypes.byref(c), None))
        if not done.value:
            raise TimeoutError(f"request {ticket} still in flight after {self.timeout_ms} ms")
        rows, nnz = int(c.rows), int(c.nnz)
        vt = torch.float32 if self.prec == FP32_SOUND else torch.float64
        rp = _view(c.row_ptr, rows + 1, torch.int64)
        base = int(rp[0].item())
        col_all = _view(c.col, base + nnz, torch.int32)
        lo_all = _view(c.lo, base + nnz, vt)
        up_all = _view(c.up, base + nnz, vt)
        return CSR(self.precision, rp - base, col_all[base:], lo_all[base:], up_all[base:],
                   _view(c.sink_lo, rows, torch.float64), _view(c.sink_up, rows, torch.float64),
                   _view(c.trunc, rows, torch.float64), _view(c.row_flags, rows, torch.int32))

    def cancel(self, ticket: int):
        """impact_server_cancel: withdraw a request still waiting for admission
        (poll then raises ImpactError with IMPACT_ERR_CANCELLED)."""
        _check(load().impact_server_cancel(self.handle, int(ticket)))

    def timing(self, ticket: int) -> dict:
        """impact_server_timing: where a finished request's latency went (ms)."""
        v = [ctypes.c_double() for _ in range(4)]
        _check(load().impact_server_timing(self.handle, int(ticket), *[ctypes.byref(x) for x in v]))
        return dict(zip(("queue", "count", "emit_wait", "emit"), (x.value for x in v)))

    def release(self, ticket: int):
        _check(load().impact_server_release(self.handle, int(ticket)))
        self._args.pop(int(ticket), None)

    def stats(self) -> dict:
        st = _ServerStats()
        _check(load().impact_server_stats(self.handle, ctypes.byref(st)))
        return {k: int(getattr(st, k)) for k, _ in st._fields_}

    def close(self):
        if self.handle:
            load().impact_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# controller synthesis (impact_synthesize)
# --------------------------------------------------------------------------

REACH_AVOID, SAFETY = 0, 1


@dataclass
class Controller:
    p_min: torch.Tensor     # float64 [cells]
    p_max: torch.Tensor     # float64 [cells]
    policy: torch.Tensor    # int32 [cells]
    iterations: tuple


class _RegionArgs:
    """impact_regions for lists of (lo, hi) boxes; keeps the arrays alive."""

    def __init__(self, n, target=(), avoid=()):
        def arr(boxes, k):
            a = np.zeros((max(len(boxes), 1), n))
            for i, b in enumerate(boxes):
                a[i] = np.asarray(b[k], np.float64).reshape(n)
            return np.ascontiguousarray(a)
        self.t_lo, self.t_hi = arr(target, 0), arr(target, 1)
        self.a_lo, self.a_hi = arr(avoid, 0), arr(avoid, 1)
        self.struct = _Regions(len(target), len(avoid), self.t_lo.ctypes.data,
                               self.t_hi.ctypes.data, self.a_lo.ctypes.data, self.a_hi.ctypes.data)


def label_cells(prob, target=(), avoid=(), stream=None) -> torch.Tensor:
    """uint8 label per cell on the GPU: 0 free, 1 target, 2 avoid
    (impact_label_cells; a box labels the cells whose centre it contains)."""
    a = _Args(prob, need_images=False)
    r = _RegionArgs(int(a.lo.shape[0]), target, avoid)
    out = torch.empty(int(prob.total_cells), dtype=torch.uint8, device="cuda")
    _check(load().impact_label_cells(ctypes.byref(a.grid), ctypes.byref(r.struct),
                                     out.data_ptr(), ctypes.c_void_p(_stream_handle(stream))))
    return out


@dataclass
class RegionVectors:
    """Per-row bounds of landing in the target cells and in an avoid cell or
    outside the domain (float64 tensors on the GPU)."""
    r_lo: torch.Tensor
    r_up: torch.Tensor
    a_lo: torch.Tensor
    a_up: torch.Tensor


REGION_BOX, REGION_CELL_SUM = 0, 1
_MODE = {"box": REGION_BOX, "cells": REGION_CELL_SUM, REGION_BOX: REGION_BOX,
         REGION_CELL_SUM: REGION_CELL_SUM}


def region_vectors(prob, target=(), avoid=(), mode="box", precision="fp64",
                   stream=None) -> RegionVectors:
    """impact_region_vectors: mode "box" (one relaxation per region box) or
    "cells" (the paper's sums of per-cell bounds)."""
    a = _Args(prob)
    r = _RegionArgs(int(a.lo.shape[0]), target, avoid)
    rows = int(prob.rows)
    v = [torch.empty(rows, dtype=torch.float64, device="cuda") for _ in range(4)]
    _check(load().impact_region_vectors(ctypes.byref(a.sys), ctypes.byref(a.grid),
                                        ctypes.byref(a.inp), a.sigma_ptr, ctypes.byref(r.struct),
                                        _MODE[mode], _PREC[precision],
                                        *[t.data_ptr() for t in v],
                                        ctypes.c_void_p(_stream_handle(stream))))
    return RegionVectors(*v)


def synthesize(csr: CSR, prob, labels, spec=REACH_AVOID, eps=1e-6, max_iters=10000,
               optimistic=False, horizon=0, n_disturb=1, regions: Optional[RegionVectors] = None,
               stream=None) -> Controller:
    """Interval iteration on a device IMDP built for `prob`
    (impact_synthesize_ex). With disturbances the build's input points are
    the (input, disturbance) pairs, disturbance fastest: prob.n_inputs =
    inputs * n_disturb."""
    cells = int(prob.total_cells)
    if int(prob.n_inputs) % int(n_disturb):
        raise ValueError("the build's input count is not a multiple of n_disturb")
    n_inputs = int(prob.n_inputs) // int(n_disturb)
    if isinstance(labels, torch.Tensor):
        lab = labels.to(device="cuda", dtype=torch.uint8).contiguous()
    else:
        lab = torch.as_tensor(np.asarray(labels, np.uint8)).cuda()
    dev = lab.device
    p_min = torch.empty(cells, dtype=torch.float64, device=dev)
    p_max = torch.empty(cells, dtype=torch.float64, device=dev)
    pol = torch.empty(cells, dtype=torch.int32, device=dev)
    c = _CSR()
    c.rows = csr.rows
    c.nnz = csr.nnz
    p = lambda t: t.data_ptr()
    c.row_ptr, c.col, c.lo, c.up = p(csr.row_ptr), p(csr.col), p(csr.lo), p(csr.up)
    c.sink_lo, c.sink_up, c.trunc = p(csr.sink_lo), p(csr.sink_up), p(csr.trunc)
    o = _SynthOptions(int(spec), int(bool(optimistic)), int(horizon), int(n_disturb), float(eps),
                      int(max_iters), None, None, None, None)
    if regions is not None:
        o.r_lo, o.r_up = p(regions.r_lo), p(regions.r_up)
        o.a_lo, o.a_up = p(regions.a_lo), p(regions.a_up)
    its = (ctypes.c_int * 2)()
    _check(load().impact_synthesize_ex(ctypes.byref(c), _PREC[csr.precision], cells, n_inputs,
                                       p(lab), ctypes.byref(o), p(p_min), p(p_max), p(pol), its,
                                       ctypes.c_void_p(_stream_handle(stream))))
    return Controller(p_min, p_max, pol, (int(its[0]), int(its[1])))
