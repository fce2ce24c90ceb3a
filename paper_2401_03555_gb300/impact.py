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
IMPACT_ERR_CUDA, IMPACT_ERR_TIMEOUT, IMPACT_ERR_UNSOUND = 4, 5, 6
FP64_PLAIN, FP32_SOUND = 0, 1
_PREC = {"fp64": FP64_PLAIN, "fp32": FP32_SOUND, FP64_PLAIN: FP64_PLAIN, FP32_SOUND: FP32_SOUND}

ENTRY_POINTS = ("impact_plan", "impact_workspace_bytes", "impact_build", "impact_count",
                "impact_emit", "impact_free", "impact_last_error", "impact_version",
                "impact_scan_rows_static")


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
    """Device scratch bytes of one build (descriptor, tables, scan, row records)."""
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


def alloc_pairs(nnz: int, precision="fp32", device=None):
    dev = device or torch.device("cuda")
    vt = torch.float32 if _PREC[precision] == FP32_SOUND else torch.float64
    k = max(int(nnz), 1)
    return dict(col=torch.empty(k, dtype=torch.int32, device=dev),
                lo=torch.empty(k, dtype=vt, device=dev), up=torch.empty(k, dtype=vt, device=dev))


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


class Builder:
    """Repeated builds of one problem into preallocated device buffers through
    the single-call entry point impact_build (caller-owned arrays)."""

    def __init__(self, prob, precision="fp32", capacity: Optional[int] = None, images=None):
        self.prob = prob
        self.precision = precision
        self.prec = _PREC[precision]
        self.args = _Args(prob, images=images)
        self.rows_buf = alloc_rows(prob.rows)
        if capacity is None:
            capacity = build(prob, precision).nnz
        self.capacity = int(capacity)
        self.pairs_buf = alloc_pairs(self.capacity, precision)
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
    if row_ptr.dtype != torch.int64 or not row_ptr.is_cuda or row_ptr.numel() < rows + 1:
        raise ValueError("row_ptr must be a CUDA int64 tensor of rows+1 entries")
    _check(load().impact_scan_rows_static(ctypes.c_void_p(row_ptr.data_ptr()), int(rows),
                                          ctypes.c_void_p(_stream_handle(stream))))


def version() -> int:
    return int(load().impact_version())
