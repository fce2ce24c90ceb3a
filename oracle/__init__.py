"""Plain FP64 CPU oracle for the IMDP abstraction (test infrastructure).

This package is the reference the CUDA path is checked against. Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` /
``--impl reference`` legs may import it; the product path never does. It
shares no code with the CUDA library: the arithmetic lives in
``impact_oracle.c`` (compiled with gcc by :func:`build`), this module only
marshals arguments through ctypes.

A *problem* is any object with the attributes ``kind`` (0 affine, 1 unicycle,
2 caller images), ``A``, ``B``, ``c``, ``images``, ``lo``, ``hi``, ``cells``,
``inputs``, ``sigma`` and ``cutoff`` (numpy-convertible; unused ones may be
``None``). Rows are numbered ``cell * n_inputs + j`` with the cell id in C
order (last dimension fastest).

Regions (Sec. 3.1, Alg. 1, Remark 4.1): cells are labelled target / avoid
when their centre lies in a target / avoid box; the per-row vectors R and A
are either the paper's sums of the per-cell bounds over the labelled cells
or one box relaxation per region box (the box's cells taken as one big
target), the sink added to A.

Sampled noise (Sec. 4.1, full covariance or a custom distribution by
Monte-Carlo integration): given noise draws w_s, a row's up / lo for target
t are the fractions of draws for which the image box moved by w_s meets t /
lies inside t; the sink counts draws that leave the domain in part / whole.

Parity pins: every function here is pinned by ``tests/test_oracle_pins.py``
(library CDF, telescoping identity, 1-D closed form, brute-force argmax for
separable systems, Monte-Carlo containment, noise sampling, invariants,
degenerate cells, Table 1 row counts). The relaxation is pinned to the
paper's exact per-cell min/max (Def. 3.1) only where the two coincide
(separable dynamics); for coupled dynamics only its soundness is pinned, and
agreement with the paper's NLopt optimiser is "parity unpinned" (the paper
prints no probability values).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "impact_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``impact_oracle.c`` with gcc (OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("n", ctypes.c_int),
        ("m", ctypes.c_int),
        ("A", ctypes.c_void_p),
        ("B", ctypes.c_void_p),
        ("c", ctypes.c_void_p),
        ("images", ctypes.c_void_p),
        ("lo", ctypes.c_void_p),
        ("hi", ctypes.c_void_p),
        ("cells", ctypes.c_void_p),
        ("n_inputs", ctypes.c_int),
        ("inputs", ctypes.c_void_p),
        ("sigma", ctypes.c_void_p),
        ("cutoff", ctypes.c_double),
    ]


class Oracle:
    """One compiled oracle library (the default build, or a variant built from
    another source file, e.g. by the pin tests' planted-mistake checks)."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        P = ctypes.POINTER(_Problem)
        lib.oracle_phi_diff.restype = ctypes.c_double
        lib.oracle_phi_diff.argtypes = [ctypes.c_double] * 4
        lib.oracle_edge.restype = ctypes.c_double
        lib.oracle_edge.argtypes = [P, ctypes.c_int, ctypes.c_int]
        lib.oracle_image.restype = None
        lib.oracle_image.argtypes = [P, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_row_dense.restype = None
        lib.oracle_row_dense.argtypes = [P, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_run.restype = ctypes.c_void_p
        lib.oracle_run.argtypes = [P, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int64)]
        lib.oracle_fetch.restype = None
        lib.oracle_fetch.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 7
        lib.oracle_release.restype = None
        lib.oracle_release.argtypes = [ctypes.c_void_p]
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_max_threads.argtypes = []
        lib.oracle_cell_of.restype = ctypes.c_int
        lib.oracle_cell_of.argtypes = [P, ctypes.c_int, ctypes.c_double]
        lib.oracle_run_mc.restype = ctypes.c_void_p
        lib.oracle_run_mc.argtypes = [P, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
        lib.oracle_box_cells.restype = ctypes.c_int
        lib.oracle_box_cells.argtypes = [P] + [ctypes.c_void_p] * 4
        lib.oracle_labels.restype = None
        lib.oracle_labels.argtypes = [P, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]
        lib.oracle_region_rows.restype = None
        lib.oracle_region_rows.argtypes = [P, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]
        self.lib = lib
        self.path = lib_path

    def phi_diff(self, c: float, e: float, m: float, sigma: float) -> float:
        """g(c, e; m) = Phi((e-m)/sigma) - Phi((c-m)/sigma) (Def. 2.2, one dimension)."""
        return self.lib.oracle_phi_diff(float(c), float(e), float(m), float(sigma))

    def edges(self, prob, d: int) -> np.ndarray:
        """All N_d + 1 edges of dimension d."""
        mp = _Marshalled(prob)
        return np.array([self.lib.oracle_edge(ctypes.byref(mp.struct), d, i)
                         for i in range(int(mp.cells[d]) + 1)])

    def image(self, prob, row: int):
        """Interval image (m_lo, m_hi) of f(., u_j) over the source cell of ``row``."""
        mp = _Marshalled(prob)
        lo = np.zeros(mp.n)
        hi = np.zeros(mp.n)
        self.lib.oracle_image(ctypes.byref(mp.struct), int(row), lo.ctypes.data, hi.ctypes.data)
        return lo, hi

    def row_dense(self, prob, row: int):
        """Dense (up, lo) over every target cell plus (sink_lo, sink_up) for one row."""
        mp = _Marshalled(prob)
        T = mp.total_cells
        up = np.empty(T)
        lo = np.empty(T)
        sl = ctypes.c_double()
        su = ctypes.c_double()
        self.lib.oracle_row_dense(ctypes.byref(mp.struct), int(row), up.ctypes.data,
                                  lo.ctypes.data, ctypes.addressof(sl), ctypes.addressof(su))
        return up, lo, sl.value, su.value

    def build_rows(self, prob, rows=None, threads: int = 0) -> "OracleCSR":
        """CSR bounds of the given rows (all rows when ``rows`` is None)."""
        mp = _Marshalled(prob)
        if rows is None:
            rows = np.arange(mp.rows, dtype=np.int64)
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        lib = self.lib
        nnz = ctypes.c_int64()
        h = lib.oracle_run(ctypes.byref(mp.struct), rows.ctypes.data, int(rows.shape[0]),
                           int(threads), ctypes.byref(nnz))
        try:
            R = int(rows.shape[0])
            k = max(nnz.value, 1)
            out = OracleCSR(rows=rows, row_ptr=np.empty(R + 1, np.int64),
                            col=np.empty(k, np.int32), lo=np.empty(k), up=np.empty(k),
                            sink_lo=np.empty(R), sink_up=np.empty(R), trunc=np.empty(R))
            lib.oracle_fetch(h, out.row_ptr.ctypes.data, out.col.ctypes.data,
                             out.lo.ctypes.data, out.up.ctypes.data, out.sink_lo.ctypes.data,
                             out.sink_up.ctypes.data, out.trunc.ctypes.data)
            out.col = out.col[:nnz.value]
            out.lo = out.lo[:nnz.value]
            out.up = out.up[:nnz.value]
        finally:
            lib.oracle_release(h)
        return out

    def cell_of(self, prob, d: int, y: float) -> int:
        """Cell of dimension d holding coordinate y (-1 below, N above)."""
        mp = _Marshalled(prob)
        return int(self.lib.oracle_cell_of(ctypes.byref(mp.struct), int(d), float(y)))

    def build_rows_mc(self, prob, samples, rows=None, threads: int = 0) -> "OracleCSR":
        """Rows built from sampled noise: samples is an (S, n) array of noise
        draws; lo / up / sink are sample fractions (see oracle_mc_row)."""
        mp = _Marshalled(prob)
        if rows is None:
            rows = np.arange(mp.rows, dtype=np.int64)
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        W = np.ascontiguousarray(np.asarray(samples, np.float64).reshape(-1, mp.n).T)
        S = int(W.shape[1])
        nnz = ctypes.c_int64()
        h = self.lib.oracle_run_mc(ctypes.byref(mp.struct), rows.ctypes.data, int(rows.shape[0]),
                                   W.ctypes.data, S, int(threads), ctypes.byref(nnz))
        return self._fetch(h, rows, nnz.value)

    def _fetch(self, h, rows, nnz):
        lib = self.lib
        try:
            R = int(rows.shape[0])
            k = max(nnz, 1)
            out = OracleCSR(rows=rows, row_ptr=np.empty(R + 1, np.int64),
                            col=np.empty(k, np.int32), lo=np.empty(k), up=np.empty(k),
                            sink_lo=np.empty(R), sink_up=np.empty(R), trunc=np.empty(R))
            lib.oracle_fetch(h, out.row_ptr.ctypes.data, out.col.ctypes.data,
                             out.lo.ctypes.data, out.up.ctypes.data, out.sink_lo.ctypes.data,
                             out.sink_up.ctypes.data, out.trunc.ctypes.data)
            out.col = out.col[:nnz]
            out.lo = out.lo[:nnz]
            out.up = out.up[:nnz]
        finally:
            lib.oracle_release(h)
        return out

    def max_threads(self) -> int:
        """OpenMP threads the oracle uses by default."""
        return int(self.lib.oracle_max_threads())

    def box_cells(self, prob, box):
        """Index range (first, last) per dimension of the cells whose centre
        lies in the closed box ``(lo, hi)``, or None when there is none."""
        mp = _Marshalled(prob)
        lo, hi = (_f64(b).reshape(mp.n) for b in box)
        first = np.zeros(mp.n, np.int32)
        last = np.zeros(mp.n, np.int32)
        ok = self.lib.oracle_box_cells(ctypes.byref(mp.struct), lo.ctypes.data, hi.ctypes.data,
                                       first.ctypes.data, last.ctypes.data)
        return (first, last) if ok else None

    def region_labels(self, prob, target=(), avoid=()) -> np.ndarray:
        """uint8 label per cell: 0 free, 1 target, 2 avoid (avoid wins)."""
        mp = _Marshalled(prob)
        (tl, th), (al, ah) = _box_arrays(target, mp.n), _box_arrays(avoid, mp.n)
        out = np.zeros(mp.total_cells, np.uint8)
        self.lib.oracle_labels(ctypes.byref(mp.struct), len(target), tl.ctypes.data,
                               th.ctypes.data, len(avoid), al.ctypes.data, ah.ctypes.data,
                               out.ctypes.data)
        return out

    def region_vectors(self, prob, rows=None, target=(), avoid=(), mode: str = "box"):
        """(R_min, R_max, A_min, A_max) per row; mode "box" (one relaxation
        per region box) or "cells" (the paper's sums of per-cell bounds)."""
        mp = _Marshalled(prob)
        if rows is None:
            rows = np.arange(mp.rows, dtype=np.int64)
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        if mode == "box":
            spans = [self.box_cells(prob, b) for b in list(target) + list(avoid)]
            spans = [s for s in spans if s is not None]
            for i in range(len(spans)):
                for k in range(i):
                    (f1, l1), (f2, l2) = spans[i], spans[k]
                    if np.all(np.maximum(f1, f2) <= np.minimum(l1, l2)):
                        raise ValueError("region boxes share cells")
        (tl, th), (al, ah) = _box_arrays(target, mp.n), _box_arrays(avoid, mp.n)
        labels = self.region_labels(prob, target, avoid)
        out = np.zeros((rows.shape[0], 4))
        self.lib.oracle_region_rows(ctypes.byref(mp.struct), rows.ctypes.data,
                                    int(rows.shape[0]), 0 if mode == "box" else 1,
                                    labels.ctypes.data, len(target), tl.ctypes.data,
                                    th.ctypes.data, len(avoid), al.ctypes.data, ah.ctypes.data,
                                    out.ctypes.data)
        return out[:, 0].copy(), out[:, 1].copy(), out[:, 2].copy(), out[:, 3].copy()


def default() -> Oracle:
    """The oracle compiled from ``impact_oracle.c`` (built on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build())
    return _lib


def compile_variant(source_text: str, out_dir: str) -> str:
    """Compile another version of the oracle source (same flags) into out_dir."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "variant.c")
    with open(src, "w") as f:
        f.write(source_text)
    lib = os.path.join(out_dir, "libvariant.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", "-fno-fast-math", src, "-o", lib, "-lm"], check=True)
    return lib


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _f64(x):
    return None if x is None else np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _box_arrays(boxes, n):
    """[(lo, hi), ...] -> two contiguous [count][n] arrays (at least one row)."""
    lo = np.zeros((max(len(boxes), 1), n))
    hi = np.zeros((max(len(boxes), 1), n))
    for k, (a, b) in enumerate(boxes):
        lo[k] = np.asarray(a, np.float64).reshape(n)
        hi[k] = np.asarray(b, np.float64).reshape(n)
    return np.ascontiguousarray(lo), np.ascontiguousarray(hi)


class _Marshalled:
    """Keeps the numpy buffers alive while the C struct points into them."""

    def __init__(self, prob):
        self.kind = int(prob.kind)
        self.lo = _f64(prob.lo)
        self.hi = _f64(prob.hi)
        self.cells = np.ascontiguousarray(np.asarray(prob.cells, dtype=np.int32))
        self.sigma = _f64(prob.sigma)
        self.n = int(self.lo.shape[0])
        inputs = np.asarray(prob.inputs if prob.inputs is not None else np.zeros((1, 0)),
                            dtype=np.float64)
        if inputs.ndim == 1:
            inputs = inputs.reshape(-1, 1)
        self.inputs = np.ascontiguousarray(inputs)
        self.n_inputs = int(self.inputs.shape[0])
        self.m = int(self.inputs.shape[1])
        self.A = _f64(getattr(prob, "A", None))
        self.B = _f64(getattr(prob, "B", None))
        self.c = _f64(getattr(prob, "c", None))
        self.images = _f64(getattr(prob, "images", None))
        if self.B is not None and self.B.size == 0:
            self.B = None

        def ptr(a):
            return None if a is None else a.ctypes.data

        self.struct = _Problem(self.kind, self.n, self.m, ptr(self.A), ptr(self.B), ptr(self.c),
                               ptr(self.images), ptr(self.lo), ptr(self.hi), ptr(self.cells),
                               self.n_inputs, ptr(self.inputs), ptr(self.sigma),
                               float(prob.cutoff))

    @property
    def total_cells(self) -> int:
        return int(np.prod(self.cells.astype(np.int64)))

    @property
    def rows(self) -> int:
        return self.total_cells * self.n_inputs


@dataclass
class OracleCSR:
    rows: np.ndarray      # int64 [R]   the row ids, in the order built
    row_ptr: np.ndarray   # int64 [R+1]
    col: np.ndarray       # int32 [nnz]
    lo: np.ndarray        # f64   [nnz]
    up: np.ndarray        # f64   [nnz]
    sink_lo: np.ndarray   # f64   [R]
    sink_up: np.ndarray   # f64   [R]
    trunc: np.ndarray     # f64   [R]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row(self, k: int):
        a, b = int(self.row_ptr[k]), int(self.row_ptr[k + 1])
        return self.col[a:b], self.lo[a:b], self.up[a:b]


def phi_diff(c, e, m, sigma):
    return default().phi_diff(c, e, m, sigma)


def edges(prob, d):
    return default().edges(prob, d)


def image(prob, row):
    return default().image(prob, row)


def row_dense(prob, row):
    return default().row_dense(prob, row)


def build_rows(prob, rows=None, threads: int = 0) -> OracleCSR:
    return default().build_rows(prob, rows, threads)


def max_threads() -> int:
    return default().max_threads()


def region_labels(prob, target=(), avoid=()):
    return default().region_labels(prob, target, avoid)


def build_rows_mc(prob, samples, rows=None, threads: int = 0) -> OracleCSR:
    return default().build_rows_mc(prob, samples, rows, threads)


def region_vectors(prob, rows=None, target=(), avoid=(), mode="box"):
    return default().region_vectors(prob, rows, target, avoid, mode)
