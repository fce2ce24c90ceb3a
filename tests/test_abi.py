"""The C-ABI library builds, loads and exports what include/impact.h declares
(CPU only: no compute call needs a GPU here)."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2401_03555_gb300 import build as B
from paper_2401_03555_gb300 import impact, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "impact.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(impact_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return impact.load()


def test_header_lists_the_entry_points():
    assert set(declared_functions()) == set(impact.ENTRY_POINTS)


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(B.LIB)
    for name in declared_functions():
        assert hasattr(raw, name), name


def test_version(lib):
    assert impact.version() == 301


@pytest.mark.parametrize("make", [W.robot_2d, W.room_5d, W.unicycle_3d, W.building_7d])
def test_plan_counts_rows_and_bounds(lib, make):
    prob = make()
    rows, nnz_bound, nbytes = impact.plan(prob, "fp32")
    assert rows == prob.rows
    assert prob.rows <= nnz_bound <= prob.rows * prob.total_cells
    assert nbytes >= nnz_bound * 12


def test_plan_dense_bound_is_exact(lib):
    prob = W.robot_2d()
    rows, nnz_bound, _ = impact.plan(prob, "fp64")
    assert nnz_bound == prob.rows * prob.total_cells   # cutoff 0 keeps every pair


@pytest.mark.parametrize("mutate, msg", [
    (lambda p: setattr(p, "cutoff", 1.0), "cutoff"),
    (lambda p: setattr(p, "cutoff", -0.1), "cutoff"),
    (lambda p: setattr(p, "sigma", np.zeros(p.n)), "sigma"),
    (lambda p: setattr(p, "hi", p.lo.copy()), "lo < hi"),
    (lambda p: setattr(p, "cells", np.zeros(p.n, np.int32)), "cells"),
    (lambda p: setattr(p, "cells", np.full(p.n, 50000, np.int32)), "2^31"),
    (lambda p: setattr(p, "inputs", np.zeros((0, 2))), "inputs.count"),
    (lambda p: setattr(p, "sigma", np.full(p.n, np.nan)), "sigma"),
    (lambda p: setattr(p, "hi", np.full(p.n, np.inf)), "finite lo < hi"),
    (lambda p: (setattr(p, "inputs", np.zeros((1, 9))), setattr(p, "B", np.zeros((p.n, 9)))),
     "inputs.m"),
])
def test_plan_rejects_bad_arguments(lib, mutate, msg):
    prob = W.room_5d()
    mutate(prob)
    with pytest.raises(impact.ImpactError) as e:
        impact.plan(prob, "fp32")
    assert e.value.status == impact.IMPACT_ERR_ARG
    assert msg in str(e.value)


def test_plan_accepts_wide_fp32_windows(lib):
    """Dense 400^2 robot: a 400-cell window per dimension fits one warp's
    shared memory (8 bytes per window target, 48 per edge during setup)."""
    rows, nnz_bound, _ = impact.plan(W.robot_2d(cells_per_dim=400), "fp32")
    assert rows == 400 * 400 * 9 and nnz_bound == rows * 400 * 400


def test_plan_rejects_windows_beyond_one_warp(lib):
    prob = W.robot_2d(cells_per_dim=4000)   # dense: 8000 window targets per row
    with pytest.raises(impact.ImpactError) as e:
        impact.plan(prob, "fp32")
    assert e.value.status == impact.IMPACT_ERR_ARG and "shared memory" in str(e.value)


def test_fast_division_constants_are_exact():
    """The kernels divide cell ids by N with q = (umulhi(x, m) + x) >> s; the
    host builds (m, s). Check the formula on every x class that matters."""
    rng = np.random.default_rng(0)
    for N in list(range(1, 300)) + [1021, 4096, 65535, 65536, 100003, 2**20 + 7, 2**30 + 3]:
        l = 0
        while (1 << l) < N:
            l += 1
        m = ((((1 << l) - N) << 32) // N + 1) & 0xffffffff
        ks = np.unique(np.concatenate([np.arange(0, 64), rng.integers(0, (2**31 - 1) // N + 1, 64)]))
        near = (ks[:, None] * N + np.arange(-2, 3)[None, :]).ravel()   # around multiples of N
        xs = np.concatenate([rng.integers(0, 2**31, 2000), np.arange(0, min(3 * N + 5, 4096)),
                             near, [2**31 - 1, 2**31 - N, (2**31 - 1) // N * N]]).astype(np.int64)
        xs = xs[(xs >= 0) & (xs < 2**31)]
        q = ((xs * m) >> 32) + xs >> l
        assert np.array_equal(q, xs // N), N


def test_batch_plan_concatenates_rows_and_bounds(lib):
    probs = [W.robot_2d(cells_per_dim=7), W.room_5d(cells_per_dim=4),
             W.random_linear(3, min_cells=300, max_cells=3000)]
    b = impact.Batch(probs, "fp32")
    want = np.concatenate([[0], np.cumsum([p.rows for p in probs])])
    assert np.array_equal(b.row_offsets, want)
    bounds = [impact.plan(p, "fp32")[1] for p in probs]
    assert b.nnz_bound == sum(bounds)
    assert b.ws_bytes >= sum(impact.workspace_bytes(p, "fp32") for p in probs) // 2


def test_batch_plan_names_the_failing_request(lib):
    bad = W.room_5d(cells_per_dim=4)
    bad.sigma = np.array([0.2, 0.2, -1.0, 0.2, 0.2])
    with pytest.raises(impact.ImpactError, match="request 1"):
        impact.Batch([W.robot_2d(cells_per_dim=5), bad], "fp32")


@pytest.mark.parametrize("field,value,msg", [("count_warps", 9, "warps"),
                                              ("emit_warps", -1, "warps"),
                                              ("spin_limit", -5, "spin_limit"),
                                              ("guard_row", -6, "guard_row")])
def test_batch_plan_rejects_bad_tuning(lib, field, value, msg):
    t = impact.tuning(**{field: value})
    with pytest.raises(impact.ImpactError, match=msg):
        impact.Batch([W.robot_2d(cells_per_dim=5)], "fp32", tune=t)


def test_batch_plan_rejects_a_one_pass_flag_other_than_0_or_1(lib):
    t = impact.tuning()
    t.one_pass = 2
    with pytest.raises(impact.ImpactError, match="one_pass"):
        impact.Batch([W.robot_2d(cells_per_dim=5)], "fp32", tune=t)


def test_plan_accepts_the_largest_dimension(lib):
    prob = W.random_linear(2, min_cells=5000, max_cells=7000, dims=(8,))
    assert prob.n == 8
    for precision in ("fp32", "fp64"):
        rows, nnz_bound, _ = impact.plan(prob, precision)
        assert rows == prob.rows
        assert rows <= nnz_bound <= prob.rows * prob.total_cells


def test_plan_rejects_more_than_eight_dimensions(lib):
    n = 9
    prob = W.Problem(name="9d", kind=W.AFFINE, lo=np.full(n, -1.0), hi=np.full(n, 1.0),
                     cells=np.full(n, 2, np.int32), inputs=np.zeros((1, 1)),
                     sigma=np.full(n, 0.3), cutoff=1e-8, A=0.9 * np.eye(n),
                     B=np.zeros((n, 1)), c=np.zeros(n))
    with pytest.raises(impact.ImpactError) as e:
        impact.plan(prob, "fp32")
    assert e.value.status == impact.IMPACT_ERR_ARG
    assert "[1, 8]" in str(e.value)


def test_plan_rejects_a_unicycle_of_other_dimension(lib):
    prob = W.unicycle_3d(nx=5, ny=5, nth=5)
    prob.lo, prob.hi = np.r_[prob.lo, 0.0], np.r_[prob.hi, 1.0]
    prob.cells = np.r_[prob.cells, 2].astype(np.int32)
    prob.sigma = np.r_[prob.sigma, 0.3]
    with pytest.raises(impact.ImpactError, match="unicycle needs n = 3"):
        impact.plan(prob, "fp32")


STRUCTS = [("_System", "impact_system"), ("_Grid", "impact_grid"), ("_Inputs", "impact_inputs"),
           ("_CSR", "impact_csr"), ("_Request", "impact_request"), ("_Tuning", "impact_tuning"),
           ("_Regions", "impact_regions"), ("_SynthOptions", "impact_synth_options"),
           ("_ServerConfig", "impact_server_config"), ("_ServerStats", "impact_server_stats_t")]


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes mirror in the binding has the size and field offsets that
    a C compiler gives the header's struct (host-only: gcc and the header)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    header = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "include", "impact.h")
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{header}"',
             "int main(void) {"]
    want = []
    for py, c in STRUCTS:
        st = getattr(impact, py)
        lines.append(f'  printf("%zu\\n", sizeof({c}));')
        want.append(ctypes.sizeof(st))
        for name, _ in st._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({c}, {name}));')
            want.append(getattr(st, name).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-o", str(exe), str(src)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got == want
