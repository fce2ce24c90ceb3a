"""Batches of builds through the C ABI (impact_batch_*, impact_graph_*,
impact_batch_tune) against single builds and the CPU oracle (needs a GPU).

A batch runs each kernel once for all its builds; its result must equal,
bit for bit, the builds run one at a time, and match the oracle row by row
with the same tolerances as a single build."""

import numpy as np
import pytest
import torch

import oracle
import parity as PA
from paper_2401_03555_gb300 import impact, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    impact.load()


def mixed_small():
    return [W.robot_2d(cells_per_dim=7), W.room_5d(cells_per_dim=4),
            W.unicycle_3d(nx=9, ny=9, nth=7), W.random_linear(3, min_cells=300, max_cells=3000),
            W.building_7d(cells_per_dim=3), W.random_linear(8, min_cells=300, max_cells=3000),
            W.bas_4d(eta_scale=1.0)]


def host(csr):
    t = lambda x: x.cpu().numpy()
    return (t(csr.row_ptr), t(csr.col), t(csr.lo), t(csr.up), t(csr.sink_lo), t(csr.sink_up),
            t(csr.trunc), t(csr.row_flags))


def assert_same(a, b, what):
    names = ("row_ptr", "col", "lo", "up", "sink_lo", "sink_up", "trunc", "row_flags")
    for n, x, y in zip(names, host(a), host(b)):
        assert x.shape == y.shape and np.array_equal(x.view(np.uint8), y.view(np.uint8)), \
            f"{what}: {n} differs"


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_equals_single_builds_and_oracle(orc, precision):
    probs = mixed_small()
    res = impact.Batch(probs, precision).build()
    torch.cuda.synchronize()
    assert res.count == len(probs)
    for q, p in enumerate(probs):
        part = res.part(q)
        single = impact.build(p, precision)
        assert_same(part, single, f"{p.name} in the batch vs alone")
        rep = PA.compare(p, part, orc.build_rows(p, np.arange(p.rows)), orc, precision)
        rep.assert_ok()


def test_launch_shapes_give_identical_results():
    probs = mixed_small()
    ref = impact.Batch(probs, "fp32").build()
    for t in (impact.tuning(count_warps=2, emit_warps=8),
              impact.tuning(count_warps=8, emit_warps=2),
              impact.tuning(count_warps=3, emit_warps=5),
              impact.tuning(count_warps=1, emit_warps=1)):
        b = impact.Batch(probs, "fp32", tune=t)
        assert_same(b.build().csr, ref.csr, f"tuning {t.as_dict()} (library-owned, two passes)")
        nnz = ref.csr.nnz
        rb = impact.alloc_rows(b.rows)
        pb = impact.alloc_pairs(nnz, "fp32")
        assert b.build_into(rb, pb, nnz) == nnz
        got = impact.CSR("fp32", rb["row_ptr"], pb["col"][:nnz], pb["lo"][:nnz], pb["up"][:nnz],
                         rb["sink_lo"], rb["sink_up"], rb["trunc"], rb["row_flags"])
        assert_same(got, ref.csr, f"tuning {t.as_dict()} (caller arrays, one pass)")


def test_graph_replays_equal_the_batch_build():
    probs = mixed_small()
    b = impact.Batch(probs, "fp32")
    ref = b.build()
    nnz = ref.csr.nnz
    rb = impact.alloc_rows(b.rows)
    pb = impact.alloc_pairs(nnz, "fp32")
    g = b.graph(rb, pb, nnz)
    for _ in range(2):
        for t in list(rb.values()) + list(pb.values()):
            t.fill_(0)
        g.launch()
        torch.cuda.synchronize()
        assert g.result() == nnz
        got = impact.CSR("fp32", rb["row_ptr"], pb["col"][:nnz], pb["lo"][:nnz], pb["up"][:nnz],
                         rb["sink_lo"], rb["sink_up"], rb["trunc"], rb["row_flags"])
        assert_same(got, ref.csr, "graph replay")
    g.close()


def test_graph_reports_short_capacity():
    probs = mixed_small()[:3]
    b = impact.Batch(probs, "fp32")
    nnz = b.build().csr.nnz
    rb = impact.alloc_rows(b.rows)
    pb = impact.alloc_pairs(nnz - 1, "fp32")
    g = b.graph(rb, pb, nnz - 1)
    g.launch()
    torch.cuda.synchronize()
    with pytest.raises(impact.ImpactError) as ei:
        g.result()
    assert ei.value.status == impact.IMPACT_ERR_CAPACITY
    g.close()


def test_autotuner_returns_a_listed_shape():
    probs = mixed_small()
    b = impact.Batch(probs, "fp32")
    ref = b.build()
    nnz = ref.csr.nnz
    rb = impact.alloc_rows(b.rows)
    pb = impact.alloc_pairs(nnz, "fp32")
    best, ms = b.tune(rb, pb, nnz, reps=2)
    d = best.as_dict()
    assert d["count_warps"] in (2, 4, 6, 8) and d["emit_warps"] in (2, 4, 6, 8) and ms > 0
    assert_same(impact.Batch(probs, "fp32", tune=best).build().csr, ref.csr, "tuned shape")


def test_batched_family_sampled_rows(orc):
    """The batched workload's first 32 seeded systems in one batch (2.2e9
    pairs), tuned, on seeded sampled rows of every system."""
    probs = W.batched_family(32)
    b = impact.Batch(probs, "fp32")
    res = b.build()
    torch.cuda.synchronize()
    for q, p in enumerate(probs):
        rows = W.sample_rows(p, 12, seed=q)
        rep = PA.compare(p, res.part(q), orc.build_rows(p, rows), orc, "fp32")
        rep.assert_ok()
