"""The CUDA path against the CPU oracle, element by element (needs a GPU).

Every build goes through the C ABI (impact_count + impact_emit via the
binding, or impact_build through impact.Builder). Small problems are compared
on every row; the full-size workloads on seeded samples of rows (plus the
domain's corner rows), in the same launch configuration the benchmark times.
"""

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


def run_and_compare(orc, prob, precision, rows=None, builder=False):
    if builder and precision == "fp32":
        b = impact.Builder(prob, precision)
        b.run()
        csr = b.result()
    else:
        csr = impact.build(prob, precision)
    torch.cuda.synchronize()
    if rows is None:
        rows = np.arange(prob.rows)
    ocsr = orc.build_rows(prob, rows)
    rep = PA.compare(prob, csr, ocsr, orc, precision)
    rep.assert_ok()
    return rep, csr


SMALL = {
    "robot2d-21": lambda: W.robot_2d(),
    "robot2d-5": lambda: W.robot_2d(cells_per_dim=5),
    "unicycle-9x9x7": lambda: W.unicycle_3d(nx=9, ny=9, nth=7),
    "room5d-4": lambda: W.room_5d(cells_per_dim=4),
    "bas4d": lambda: W.bas_4d(eta_scale=1.0),
    "linear-seed3": lambda: W.random_linear(3, min_cells=300, max_cells=3000),
    "linear-seed8": lambda: W.random_linear(8, min_cells=300, max_cells=3000),
    "building7d-3": lambda: W.building_7d(cells_per_dim=3),
    # the boundary's largest dimension: 8-D coupled linear system, 3^8 cells
    "linear-8d": lambda: W.random_linear(2, min_cells=5000, max_cells=7000, dims=(8,)),
}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(SMALL))
def test_small_problems_every_row(orc, name, precision):
    prob = SMALL[name]()
    rows = None if prob.rows <= 4000 else W.sample_rows(prob, 400, seed=1)
    rep, csr = run_and_compare(orc, prob, precision, rows)
    assert rep.pairs > 0
    if precision == "fp64":
        assert rep.max_dup <= PA.TOL64


def test_robot_dense_is_complete(orc):
    prob = W.robot_2d()
    csr = impact.build(prob, "fp64")
    assert csr.nnz == prob.rows * prob.total_cells   # cutoff 0: every pair kept


FULL = {
    "room5d-11": (lambda: W.room_5d(), 24),
    "unicycle-51x51x25": (lambda: W.unicycle_3d(), 24),
    "building7d-6": (lambda: W.building_7d(), 12),
}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name", list(FULL))
def test_full_size_sampled_rows(orc, name, precision):
    make, count = FULL[name]
    prob = make()
    rows = W.sample_rows(prob, count, seed=7)
    rep, csr = run_and_compare(orc, prob, precision, rows, builder=True)
    flags = csr.row_flags
    assert int((flags != 0).sum()) == 0


def wide_unicycle():
    """A unicycle on a fine grid of a small domain with cutoff 1e-10: in x
    and y the window spans all 70 cells (the noise reaches 44 cells)."""
    p = W.unicycle_3d(nx=70, ny=70, nth=3, cutoff=1e-10)
    p.lo, p.hi = np.array([-1.5, -1.5, -np.pi]), np.array([1.5, 1.5, np.pi])
    p.inputs = p.inputs[[3, 17]]
    return p


WIDE = {
    "robot2d-100-dense": (lambda: W.robot_2d(cells_per_dim=100), 40),
    "unicycle-70x70x3-1e-10": (wide_unicycle, 30),
}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name", list(WIDE))
def test_wide_windows_sampled_rows(orc, name, precision):
    """Windows of more than 64 cells per dimension (the first FP32 walk
    refused them): dense builds and a small cutoff on a fine grid."""
    make, count = WIDE[name]
    prob = make()
    rows = W.sample_rows(prob, count, seed=5)
    rep, csr = run_and_compare(orc, prob, precision, rows, builder=True)
    assert rep.pairs > 64 * len(rows)


def test_fp32_vs_fp64_gpu_bracketing_full(orc):
    """Every FP32 pair brackets the FP64 GPU pair of the same target."""
    prob = W.room_5d(cells_per_dim=6)
    c64 = impact.build(prob, "fp64")
    c32 = impact.build(prob, "fp32")
    rp64, rp32 = c64.row_ptr.cpu().numpy(), c32.row_ptr.cpu().numpy()
    col64, col32 = c64.col.cpu().numpy(), c32.col.cpu().numpy()
    lo64, up64 = c64.lo.cpu().numpy(), c64.up.cpu().numpy()
    lo32, up32 = c32.lo.cpu().numpy().astype(np.float64), c32.up.cpu().numpy().astype(np.float64)
    for r in range(prob.rows):
        a, b = rp64[r], rp64[r + 1]
        a2, b2 = rp32[r], rp32[r + 1]
        c, i64, i32 = np.intersect1d(col64[a:b], col32[a2:b2], return_indices=True)
        assert len(c) == b - a, r     # FP32 keeps every FP64-kept target
        assert np.all(lo32[a2:b2][i32] <= lo64[a:b][i64])
        assert np.all(up32[a2:b2][i32] >= up64[a:b][i64])
        assert np.all(np.abs(lo32[a2:b2][i32] - lo64[a:b][i64]) <= PA.TOL32)
        assert np.all(np.abs(up32[a2:b2][i32] - up64[a:b][i64]) <= PA.TOL32)
    s = c32.sink_lo.cpu().numpy() <= c64.sink_lo.cpu().numpy()
    assert np.all(s)
    assert np.all(c32.sink_up.cpu().numpy() >= c64.sink_up.cpu().numpy())


def test_degenerate_point_images(orc):
    rng = np.random.default_rng(4)
    base = W.room_5d(cells_per_dim=5)
    pts = rng.uniform(16.5, 23.5, size=(base.rows, 5))
    prob = W.with_images(base, np.stack([pts, pts], axis=2))
    rows = W.sample_rows(prob, 150, seed=2)
    rep64, c64 = run_and_compare(orc, prob, "fp64", rows)
    assert torch.equal(c64.lo, c64.up)                 # lo == up bit for bit
    assert torch.equal(c64.sink_lo, c64.sink_up)
    rep32, c32 = run_and_compare(orc, prob, "fp32", rows)
    gap = (c32.up.double() - c32.lo.double()).max().item()
    assert gap <= 2 * PA.TOL32


def test_rows_leaving_the_domain_are_empty(orc):
    prob = W.room_5d(cells_per_dim=4)
    prob.c = prob.c + 40.0            # every image lands far above the domain
    for precision in ("fp64", "fp32"):
        rep, csr = run_and_compare(orc, prob, precision, W.sample_rows(prob, 50, seed=3))
        assert csr.nnz == 0
        assert torch.all(csr.sink_lo > 1 - 1e-9)


def test_one_dimension_one_cell(orc):
    prob = W.Problem(name="tiny", kind=W.AFFINE, lo=np.array([0.0]), hi=np.array([1.0]),
                     cells=np.array([1], np.int32), inputs=np.array([[0.0], [0.7]]),
                     sigma=np.array([0.3]), cutoff=1e-8, A=np.eye(1) * 0.5,
                     B=np.eye(1), c=np.zeros(1))
    for precision in ("fp64", "fp32"):
        run_and_compare(orc, prob, precision)


def test_library_owned_output_matches():
    prob = W.unicycle_3d(nx=11, ny=11, nth=9)
    rows, nnz, owned = impact.build_library_owned(prob, "fp32")
    assert owned == 1 and rows == prob.rows
    assert nnz == impact.build(prob, "fp32").nnz


def test_repeat_builds_are_bitwise_identical():
    prob = W.room_5d(cells_per_dim=6)
    b = impact.Builder(prob, "fp32")
    b.run()
    first = [t.clone() for t in (b.result().col, b.result().lo, b.result().up,
                                 b.result().trunc, b.result().sink_lo)]
    b.run()
    second = (b.result().col, b.result().lo, b.result().up, b.result().trunc,
              b.result().sink_lo)
    for x, y in zip(first, second):
        assert torch.equal(x, y)


def test_capacity_too_small_reports_needed_pairs():
    prob = W.room_5d(cells_per_dim=5)
    need = impact.build(prob, "fp32").nnz
    b = impact.Builder(prob, "fp32", capacity=need - 1)
    with pytest.raises(impact.ImpactError) as e:
        b.run()
    assert e.value.status == impact.IMPACT_ERR_CAPACITY
    assert str(need) in str(e.value)


def test_pairs_written_straight_to_pinned_host_memory():
    """col/lo/up in pinned host memory: the emit kernel writes them over the
    host link; the result equals the device build bit for bit."""
    prob = W.room_5d(cells_per_dim=5)
    ref = impact.build(prob, "fp32")
    b = impact.Builder(prob, "fp32", capacity=ref.nnz, pairs_on_host=True)
    assert not b.pairs_buf["col"].is_cuda
    assert b.run() == ref.nnz
    torch.cuda.synchronize()
    got = b.result()
    for name in ("col", "lo", "up"):
        x = getattr(got, name).numpy()
        y = getattr(ref, name).cpu().numpy()
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8)), name
    assert torch.equal(got.row_ptr.cpu(), ref.row_ptr.cpu())
