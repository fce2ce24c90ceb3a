"""Sampled noise through the C ABI (impact_build_mc) against the CPU oracle
(needs a GPU). The draws are inputs shared by both sides, so the counts -- and
with them every value count / S -- must agree exactly."""

import numpy as np
import pytest
import torch

import oracle
import oracle_pins as OP
from paper_2401_03555_gb300 import impact, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    impact.load()


def correlated(rng, S, scales, rho=0.5):
    n = len(scales)
    C = np.full((n, n), rho) + (1.0 - rho) * np.eye(n)
    C = C * np.outer(scales, scales)
    return rng.normal(size=(S, n)) @ np.linalg.cholesky(C).T


def cases():
    rng = np.random.default_rng(71)
    robot = W.robot_2d(cells_per_dim=9)                        # cutoff 0: dense rows
    room = W.room_5d(cells_per_dim=4, cutoff=2e-3)
    img = OP.mc_images(W.robot_2d(cells_per_dim=7), 5, [1.3, 0.4])
    img.cutoff = 0.01
    lin = W.random_linear(5, min_cells=200, max_cells=2000)
    lin.cutoff = 5e-3
    uni = W.unicycle_3d(nx=8, ny=8, nth=7, cutoff=5e-3)
    return [
        ("robot full covariance", robot, correlated(rng, 4000, [0.75, 0.75], 0.6), None),
        ("unicycle correlated", uni, correlated(rng, 2000, [0.3, 0.3, 0.2], 0.5),
         W.sample_rows(uni, 24, seed=5)),
        ("room 4^5 correlated", room, correlated(rng, 3000, [0.2] * 5, 0.3),
         W.sample_rows(room, 24, seed=3)),
        ("wide images", img, rng.normal(size=(5000, 2)) * 0.9, None),
        ("random linear", lin, correlated(rng, 2000, np.full(lin.n, 0.3), 0.4),
         W.sample_rows(lin, 24, seed=4)),
    ]


CASES = cases()


def counts(v, S):
    return np.round(np.asarray(v, np.float64) * S).astype(np.int64)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("k", range(len(CASES)))
def test_counts_equal_the_oracle(k, precision):
    name, prob, w, rows = CASES[k]
    S = w.shape[0]
    got = impact.build_mc(prob, w, precision)
    rows = np.arange(prob.rows) if rows is None else np.asarray(rows, np.int64)
    ref = oracle.build_rows_mc(prob, w, rows)
    rp = got.row_ptr.cpu().numpy()
    col, lo, up = got.col.cpu().numpy(), got.lo.cpu().numpy(), got.up.cpu().numpy()
    sl, su, tr = (t.cpu().numpy() for t in (got.sink_lo, got.sink_up, got.trunc))
    for i, r in enumerate(rows):
        a, b = rp[r], rp[r + 1]
        rc, rlo, rup = ref.row(i)
        assert np.array_equal(col[a:b], rc), (name, r)
        if precision == "fp64":
            assert np.array_equal(lo[a:b], rlo) and np.array_equal(up[a:b], rup), (name, r)
        else:
            assert np.array_equal(counts(lo[a:b], S), counts(rlo, S)), (name, r)
            assert np.array_equal(counts(up[a:b], S), counts(rup, S)), (name, r)
            assert np.all(lo[a:b] <= rlo) and np.all(up[a:b] >= rup), (name, r)
        assert sl[r] == ref.sink_lo[i] and su[r] == ref.sink_up[i] and tr[r] == ref.trunc[i], \
            (name, r)


def test_window_limit_is_reported():
    prob = W.room_5d(cells_per_dim=11)
    w = np.random.default_rng(1).normal(size=(64, 5)) * 50.0     # reaches every cell
    with pytest.raises(impact.ImpactError) as ei:
        impact.build_mc(prob, w)
    assert ei.value.status == impact.IMPACT_ERR_ARG


def test_point_images_agree_with_the_gaussian_build():
    """Zero-width images and many Gaussian draws: the sampled bounds close in
    on the closed-form Gaussian masses of impact_build."""
    base = W.robot_2d(cells_per_dim=9)
    prob = OP.mc_images(base, 8, [0.0, 0.0])
    S = 200_000
    w = np.random.default_rng(2).normal(size=(S, 2)) * np.asarray(base.sigma)
    mc = impact.build_mc(prob, w, "fp64")
    ex = impact.build(prob, "fp64")
    assert torch.equal(mc.lo, mc.up)
    assert torch.equal(mc.row_ptr, ex.row_ptr) and torch.equal(mc.col, ex.col)
    p = ex.up.cpu().numpy()
    sd = np.sqrt(p * (1 - p) / S)
    assert np.all(np.abs(mc.up.cpu().numpy() - p) <= 5 * sd + 1.0 / S)
