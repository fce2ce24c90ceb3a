"""Interval-iteration synthesis on the GPU (impact_synthesize) against the
CPU oracle's synthesis on the oracle's own IMDP (needs a GPU)."""

import numpy as np
import pytest
import torch

import oracle
from oracle import synthesis as SY
from paper_2401_03555_gb300 import impact, workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    impact.load()


def robot(cells):
    prob = W.robot_2d(cells_per_dim=cells)
    labels = W.region_labels(prob, target=([3, 3], [7, 7]), avoid=([-7, -7], [-3, -3]))
    return prob, labels


def optimal_margin_ok(ocsr, res, labels, U, gpu_policy, spec):
    """The GPU policy reaches the oracle's phase-1 optimum at the oracle's
    final V0 (several inputs may tie)."""
    free = np.nonzero(labels == SY.FREE)[0]
    reach = spec == SY.REACH_AVOID
    V0 = res.p_min if reach else 1.0 - res.p_min   # phase 1 vector (reach: V0)
    bad = 0
    for c in free:
        vals = [SY._row_value(ocsr, c * U + j, V0, 0.0 if reach else 1.0,
                              0.0 if reach else 1.0, not reach) for j in range(U)]
        best = max(vals) if reach else min(vals)
        if abs(vals[gpu_policy[c]] - best) > 1e-7:
            bad += 1
    return bad


@pytest.mark.parametrize("spec", [SY.REACH_AVOID, SY.SAFETY])
def test_robot_synthesis_matches_oracle(spec):
    prob, labels = robot(9)
    ocsr = oracle.build_rows(prob)
    ref = SY.interval_iteration(ocsr, labels, prob.n_inputs, spec, eps=1e-9, max_iters=5000)
    csr = impact.build(prob, "fp64")
    got = impact.synthesize(csr, prob, labels, spec=spec, eps=1e-9, max_iters=5000)
    p_min, p_max = got.p_min.cpu().numpy(), got.p_max.cpu().numpy()
    pol = got.policy.cpu().numpy()
    assert np.max(np.abs(p_min - ref.p_min)) < TOL
    assert np.all(p_min <= p_max + 1e-9)
    assert abs(got.iterations[0] - ref.iterations[0]) <= 1
    # tied inputs may be picked differently: every GPU choice is optimal, and
    # the oracle's phase 2 under the GPU's policy gives the GPU's P_max on
    # every cell
    assert optimal_margin_ok(ocsr, ref, labels, prob.n_inputs, pol, spec) == 0
    ref2 = SY.interval_iteration(ocsr, labels, prob.n_inputs, spec, eps=1e-9, max_iters=5000,
                                 phase2_policy=pol)
    assert np.max(np.abs(p_max - ref2.p_max)) < TOL
    assert np.max(np.abs(ref2.p_min - ref.p_min)) == 0.0   # phase 1 is untouched


@pytest.mark.parametrize("spec", [SY.REACH_AVOID, SY.SAFETY])
def test_long_rows_match_oracle(spec):
    """Dense 23^2 robot: every row has 529 targets plus the sink and the
    truncated mass, past the 512 successors the warp keeps in registers, so
    the row LPs take the branch that re-reads the successors on every
    bisection pass. A finite horizon (Remark 5.1) keeps the oracle short."""
    prob, labels = robot(23)
    ocsr = oracle.build_rows(prob)
    assert np.min(np.diff(ocsr.row_ptr)) + 2 > 512
    K = 4
    csr = impact.build(prob, "fp64")
    got = impact.synthesize(csr, prob, labels, spec=spec, horizon=K)
    p_min, p_max = got.p_min.cpu().numpy(), got.p_max.cpu().numpy()
    pol = got.policy.cpu().numpy()
    # phase 1 does not depend on phase2_policy; phase 2 runs under the GPU's
    # (optimal, tie-broken) choice
    ref = SY.interval_iteration(ocsr, labels, prob.n_inputs, spec, horizon=K,
                                phase2_policy=pol)
    assert np.max(np.abs(p_min - ref.p_min)) < TOL
    assert np.max(np.abs(p_max - ref.p_max)) < TOL
    assert np.max(p_max - p_min) > 1e-3   # the two bounds differ: both are checked


def test_fp32_abstraction_gives_a_lower_pessimistic_bound():
    prob, labels = robot(11)
    c64 = impact.build(prob, "fp64")
    c32 = impact.build(prob, "fp32")
    g64 = impact.synthesize(c64, prob, labels, eps=1e-8)
    g32 = impact.synthesize(c32, prob, labels, eps=1e-8)
    # wider FP32 intervals: the pessimistic (min LP) optimum can only drop
    assert np.all(g32.p_min.cpu().numpy() <= g64.p_min.cpu().numpy() + 1e-7)
    assert np.max(np.abs(g32.p_min.cpu().numpy() - g64.p_min.cpu().numpy())) < 1e-4


def test_gamblers_ruin_closed_form_on_device():
    """A hand-made degenerate IMDP (lo == up) uploaded as a CSR."""
    N, p = 10, 0.45
    rows_col, rows_w = [], []
    for i in range(N + 1):
        if 0 < i < N:
            rows_col.append([i - 1, i + 1])
            rows_w.append([1 - p, p])
        else:
            rows_col.append([i])
            rows_w.append([1.0])
    ptr = np.concatenate([[0], np.cumsum([len(c) for c in rows_col])]).astype(np.int64)
    col = np.concatenate(rows_col).astype(np.int32)
    w = np.concatenate(rows_w).astype(np.float64)
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(a).to(dev)
    zero = torch.zeros(N + 1, dtype=torch.float64, device=dev)
    csr = impact.CSR("fp64", t(ptr), t(col), t(w), t(w), zero, zero.clone(), zero.clone(),
                     torch.zeros(N + 1, dtype=torch.int32, device=dev))

    class Chain:
        total_cells = N + 1
        n_inputs = 1

    labels = np.zeros(N + 1, np.uint8)
    labels[0], labels[N] = 2, 1
    got = impact.synthesize(csr, Chain, labels, eps=1e-13, max_iters=200000)
    r = (1 - p) / p
    i = np.arange(N + 1)
    exact = (1 - r ** i) / (1 - r ** N)
    assert np.max(np.abs(got.p_min.cpu().numpy() - exact)) < 1e-10
    assert np.max(np.abs(got.p_max.cpu().numpy() - exact)) < 1e-10
