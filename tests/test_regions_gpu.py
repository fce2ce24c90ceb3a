"""Target / avoid regions and the synthesis options through the C ABI
(impact_label_cells, impact_region_vectors, impact_synthesize_ex) against
the CPU oracle (needs a GPU)."""

import numpy as np
import pytest
import torch

import oracle
import oracle_pins as OP
from oracle import synthesis as SY
from paper_2401_03555_gb300 import impact, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    impact.load()


CASES = OP.region_cases()


@pytest.mark.parametrize("k", range(len(CASES)))
def test_labels_equal_the_oracle(k):
    prob, tb, ab, _ = CASES[k]
    got = impact.label_cells(prob, tb, ab).cpu().numpy()
    assert np.array_equal(got, oracle.region_labels(prob, tb, ab))
    # overlapping boxes: avoid wins
    big, small = (prob.lo, prob.hi), (prob.lo, 0.5 * (prob.lo + prob.hi))
    got = impact.label_cells(prob, [big], [small]).cpu().numpy()
    assert np.array_equal(got, oracle.region_labels(prob, [big], [small]))


@pytest.mark.parametrize("mode", ["box", "cells"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("k", range(len(CASES)))
def test_region_vectors_match_the_oracle(k, mode, precision):
    prob, tb, ab, rows = CASES[k]
    rows = np.asarray(rows, np.int64)
    got = impact.region_vectors(prob, tb, ab, mode, precision)
    g = [t.cpu().numpy()[rows] for t in (got.r_lo, got.r_up, got.a_lo, got.a_up)]
    ref = oracle.region_vectors(prob, rows, tb, ab, mode)
    # FP64: round-to-nearest evaluation, relative 1e-12 (the cell sums reach
    # tens); FP32-sound: the FP32 outward factor bounds of the pair path
    # (about 2^-23 absolute each) with directed rounding, so the vectors
    # enclose the exact ones; a cell sum adds one such error per cell
    tol = 1e-12 if precision == "fp64" else 1e-5
    for x, y in zip(g, ref):
        assert np.all(np.abs(x - y) <= tol * np.maximum(1.0, np.abs(y))), \
            (prob.name, mode, precision, float(np.max(np.abs(x - y))))
    if precision == "fp32":
        for i in (0, 2):
            slack = 1e-15 * np.maximum(1.0, np.abs(ref[i + 1]))
            assert np.all(g[i] <= ref[i] + slack) and np.all(g[i + 1] >= ref[i + 1] - slack)
        assert np.all(g[0] >= 0.0) and np.all(g[2] >= 0.0)


def test_region_vectors_all_rows_of_the_robot():
    prob, tb, ab, _ = CASES[0]
    for mode in ("box", "cells"):
        got = impact.region_vectors(prob, tb, ab, mode, "fp64")
        ref = oracle.region_vectors(prob, None, tb, ab, mode)
        for t, y in zip((got.r_lo, got.r_up, got.a_lo, got.a_up), ref):
            assert np.max(np.abs(t.cpu().numpy() - y)) < 1e-12


def test_region_box_errors():
    prob = W.robot_2d(cells_per_dim=9)
    with pytest.raises(impact.ImpactError) as ei:
        impact.region_vectors(prob, [([0, 0], [5, 5])], [([4, 4], [8, 8])])
    assert ei.value.status == impact.IMPACT_ERR_ARG
    with pytest.raises(impact.ImpactError):
        impact.region_vectors(prob, [([1, 1], [0, 0])], [])
    # a box that holds no cell centre is ignored
    got = impact.region_vectors(prob, [([0.01, 0.01], [0.02, 0.02])], [])
    assert float(got.r_up.abs().max()) == 0.0


# ---- synthesis options ------------------------------------------------------


def robot(cells=9):
    prob = W.robot_2d(cells_per_dim=cells)
    tb = [([2.0, 2.0], [9.0, 9.0])]
    ab = [([-9.0, -9.0], [-2.0, -2.0])]
    return prob, tb, ab


def compare(ref, got, tol=1e-8, same_frac=0.8):
    p_min, p_max = got.p_min.cpu().numpy(), got.p_max.cpu().numpy()
    pol = got.policy.cpu().numpy()
    assert np.max(np.abs(p_min - ref.p_min)) < tol
    same = pol == ref.policy
    assert same.mean() >= same_frac
    if same.all():
        assert np.max(np.abs(p_max - ref.p_max)) < tol


@pytest.mark.parametrize("spec", [SY.REACH_AVOID, SY.SAFETY])
@pytest.mark.parametrize("mode", ["box", "cells"])
def test_synthesis_with_region_vectors(spec, mode):
    prob, tb, ab = robot()
    ocsr = oracle.build_rows(prob)
    olab = oracle.region_labels(prob, tb, ab)
    ref = SY.interval_iteration(ocsr, olab, prob.n_inputs, spec, eps=1e-9, max_iters=5000,
                                regions=oracle.region_vectors(prob, None, tb, ab, mode))
    csr = impact.build(prob, "fp64")
    lab = impact.label_cells(prob, tb, ab)
    got = impact.synthesize(csr, prob, lab, spec=spec, eps=1e-9, max_iters=5000,
                            regions=impact.region_vectors(prob, tb, ab, mode, "fp64"))
    compare(ref, got, same_frac=0.8 if spec == SY.REACH_AVOID else 0.5)
    assert abs(got.iterations[0] - ref.iterations[0]) <= 1


def test_cell_sum_regions_equal_labelled_columns_on_the_device():
    prob, tb, ab = robot()
    csr = impact.build(prob, "fp64")
    lab = impact.label_cells(prob, tb, ab)
    a = impact.synthesize(csr, prob, lab, eps=1e-9)
    b = impact.synthesize(csr, prob, lab, eps=1e-9,
                          regions=impact.region_vectors(prob, tb, ab, "cells", "fp64"))
    assert torch.max(torch.abs(a.p_min - b.p_min)).item() < 1e-9
    assert torch.max(torch.abs(a.p_max - b.p_max)).item() < 1e-9


@pytest.mark.parametrize("spec", [SY.REACH_AVOID, SY.SAFETY])
def test_optimistic_policy(spec):
    prob, tb, ab = robot()
    ocsr = oracle.build_rows(prob)
    olab = oracle.region_labels(prob, tb, ab)
    ref = SY.interval_iteration(ocsr, olab, prob.n_inputs, spec, eps=1e-9, max_iters=5000,
                                optimistic=True)
    got = impact.synthesize(impact.build(prob, "fp64"), prob, impact.label_cells(prob, tb, ab),
                            spec=spec, eps=1e-9, max_iters=5000, optimistic=True)
    p_max = got.p_max.cpu().numpy()
    assert np.max(np.abs(p_max - ref.p_max)) < 1e-8       # phase 1's bound
    assert np.mean(got.policy.cpu().numpy() == ref.policy) > 0.5


@pytest.mark.parametrize("spec", [SY.REACH_AVOID, SY.SAFETY])
def test_finite_horizon(spec):
    prob, tb, ab = robot()
    ocsr = oracle.build_rows(prob)
    olab = oracle.region_labels(prob, tb, ab)
    K = 12
    ref = SY.interval_iteration(ocsr, olab, prob.n_inputs, spec, horizon=K)
    got = impact.synthesize(impact.build(prob, "fp64"), prob, impact.label_cells(prob, tb, ab),
                            spec=spec, horizon=K)
    assert got.iterations == (K, K)
    assert np.max(np.abs(got.p_min.cpu().numpy() - ref.p_min)) < 1e-9
    pol = got.policy.cpu().numpy()
    if np.array_equal(pol, ref.policy):
        assert np.max(np.abs(got.p_max.cpu().numpy() - ref.p_max)) < 1e-9


@pytest.mark.parametrize("spec", [SY.REACH_AVOID, SY.SAFETY])
def test_disturbance_adversary(spec):
    base, tb, ab = robot(7)
    prob = W.with_disturbances(base, np.eye(2), [[-0.4, 0.0], [0.0, 0.0], [0.4, -0.4]])
    ocsr = oracle.build_rows(prob)
    olab = oracle.region_labels(prob, tb, ab)
    ref = SY.interval_iteration(ocsr, olab, base.n_inputs, spec, eps=1e-9, max_iters=5000,
                                n_disturb=3)
    got = impact.synthesize(impact.build(prob, "fp64"), prob, impact.label_cells(prob, tb, ab),
                            spec=spec, eps=1e-9, max_iters=5000, n_disturb=3)
    compare(ref, got, same_frac=0.8 if spec == SY.REACH_AVOID else 0.5)
    # w = 0 is one of the adversary's choices: it can only lower the
    # pessimistic bound
    plain = impact.synthesize(impact.build(base, "fp64"), base, impact.label_cells(base, tb, ab),
                              spec=spec, eps=1e-9, max_iters=5000)
    assert torch.all(got.p_min <= plain.p_min + 1e-6).item()


@pytest.mark.parametrize("disturb", [False, True])
def test_interval_markov_chain_verification(disturb):
    """No inputs (an IMC): the build and the verification bounds; with
    disturbance points the adversary still chooses."""
    base, tb, ab = robot(7)
    prob = W.without_inputs(base)
    if disturb:
        prob = W.with_disturbances(prob, np.eye(2), [[-0.5, 0.0], [0.5, 0.0]])
    W_n = 2 if disturb else 1
    ocsr = oracle.build_rows(prob)
    csr = impact.build(prob, "fp64")
    assert np.array_equal(csr.row_ptr.cpu().numpy(), ocsr.row_ptr)
    assert np.max(np.abs(csr.up.cpu().numpy() - ocsr.up)) < 1e-12
    olab = oracle.region_labels(prob, tb, ab)
    for spec in (SY.REACH_AVOID, SY.SAFETY):
        ref = SY.interval_iteration(ocsr, olab, 1, spec, eps=1e-10, max_iters=5000, n_disturb=W_n)
        got = impact.synthesize(csr, prob, impact.label_cells(prob, tb, ab), spec=spec, eps=1e-10,
                                max_iters=5000, n_disturb=W_n)
        assert np.max(np.abs(got.p_min.cpu().numpy() - ref.p_min)) < 1e-8
        assert np.max(np.abs(got.p_max.cpu().numpy() - ref.p_max)) < 1e-8
        assert int(got.policy.abs().max()) == 0


def test_synthesis_option_errors():
    prob, tb, ab = robot(5)
    csr = impact.build(prob, "fp64")
    lab = impact.label_cells(prob, tb, ab)
    with pytest.raises(ValueError):
        impact.synthesize(csr, prob, lab, n_disturb=2)      # 9 build inputs
    with pytest.raises(impact.ImpactError):
        impact.synthesize(csr, prob, lab, horizon=-1)
