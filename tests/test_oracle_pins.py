"""The CPU oracle against the mathematics and the paper (no GPU needed)."""

import os

import numpy as np
import pytest

import oracle
import oracle_pins as P
from paper_2401_03555_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


def test_phi_matches_high_precision_cdf(orc):
    worst = P.pin_phi_library(orc)
    assert worst < 1e-15  # absolute


def test_edges_and_axis_telescoping(orc):
    P.pin_edges_telescoping(orc)


def test_one_dimensional_closed_form(orc):
    P.pin_closed_form_1d(orc)


def test_separable_2d_equals_exact_min_max(orc):
    P.pin_bruteforce_2d(orc)


@pytest.mark.parametrize("case", range(5))
def test_monte_carlo_containment(orc, case):
    prob, rows = P.coupled_cases()[case]
    P.pin_mc_containment(orc, prob, rows)


def test_unicycle_interval_image(orc):
    P.pin_unicycle_image(orc)


@pytest.mark.parametrize("which", ["bas4d", "unicycle", "room5d"])
def test_noise_sampling(orc, which):
    prob = {"bas4d": W.bas_4d(eta_scale=2.0), "unicycle": W.unicycle_3d(nx=8, ny=8, nth=6),
            "room5d": W.room_5d(cells_per_dim=5)}[which]
    row = W.sample_rows(prob, 1, seed=9, include_boundary=False)[0]
    P.pin_noise_sampling(orc, prob, row)


@pytest.mark.parametrize("case", range(5))
def test_invariants_coupled(orc, case):
    prob, rows = P.coupled_cases()[case]
    P.pin_invariants(orc, prob, rows)


def test_invariants_robot_dense(orc):
    prob = W.robot_2d(cells_per_dim=9)
    P.pin_invariants(orc, prob, np.arange(prob.rows))


def test_degenerate_point_images(orc):
    P.pin_degenerate(orc)


@pytest.mark.parametrize("case", [0, 2, 3])
def test_sum_of_uppers_is_product_of_axis_sums(orc, case):
    prob, rows = P.coupled_cases()[case]
    P.pin_separable_sum(orc, prob, rows)


def test_region_labels(orc):
    P.pin_region_labels(orc)


def test_region_vectors_contain_the_exact_probabilities(orc):
    P.pin_region_containment(orc)


def test_region_box_is_exact_for_separable_dynamics(orc):
    P.pin_region_box_exact_separable(orc)


def test_region_vectors_reduce_to_cells_and_sink(orc):
    P.pin_region_reductions(orc)


def test_mc_cell_of(orc):
    P.pin_mc_cell_of(orc)


def test_mc_point_images_match_closed_forms_and_library_cdf(orc):
    P.pin_mc_point_images(orc)


def test_mc_box_images_match_closed_forms(orc):
    P.pin_mc_box_images(orc)


def test_mc_counts_equal_brute_force(orc):
    P.pin_mc_counting(orc)


def test_interval_markov_chain_is_the_zero_input_row(orc):
    """Without inputs (an IMC, Sec. 6.4) the robot's rows equal its rows for
    the input point u = 0."""
    prob = W.robot_2d(cells_per_dim=9)
    imc = W.without_inputs(prob)
    j0 = int(np.nonzero(np.all(prob.inputs == 0.0, axis=1))[0][0])
    cells = np.arange(0, 81, 7)
    a = orc.build_rows(imc, cells)
    b = orc.build_rows(prob, cells * prob.n_inputs + j0)
    for x, y in ((a.row_ptr, b.row_ptr), (a.col, b.col), (a.lo, b.lo), (a.up, b.up),
                 (a.sink_lo, b.sink_lo), (a.sink_up, b.sink_up), (a.trunc, b.trunc)):
        assert np.array_equal(x, y)


def test_overlapping_region_boxes_are_refused(orc):
    prob = W.robot_2d(cells_per_dim=9)
    with pytest.raises(ValueError):
        orc.region_vectors(prob, [0], [([0, 0], [5, 5])], [([4, 4], [8, 8])], "box")


def test_ties_with_cutoff_are_kept(orc):
    P.pin_tie_kept(orc)


def _parse_golden():
    rows = []
    with open(os.path.join(GOLDEN, "table1_grid_counts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([x.strip() for x in line.split("|")])
    return rows


@pytest.mark.parametrize("entry", _parse_golden(), ids=lambda e: e[0])
def test_table1_grid_counts(entry):
    name, slb, sub, seta, ilb, iub, ieta, wpts, nx, nu, nrows = entry
    vec = lambda s: [float(v) for v in s.split(",")]
    lo, hi, cells = W.grid_from_points(vec(slb), vec(sub), vec(seta))
    assert int(np.prod(cells.astype(np.int64))) == int(nx)
    n_inputs = 1 if ilb == "-" else len(W.input_points(vec(ilb), vec(iub), vec(ieta)))
    assert n_inputs == int(nu)
    prob = W.Problem(name=name, kind=W.AFFINE, lo=lo, hi=hi, cells=cells,
                     inputs=np.zeros((n_inputs, 1)), sigma=np.ones(len(lo)), cutoff=0.0)
    # rows of the transition matrices: |X| x |U| x |W| (Def. 3.1 / Table 1)
    assert prob.rows * int(wpts) == int(nrows)
    assert np.allclose(hi - lo, cells * np.array(vec(seta)))


def eight_dim_case():
    """The largest dimension the boundary accepts: a seeded 8-D linear system
    on 3^8 cells (coupled A, two or three input dimensions)."""
    prob = W.random_linear(2, min_cells=5000, max_cells=7000, dims=(8,))
    assert prob.n == 8
    return prob, W.sample_rows(prob, 3, seed=12, include_boundary=False)


def test_eight_dimensions_contain_sampled_probabilities(orc):
    prob, rows = eight_dim_case()
    P.pin_mc_containment(orc, prob, rows, samples=24)


def test_eight_dimensions_invariants_and_axis_sums(orc):
    prob, rows = eight_dim_case()
    P.pin_invariants(orc, prob, rows)
    P.pin_separable_sum(orc, prob, rows)
