"""Host-side input generators for the synthesis options (no GPU): disturbance
points as extra inputs, the autonomous (IMC) build, region labels."""

import numpy as np
import pytest

import oracle
from paper_2401_03555_gb300 import workloads as W


def test_disturbance_rows_follow_input_then_disturbance():
    base = W.robot_2d(cells_per_dim=5)
    wp = np.array([[-0.3, 0.0], [0.0, 0.2], [0.3, -0.1]])
    prob = W.with_disturbances(base, np.eye(2), wp)
    U = base.inputs.shape[0]
    assert prob.n_inputs == U * 3 and prob.B.shape == (2, 4)
    # row (cell, j, k) of the disturbed build = the base system's row for
    # input j shifted by w_k: its image is the base image plus w_k
    for cell, j, k in ((0, 0, 0), (7, 4, 2), (24, 8, 1)):
        r = (cell * U + j) * 3 + k
        lo, hi = oracle.image(prob, r)
        blo, bhi = oracle.image(base, cell * U + j)
        assert np.allclose(lo, blo + wp[k], atol=1e-12) and np.allclose(hi, bhi + wp[k], atol=1e-12)


def test_imc_has_one_empty_input():
    base = W.room_5d(cells_per_dim=3)
    imc = W.without_inputs(base)
    assert imc.n_inputs == 1 and imc.inputs.shape == (1, 0) and imc.B is None
    lo, hi = oracle.image(imc, 5)
    assert np.all(lo <= hi)
    with pytest.raises(ValueError):
        W.without_inputs(W.unicycle_3d(nx=3, ny=3, nth=3))
    dist = W.with_disturbances(imc, np.eye(5)[:, :1], [[0.1], [-0.1]])
    assert dist.n_inputs == 2 and dist.B.shape == (5, 1)


def test_region_labels_avoid_wins_and_centres_decide():
    prob = W.robot_2d(cells_per_dim=4)             # cells of width 5, centres at -7.5 .. 7.5
    lab = W.region_labels(prob, target=([-8, -8], [8, 8]), avoid=([2, 2], [8, 8])).reshape(4, 4)
    assert np.all(lab[2:, 2:] == 2) and lab[0, 0] == 1 and lab[1, 3] == 1
    assert W.region_labels(prob, target=([-2.4, -2.4], [2.4, 2.4])).sum() == 0   # no centre inside
    lab = W.region_labels(prob, target=([-2.6, -2.6], [2.6, 2.6])).reshape(4, 4)
    assert lab.sum() == 4 and np.all(lab[1:3, 1:3] == 1)
