"""Seeded synthetic workloads (problem descriptions only).

This module builds the inputs that both the CUDA path and the CPU oracle
consume: dynamics matrices, grids, input points, noise scales and cutoffs. It
holds none of the method's arithmetic (no images, no Gaussian factors, no
bounds) and imports nothing else from the package, so tests can load it on a
machine without a GPU.

The shapes follow the paper's case studies (Sec. 8): the 2-D robot, the 3-D
vehicle (here a unicycle), the 5-D room-temperature model and the 7-D
building model, plus a seeded family of random linear systems.
"""

from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

AFFINE, UNICYCLE, IMAGES = 0, 1, 2


@dataclass
class Problem:
    """One abstraction build: x+ = f(x,u) + w, w ~ N(0, diag(sigma^2)).

    kind     AFFINE (f = A x + B u + c), UNICYCLE (inputs (v, om)) or IMAGES
             (caller-supplied interval images per row).
    lo, hi   domain corners; dimension d is cut into ``cells[d]`` equal cells.
    inputs   input points, shape (n_inputs, m).
    images   IMAGES only: (rows, n, 2) array of (m_lo, m_hi).
    cutoff   keep a target iff its upper bound >= cutoff (0 = dense).
    """

    name: str
    kind: int
    lo: np.ndarray
    hi: np.ndarray
    cells: np.ndarray
    inputs: np.ndarray
    sigma: np.ndarray
    cutoff: float
    A: Optional[np.ndarray] = None
    B: Optional[np.ndarray] = None
    c: Optional[np.ndarray] = None
    images: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(len(self.lo))

    @property
    def n_inputs(self) -> int:
        return int(np.asarray(self.inputs).shape[0])

    @property
    def total_cells(self) -> int:
        return int(np.prod(np.asarray(self.cells, dtype=np.int64)))

    @property
    def rows(self) -> int:
        return self.total_cells * self.n_inputs


def _arr(x, dtype=np.float64):
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


def grid_from_points(lb, ub, eta):
    """The paper's grid convention (Sec. 4.2, space setters): representative
    points lb, lb+eta, ..., ub in each dimension, each the centre of its cell.
    Returns (lo, hi, cells) with the domain widened by eta/2 on each side."""
    lb, ub, eta = _arr(lb), _arr(ub), _arr(eta)
    cells = np.rint((ub - lb) / eta).astype(np.int64) + 1
    return lb - eta / 2, ub + eta / 2, cells.astype(np.int32)


def input_points(lb, ub, eta):
    """All input points lb:eta:ub (inclusive) per dimension, C-order product."""
    lb, ub, eta = _arr(lb), _arr(ub), _arr(eta)
    axes = [lb[k] + eta[k] * np.arange(int(np.rint((ub[k] - lb[k]) / eta[k])) + 1)
            for k in range(len(lb))]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.reshape(-1) for g in mesh], axis=1)


# --------------------------------------------------------------------------
# The named workloads
# --------------------------------------------------------------------------

def robot_2d(cells_per_dim: int = 21) -> Problem:
    """2-D robot, x+ = x + u + w on [-10,10]^2, inputs {-1,0,1}^2, sigma 0.75,
    dense (cutoff 0). Shape of the paper's 2-D robot case study (Sec. 8.1)."""
    return Problem(
        name=f"robot2d-{cells_per_dim}x{cells_per_dim}",
        kind=AFFINE,
        lo=_arr([-10.0, -10.0]), hi=_arr([10.0, 10.0]),
        cells=_arr([cells_per_dim, cells_per_dim], np.int32),
        inputs=input_points([-1, -1], [1, 1], [1, 1]),
        sigma=_arr([0.75, 0.75]), cutoff=0.0,
        A=np.eye(2), B=np.eye(2), c=np.zeros(2))


def unicycle_3d(nx: int = 51, ny: int = 51, nth: int = 25, cutoff: float = 1e-8) -> Problem:
    """3-D unicycle on [-5,5]^2 x [-pi,pi]: x+ = x + v cos th, y+ = y + v sin th,
    th+ = th + om; v in {0.25,...,1}, om in {-0.4,...,0.4}; sigma (0.3,0.3,0.2).
    Shaped like the paper's 3-D vehicle (Sec. 8.2)."""
    v = np.array([0.25, 0.5, 0.75, 1.0])
    om = np.array([-0.4, -0.2, 0.0, 0.2, 0.4])
    V, O = np.meshgrid(v, om, indexing="ij")
    return Problem(
        name=f"unicycle3d-{nx}x{ny}x{nth}",
        kind=UNICYCLE,
        lo=_arr([-5.0, -5.0, -np.pi]), hi=_arr([5.0, 5.0, np.pi]),
        cells=_arr([nx, ny, nth], np.int32),
        inputs=np.stack([V.reshape(-1), O.reshape(-1)], axis=1),
        sigma=_arr([0.3, 0.3, 0.2]), cutoff=cutoff)


def room_5d_matrices():
    """A = 0.85 I + 0.03 on ring neighbours (i+-1 mod 5); heater u1 drives
    rooms 1,3,5 and u2 rooms 2,4 with gain 0.5; offset 1.8 (Sec. 8.3 shape)."""
    n = 5
    A = 0.85 * np.eye(n)
    for i in range(n):
        A[i, (i + 1) % n] += 0.03
        A[i, (i - 1) % n] += 0.03
    B = np.zeros((n, 2))
    B[[0, 2, 4], 0] = 0.5
    B[[1, 3], 1] = 0.5
    c = np.full(n, 1.8)
    return A, B, c


def room_5d(cells_per_dim: int = 11, cutoff: float = 1e-8, lo: float = 17.0,
            hi: float = 23.0) -> Problem:
    """5-D room temperature, state [17,23]^5 on an 11^5 grid, inputs
    {0,0.5,1}^2, sigma 0.2 per dim, cutoff 1e-8."""
    A, B, c = room_5d_matrices()
    return Problem(
        name=f"room5d-{cells_per_dim}^5",
        kind=AFFINE,
        lo=np.full(5, lo), hi=np.full(5, hi),
        cells=np.full(5, cells_per_dim, dtype=np.int32),
        inputs=input_points([0, 0], [1, 1], [0.5, 0.5]),
        sigma=np.full(5, 0.2), cutoff=cutoff, A=A, B=B, c=c)


def building_7d(cells_per_dim: int = 6, cutoff: float = 1e-8) -> Problem:
    """7-D building model: A = 0.9 I + 0.02 chain couplings (no wrap),
    u1 heats room 1 and u2 room 2 with gain 0.1, inputs {0,1}^2, sigma 0.15,
    domain [-3,3]^7 (cell width 1 at 6 cells per dim). Shaped like the
    paper's 7-D building automation benchmark (Sec. 8.4)."""
    n = 7
    A = 0.9 * np.eye(n)
    for i in range(n - 1):
        A[i, i + 1] = 0.02
        A[i + 1, i] = 0.02
    B = np.zeros((n, 2))
    B[0, 0] = 0.1
    B[1, 1] = 0.1
    return Problem(
        name=f"building7d-{cells_per_dim}^7",
        kind=AFFINE,
        lo=np.full(n, -3.0), hi=np.full(n, 3.0),
        cells=np.full(n, cells_per_dim, dtype=np.int32),
        inputs=input_points([0, 0], [1, 1], [1, 1]),
        sigma=np.full(n, 0.15), cutoff=cutoff, A=A, B=B, c=np.zeros(n))


def random_linear(seed: int, min_cells: float = 1e3, max_cells: float = 1e5,
                  dims=(2, 3, 4, 5), cutoff: float = 1e-8) -> Problem:
    """One seeded random linear system x+ = A x + B u + w on [-1,1]^n:
    A = 0.9 Q D Q^T (D uniform in [0.5,1], Q orthogonal from the QR of a
    Gaussian matrix with R's diagonal made positive), B with N(0, 0.3^2)
    entries, total cells log-uniform in [min_cells, max_cells] split evenly
    over the dimensions, m in {2,3} input dimensions with 2 or 3 points each
    over [-1,1], sigma log-uniform in [0.1, 1] x cell width."""
    rng = np.random.default_rng(seed)
    n = int(rng.choice(np.asarray(dims)))
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))[None, :]
    D = rng.uniform(0.5, 1.0, size=n)
    A = 0.9 * (Q * D[None, :]) @ Q.T
    m = int(rng.choice([2, 3]))
    B = rng.normal(0.0, 0.3, size=(n, m))
    total = float(np.exp(rng.uniform(np.log(min_cells), np.log(max_cells))))
    N = max(2, int(round(total ** (1.0 / n))))
    pts = int(rng.choice([2, 3]))
    axis = np.linspace(-1.0, 1.0, pts)
    mesh = np.meshgrid(*([axis] * m), indexing="ij")
    inputs = np.stack([g.reshape(-1) for g in mesh], axis=1)
    width = 2.0 / N
    sigma = width * np.exp(rng.uniform(np.log(0.1), np.log(1.0), size=n))
    return Problem(
        name=f"linear-seed{seed}-{n}d-{N}^{n}",
        kind=AFFINE,
        lo=np.full(n, -1.0), hi=np.full(n, 1.0),
        cells=np.full(n, N, dtype=np.int32),
        inputs=inputs, sigma=sigma, cutoff=cutoff,
        A=A, B=B, c=np.zeros(n), meta={"seed": seed})


def batched_family(count: int = 256, first_seed: int = 0, **kw) -> List[Problem]:
    """The batched workload: ``count`` seeded random linear systems."""
    return [random_linear(first_seed + s, **kw) for s in range(count)]


def without_inputs(prob: Problem) -> Problem:
    """The autonomous system f(x) = A x + c of an affine `prob`: one input
    point of dimension 0, so the build is an interval Markov chain (IMC)."""
    if prob.kind != AFFINE:
        raise ValueError("only affine systems drop their inputs here")
    return replace(prob, name=prob.name + "-imc", inputs=np.zeros((1, 0)), B=None)


def with_disturbances(prob: Problem, Bw, w_points) -> Problem:
    """The affine `prob` with a disturbance input: f(x, u, w) = A x + B u +
    Bw w + c. The build's input points become the (u, w) pairs, w fastest,
    so row r = (cell * n_u + j) * n_w + k."""
    if prob.kind != AFFINE:
        raise ValueError("disturbances are added to affine systems")
    U = np.asarray(prob.inputs, np.float64)
    if U.ndim == 1:
        U = U.reshape(-1, 1)
    Wp = np.asarray(w_points, np.float64)
    if Wp.ndim == 1:
        Wp = Wp.reshape(-1, 1)
    Bw = np.asarray(Bw, np.float64).reshape(prob.n, Wp.shape[1])
    pts = np.array([np.concatenate([u, w]) for u in U for w in Wp])
    B = Bw if U.shape[1] == 0 else np.concatenate([np.asarray(prob.B, np.float64), Bw], axis=1)
    return replace(prob, name=prob.name + f"+w{Wp.shape[0]}", inputs=pts, B=B)


def with_images(prob: Problem, images: np.ndarray) -> Problem:
    """Same grid/inputs/noise, but with caller-supplied interval images."""
    return replace(prob, kind=IMAGES, images=_arr(images), name=prob.name + "+images")


def with_cells(prob: Problem, cells) -> Problem:
    """Same system on a different grid (same domain)."""
    cells = _arr(cells, np.int32)
    return replace(prob, cells=cells, name=f"{prob.name}@{'x'.join(map(str, cells))}")


def sample_rows(prob: Problem, count: int, seed: int = 0, include_boundary: bool = True):
    """Seeded random row ids plus (optionally) the first/last rows and the rows
    of the cells at the domain's corners, sorted and unique."""
    rng = np.random.default_rng(seed)
    R = prob.rows
    rows = set(rng.integers(0, R, size=min(count, R)).tolist())
    if include_boundary:
        rows.update([0, R - 1])
        cells = np.asarray(prob.cells, dtype=np.int64)
        n = len(cells)
        for corner in range(1 << n):
            idx = [(cells[d] - 1) if (corner >> d) & 1 else 0 for d in range(n)]
            cell = int(np.ravel_multi_index(idx, cells))
            rows.add(cell * prob.n_inputs + int(rng.integers(0, prob.n_inputs)))
    return np.array(sorted(rows), dtype=np.int64)


def bas_4d(eta_scale: float = 1.0) -> Problem:
    """The paper's 4-D building automation system (Sec. 8.4): the printed A, B,
    offset and diagonal covariance (variances, so sigma = sqrt), state
    [19,21]^2 x [30,36]^2 with eta (0.5,0.5,1,1) scaled by ``eta_scale``,
    input [17,20] with eta 1 (points 17,18,19,20)."""
    A = np.array([[0.6682, 0.0, 0.02632, 0.0],
                  [0.0, 0.683, 0.0, 0.02096],
                  [1.0005, 0.0, -0.000499, 0.0],
                  [0.0, 0.8004, 0.0, 0.1996]])
    B = np.array([[0.1320], [0.1402], [0.0], [0.0]])
    c = np.array([3.4378, 2.9272, 13.0207, 10.4166])
    var = np.array([12.9199, 12.9199, 2.5826, 3.2279])
    lo, hi, cells = grid_from_points([19, 19, 30, 30], [21, 21, 36, 36],
                                     np.array([0.5, 0.5, 1.0, 1.0]) * eta_scale)
    return Problem(
        name=f"bas4d-eta{eta_scale}",
        kind=AFFINE, lo=lo, hi=hi, cells=cells,
        inputs=input_points([17], [20], [1]),
        sigma=np.sqrt(var), cutoff=0.0, A=A, B=B, c=c)


def region_labels(prob: Problem, target=None, avoid=None) -> np.ndarray:
    """Per-cell labels for synthesis: 1 if the cell's centre lies in a target
    box, 2 if in an avoid box (avoid wins), else 0. Boxes are (lo, hi) pairs
    of coordinate lists; `target` / `avoid` are one box or a list of them."""
    cells = np.asarray(prob.cells, dtype=np.int64)
    lo = np.asarray(prob.lo, np.float64)
    hi = np.asarray(prob.hi, np.float64)
    h = (hi - lo) / cells
    axes = [lo[d] + (np.arange(cells[d]) + 0.5) * h[d] for d in range(len(cells))]
    mesh = np.meshgrid(*axes, indexing="ij")
    centres = np.stack([m.reshape(-1) for m in mesh], axis=1)
    labels = np.zeros(centres.shape[0], np.uint8)

    def boxes(b):
        if b is None:
            return []
        if len(b) == 2 and np.ndim(b[0]) == 1:
            return [b]
        return list(b)

    for code, spec in ((1, target), (2, avoid)):
        for blo, bhi in boxes(spec):
            inside = np.all((centres >= np.asarray(blo)) & (centres <= np.asarray(bhi)), axis=1)
            labels[inside] = code
    return labels

