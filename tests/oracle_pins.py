"""Pins that tie the CPU oracle to something other than itself.

Each ``pin_*`` function takes an oracle instance (``oracle.Oracle``) and raises
AssertionError when the oracle disagrees with the mathematics or the paper:

  pin_phi_library       the Gaussian factor vs a 60-digit mpmath normal CDF
  pin_edges_telescoping grid edges, and sum over an axis == mass of the axis
  pin_closed_form_1d    1-D shift system: covering target == erf(h/(2 sqrt2 s)),
                        lo/up == exact min/max over the cell found numerically
  pin_bruteforce_2d     separable 2-D: lo at the cell corners, up == product of
                        numerically maximised 1-D factors (the relaxation is
                        exact there, Def. 3.1)
  pin_mc_containment    coupled / nonlinear systems: P(t|x) and P(out|x) of
                        random points x of the cell lie inside the bounds, and
                        f(x) inside the interval image
  pin_noise_sampling    simulating x+ = f(x,u) + w and binning lands inside
                        [lo, up] (and the sink bounds) within 5 binomial sigma
  pin_invariants        0 <= lo <= up <= 1, row sums (Def. 3.1), cutoff rule,
                        ascending columns, trunc == dropped mass
  pin_degenerate        point images: lo == up bit for bit, and the row's mass
                        (kept + truncated + sink) sums to 1
  pin_separable_sum     sum of all up == product of the per-dim maxima sums
  pin_tie_kept          an up exactly equal to the cutoff is kept

None of them re-evaluates the oracle's own formulas: they use library CDFs
(scipy / mpmath), numerical optimisation, sampling and identities.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.optimize import minimize_scalar
from scipy.special import ndtr

from paper_2401_03555_gb300 import workloads as W

# --------------------------------------------------------------------------
# helpers written from the definitions (Def. 2.2: T(A|x,u) = P(f(x,u)+w in A))
# --------------------------------------------------------------------------


def grid_edges(prob, d):
    """Edges lo + i*h (last = hi), computed here independently of the oracle."""
    N = int(prob.cells[d])
    e = prob.lo[d] + np.arange(N + 1) * ((prob.hi[d] - prob.lo[d]) / N)
    e[-1] = prob.hi[d]
    return e


def cell_box(prob, cell):
    idx = np.unravel_index(int(cell), tuple(int(c) for c in prob.cells))
    lo = np.array([grid_edges(prob, d)[idx[d]] for d in range(prob.n)])
    hi = np.array([grid_edges(prob, d)[idx[d] + 1] for d in range(prob.n)])
    return lo, hi


def dynamics(prob, x, u):
    """f(x, u) for points x of shape (k, n)."""
    x = np.atleast_2d(x)
    if prob.kind == W.AFFINE:
        off = (prob.B @ u if prob.B is not None and len(u) else 0.0) + (
            prob.c if prob.c is not None else 0.0)
        return x @ prob.A.T + off
    if prob.kind == W.UNICYCLE:
        v, om = u
        return np.stack([x[:, 0] + v * np.cos(x[:, 2]), x[:, 1] + v * np.sin(x[:, 2]),
                         x[:, 2] + om], axis=1)
    raise ValueError("no dynamics for caller images")


def interval_mass(c, e, mu, s):
    """P(mu + w in [c, e]), w ~ N(0, s^2), via the library normal CDF; the side
    with the smaller tail is used so the difference keeps its digits."""
    a = (np.asarray(c) - mu) / s
    b = (np.asarray(e) - mu) / s
    right = ndtr(-a) - ndtr(-b)
    left = ndtr(b) - ndtr(a)
    return np.where(a + b > 0, right, left)


def exact_probs(prob, mu):
    """P(t | mean mu) for every target t (C order), and P(out | mu)."""
    per_dim = []
    inside = 1.0
    for d in range(prob.n):
        e = grid_edges(prob, d)
        per_dim.append(interval_mass(e[:-1], e[1:], mu[d], prob.sigma[d]))
        inside *= float(interval_mass(prob.lo[d], prob.hi[d], mu[d], prob.sigma[d]))
    P = per_dim[0]
    for f in per_dim[1:]:
        P = np.multiply.outer(P, f)
    return P.reshape(-1), 1.0 - inside


# --------------------------------------------------------------------------
# pins
# --------------------------------------------------------------------------


def pin_phi_library(orc, trials: int = 400, seed: int = 1):
    try:
        import mpmath as mp
    except ImportError:  # pragma: no cover - mpmath ships with sympy here
        mp = None
    rng = np.random.default_rng(seed)
    worst = 0.0
    for k in range(trials):
        s = float(np.exp(rng.uniform(np.log(0.05), np.log(5.0))))
        m = float(rng.uniform(-3, 3))
        a = float(rng.uniform(-12, 12))
        w = float(np.exp(rng.uniform(np.log(1e-3), np.log(8.0))))
        c, e = m + a * s, m + (a + w) * s
        got = orc.phi_diff(c, e, m, s)
        if mp is not None:
            mp.mp.dps = 60
            ref = float(mp.ncdf((mp.mpf(e) - m) / s) - mp.ncdf((mp.mpf(c) - m) / s))
        else:
            ref = float(interval_mass(c, e, m, s))
        err = abs(got - ref)
        assert err <= 1e-300 + 2e-13 * abs(ref) + 1e-17, (c, e, m, s, got, ref)
        worst = max(worst, err)
    # symmetry and limits
    assert orc.phi_diff(-1e300, 1e300, 0.3, 1.0) == 1.0
    assert abs(orc.phi_diff(-1.0, 1.0, 0.0, 1.0) - math.erf(1 / math.sqrt(2))) < 1e-15
    assert orc.phi_diff(0.0, 1.0, 0.5, 0.7) == orc.phi_diff(0.0, 1.0, 0.5, 0.7)
    return worst


def pin_edges_telescoping(orc):
    prob = W.room_5d(cells_per_dim=7, lo=17.0, hi=23.0)
    for d in range(prob.n):
        e = orc.edges(prob, d)
        ref = grid_edges(prob, d)
        assert e[0] == prob.lo[d] and e[-1] == prob.hi[d]
        assert np.all(np.diff(e) > 0)
        assert np.allclose(e, ref, rtol=0, atol=1e-13)
        for mu in (16.0, 17.0, 18.3, 20.0, 22.99, 24.5):
            total = sum(orc.phi_diff(e[i], e[i + 1], mu, 0.2) for i in range(len(e) - 1))
            whole = float(interval_mass(prob.lo[d], prob.hi[d], mu, 0.2))
            assert abs(total - whole) < 1e-14, (d, mu, total, whole)


def one_dim_problem(n_cells=12, sigma=0.4, inputs=(-0.5, 0.3), cutoff=0.0):
    return W.Problem(name="shift1d", kind=W.AFFINE, lo=np.array([-3.0]), hi=np.array([3.0]),
                     cells=np.array([n_cells], np.int32),
                     inputs=np.array(inputs, dtype=np.float64).reshape(-1, 1),
                     sigma=np.array([sigma]), cutoff=cutoff,
                     A=np.eye(1), B=np.eye(1), c=np.zeros(1))


def _max_over_interval(fun, a, b):
    """max of a smooth unimodal fun on [a, b]: endpoints + bounded Brent."""
    best = max(fun(a), fun(b))
    if b > a:
        r = minimize_scalar(lambda x: -fun(x), bounds=(a, b), method="bounded",
                            options={"xatol": 1e-12 * max(1.0, abs(b - a))})
        best = max(best, -r.fun)
    return best


def pin_closed_form_1d(orc):
    prob = one_dim_problem()
    e = grid_edges(prob, 0)
    h = e[1] - e[0]
    s = prob.sigma[0]
    plateau = math.erf(h / (2 * math.sqrt(2) * s))
    for row in range(prob.rows):
        cell, j = divmod(row, prob.n_inputs)
        u = prob.inputs[j, 0]
        up, lo, sink_lo, sink_up = orc.row_dense(prob, row)
        xa, xb = e[cell], e[cell + 1]
        for t in range(len(e) - 1):
            c, f = e[t], e[t + 1]
            mid = 0.5 * (c + f)
            fun = lambda x: float(interval_mass(c, f, x + u, s))
            lo_ref = min(fun(xa), fun(xb))
            up_ref = _max_over_interval(fun, xa, xb)
            assert abs(lo[t] - lo_ref) < 1e-14, (row, t, lo[t], lo_ref)
            assert up[t] >= up_ref - 1e-14 and up[t] - up_ref < 1e-9, (row, t, up[t], up_ref)
            if xa + u < mid < xb + u:
                assert abs(up[t] - plateau) < 1e-14, (row, t, up[t], plateau)
        out = lambda x: 1.0 - float(interval_mass(prob.lo[0], prob.hi[0], x + u, s))
        assert abs(sink_up - max(out(xa), out(xb))) < 1e-14
        inside_max = _max_over_interval(lambda x: 1.0 - out(x), xa, xb)
        assert abs(sink_lo - (1.0 - inside_max)) < 1e-9


def pin_bruteforce_2d(orc, cells_per_dim=5, rows=None):
    prob = W.robot_2d(cells_per_dim=cells_per_dim)
    rows = range(prob.rows) if rows is None else rows
    for row in rows:
        cell, j = divmod(row, prob.n_inputs)
        u = prob.inputs[j]
        up, lo, _, _ = orc.row_dense(prob, row)
        bl, bh = cell_box(prob, cell)
        corners = np.array([[bl[0], bl[1]], [bl[0], bh[1]], [bh[0], bl[1]], [bh[0], bh[1]]])
        Pc = np.stack([exact_probs(prob, dynamics(prob, x, u)[0])[0] for x in corners])
        assert np.all(np.abs(lo - Pc.min(axis=0)) < 1e-14), row
        # separable: max of the product = product of the 1-D maxima
        maxima = []
        for d in range(2):
            e = grid_edges(prob, d)
            md = np.array([_max_over_interval(
                lambda x, c=e[t], f=e[t + 1]: float(interval_mass(c, f, x + u[d], prob.sigma[d])),
                bl[d], bh[d]) for t in range(len(e) - 1)])
            maxima.append(md)
        up_ref = np.multiply.outer(maxima[0], maxima[1]).reshape(-1)
        assert np.all(up >= up_ref - 1e-14), row
        assert np.all(up - up_ref < 1e-9), (row, float(np.max(up - up_ref)))
        # and a 17x17 sample of the cell never leaves [lo, up]
        g0 = np.linspace(bl[0], bh[0], 17)
        g1 = np.linspace(bl[1], bh[1], 17)
        for x0 in g0[::4]:
            for x1 in g1[::4]:
                P, _ = exact_probs(prob, dynamics(prob, np.array([x0, x1]), u)[0])
                assert np.all(P <= up + 1e-14) and np.all(P >= lo - 1e-14)


def pin_mc_containment(orc, prob, rows, samples=64, seed=3):
    rng = np.random.default_rng(seed)
    csr = orc.build_rows(prob, rows)
    for k, row in enumerate(rows):
        cell, j = divmod(int(row), prob.n_inputs)
        u = prob.inputs[j]
        bl, bh = cell_box(prob, cell)
        up, lo, sink_lo, sink_up = orc.row_dense(prob, row)
        m_lo, m_hi = orc.image(prob, row)
        xs = bl + (bh - bl) * rng.random((samples, prob.n))
        corners = np.array([[bh[d] if (c >> d) & 1 else bl[d] for d in range(prob.n)]
                            for c in range(1 << prob.n)])
        xs = np.concatenate([xs, corners], axis=0)
        mus = dynamics(prob, xs, u)
        tol = 1e-12 * np.maximum(1.0, np.abs(mus))
        assert np.all(mus >= m_lo - tol) and np.all(mus <= m_hi + tol), row
        if prob.kind == W.AFFINE:
            cm = dynamics(prob, corners, u)  # a linear map's range is spanned by the corners
            assert np.allclose(cm.min(axis=0), m_lo, atol=1e-12)
            assert np.allclose(cm.max(axis=0), m_hi, atol=1e-12)
        for mu in mus:
            P, out = exact_probs(prob, mu)
            assert np.all(P <= up + 1e-13), (row, float(np.max(P - up)))
            assert np.all(P >= lo - 1e-13), (row, float(np.max(lo - P)))
            assert sink_lo - 1e-13 <= out <= sink_up + 1e-13, (row, out, sink_lo, sink_up)
        # the CSR row agrees with the dense evaluation
        cols, clo, cup = csr.row(k)
        keep = np.nonzero(up >= prob.cutoff)[0]
        assert np.array_equal(cols, keep)
        assert np.array_equal(clo, lo[keep]) and np.array_equal(cup, up[keep])


def pin_unicycle_image(orc):
    # 7 heading cells: 0 and +-pi/2 fall inside cells, not on their edges
    prob = W.unicycle_3d(nx=4, ny=4, nth=7)
    th_edges = grid_edges(prob, 2)
    for cth in range(7):
        for j in (0, 7, 13, 19):
            cell = np.ravel_multi_index((1, 2, cth), (4, 4, 7))
            row = cell * prob.n_inputs + j
            m_lo, m_hi = orc.image(prob, row)
            v, om = prob.inputs[j]
            th = np.linspace(th_edges[cth], th_edges[cth + 1], 20001)
            bl, bh = cell_box(prob, cell)
            assert abs(m_lo[0] - (bl[0] + np.min(v * np.cos(th)))) < 1e-7
            assert abs(m_hi[0] - (bh[0] + np.max(v * np.cos(th)))) < 1e-7
            assert abs(m_lo[1] - (bl[1] + np.min(v * np.sin(th)))) < 1e-7
            assert abs(m_hi[1] - (bh[1] + np.max(v * np.sin(th)))) < 1e-7
            assert abs(m_lo[2] - (bl[2] + om)) < 1e-15 and abs(m_hi[2] - (bh[2] + om)) < 1e-15


def pin_noise_sampling(orc, prob, row, draws=200_000, seed=5, top=12):
    rng = np.random.default_rng(seed)
    cell, j = divmod(int(row), prob.n_inputs)
    u = prob.inputs[j]
    bl, bh = cell_box(prob, cell)
    x = bl + (bh - bl) * rng.random(prob.n)
    mu = dynamics(prob, x, u)[0]
    xp = mu + prob.sigma * rng.standard_normal((draws, prob.n))
    inside = np.all((xp >= prob.lo) & (xp < prob.hi), axis=1)
    idx = np.zeros(draws, dtype=np.int64)
    for d in range(prob.n):
        e = grid_edges(prob, d)
        k = np.clip(np.searchsorted(e, xp[:, d], side="right") - 1, 0, len(e) - 2)
        idx = idx * int(prob.cells[d]) + k
    freq = np.bincount(idx[inside], minlength=prob.total_cells) / draws
    out = 1.0 - inside.mean()
    up, lo, sink_lo, sink_up = orc.row_dense(prob, row)
    P, Pout = exact_probs(prob, mu)
    order = np.argsort(-freq)[:top]
    for t in order:
        sd = math.sqrt(max(P[t] * (1 - P[t]), 1e-12) / draws)
        assert lo[t] - 5 * sd <= freq[t] <= up[t] + 5 * sd, (t, freq[t], lo[t], up[t])
        assert abs(freq[t] - P[t]) <= 5 * sd + 1e-6, (t, freq[t], P[t])
    sd = math.sqrt(max(Pout * (1 - Pout), 1e-12) / draws)
    assert sink_lo - 5 * sd <= out <= sink_up + 5 * sd, (out, sink_lo, sink_up)
    assert abs(out - Pout) <= 5 * sd + 1e-6


def pin_invariants(orc, prob, rows):
    csr = orc.build_rows(prob, rows)
    for k, row in enumerate(rows):
        cols, lo, up = csr.row(k)
        assert np.all(lo >= 0) and np.all(up <= 1) and np.all(lo <= up), row
        assert np.all(up >= prob.cutoff), row
        assert np.all(np.diff(cols) > 0), row
        assert lo.sum() + csr.sink_lo[k] <= 1 + 1e-12, row
        assert up.sum() + csr.sink_up[k] + csr.trunc[k] >= 1 - 1e-12, row
        assert 0 <= csr.sink_lo[k] <= csr.sink_up[k] <= 1, row
        dup, dlo, _, _ = orc.row_dense(prob, row)
        dropped = dup[dup < prob.cutoff]
        assert len(cols) + len(dropped) == prob.total_cells
        assert abs(csr.trunc[k] - math.fsum(dropped.tolist())) <= 1e-15 * max(1, len(dropped))


def pin_degenerate(orc, seed=11):
    rng = np.random.default_rng(seed)
    base = W.room_5d(cells_per_dim=4)
    base = W.Problem(name="deg3d", kind=W.IMAGES, lo=base.lo[:3], hi=base.hi[:3],
                     cells=np.array([4, 5, 3], np.int32), inputs=np.zeros((2, 1)),
                     sigma=np.array([0.3, 0.5, 0.8]), cutoff=1e-8)
    pts = rng.uniform(16.0, 24.0, size=(base.rows, 3))
    images = np.stack([pts, pts], axis=2)
    prob = W.with_images(base, images)
    rows = np.arange(prob.rows)
    csr = orc.build_rows(prob, rows)
    assert np.array_equal(csr.lo, csr.up)
    assert np.array_equal(csr.sink_lo, csr.sink_up)
    for k in range(len(rows)):
        _, lo, up = csr.row(k)
        total = math.fsum(up.tolist()) + csr.trunc[k] + csr.sink_up[k]
        assert abs(total - 1.0) < 1e-12, (k, total)
        # a point image is a point x: the bounds are the exact probabilities
        P, out = exact_probs(prob, pts[k])
        cols, _, _ = csr.row(k)
        assert np.allclose(up, P[cols], rtol=0, atol=1e-14)
        assert abs(csr.sink_lo[k] - out) < 1e-13


def pin_separable_sum(orc, prob, rows):
    csr = orc.build_rows(prob, rows)
    for k, row in enumerate(rows):
        m_lo, m_hi = orc.image(prob, row)
        total = 1.0
        for d in range(prob.n):
            one = W.Problem(name="axis", kind=W.IMAGES, lo=prob.lo[d:d + 1],
                            hi=prob.hi[d:d + 1], cells=prob.cells[d:d + 1],
                            inputs=np.zeros((1, 1)), sigma=prob.sigma[d:d + 1], cutoff=0.0,
                            images=np.array([[[m_lo[d], m_hi[d]]]] * int(prob.cells[d])))
            up1, _, _, _ = orc.row_dense(one, 0)
            total *= math.fsum(up1.tolist())
        _, _, up = csr.row(k)
        got = math.fsum(up.tolist()) + csr.trunc[k]
        assert abs(got - total) <= 1e-13 * total, (row, got, total)


def pin_tie_kept(orc):
    prob = W.robot_2d(cells_per_dim=7)
    up, _, _, _ = orc.row_dense(prob, 40)
    t = int(np.argsort(up)[len(up) // 2])
    prob.cutoff = float(up[t])
    csr = orc.build_rows(prob, [40])
    cols, _, _ = csr.row(0)
    assert t in set(cols.tolist())
    assert np.all(up[cols] >= prob.cutoff)
    assert len(cols) == int(np.sum(up >= prob.cutoff))


def coupled_cases():
    """(problem, rows) pairs with coupled or nonlinear dynamics, small grids."""
    room = W.room_5d(cells_per_dim=4)
    bas = W.bas_4d(eta_scale=2.0)
    uni = W.unicycle_3d(nx=6, ny=6, nth=7)
    lin = W.random_linear(7, min_cells=200, max_cells=2000)
    b7 = W.building_7d(cells_per_dim=3)
    return [(room, W.sample_rows(room, 4, seed=1)), (bas, W.sample_rows(bas, 4, seed=2)),
            (uni, W.sample_rows(uni, 6, seed=3)), (lin, W.sample_rows(lin, 4, seed=4)),
            (b7, W.sample_rows(b7, 2, seed=5, include_boundary=False))]


# --------------------------------------------------------------------------
# regions (Sec. 3.1, Alg. 1, Remark 4.1)
# --------------------------------------------------------------------------


def region_cases():
    """(problem, target boxes, avoid boxes, rows): regions away from cell
    centres (the labels do not hinge on a rounding), rows near and far."""
    robot = W.robot_2d(cells_per_dim=9)
    room = W.room_5d(cells_per_dim=4)
    uni = W.unicycle_3d(nx=6, ny=6, nth=5)
    b7 = W.building_7d(cells_per_dim=3)
    return [
        (robot, [([3.1, 3.1], [7.2, 7.2])],
         [([-7.2, -7.2], [-3.1, -3.1]), ([-9.6, 4.1], [-5.9, 9.3])],
         [0, 40, 120, 301, 365, 601, 700]),
        (room, [([18.4] * 5, [21.6] * 5)], [([17.0] * 5, [18.1, 23, 23, 23, 23])],
         W.sample_rows(room, 4, seed=21)),
        (uni, [([1.0, 1.0, -4.0], [5.0, 5.0, 4.0])], [([-5.0, -1.0, -4.0], [-1.2, 1.0, 4.0])],
         W.sample_rows(uni, 4, seed=22)),
        (b7, [([-3.0] * 7, [-0.5] + [3.0] * 6)], [([0.5] + [-3.0] * 6, [3.0] * 7)],
         W.sample_rows(b7, 2, seed=23, include_boundary=False)),
    ]


def pin_region_labels(orc):
    """The oracle's labels against the generator module's own restatement
    (cell centres on a mesh), and avoid winning where boxes overlap."""
    for prob, tb, ab, _ in region_cases():
        got = orc.region_labels(prob, tb, ab)
        assert np.array_equal(got, W.region_labels(prob, target=tb, avoid=ab)), prob.name
    robot = W.robot_2d(cells_per_dim=9)
    big, small = ([-8.0, -8.0], [8.0, 8.0]), ([-1.0, -1.0], [1.0, 1.0])
    lab = orc.region_labels(robot, [big], [small]).reshape(9, 9)
    assert lab[4, 4] == 2 and lab[3, 3] == 1 and lab[0, 0] == 0
    assert np.array_equal(orc.region_labels(robot, [small], [big]) == 2,
                          orc.region_labels(robot, [], [big]) == 2)


def pin_region_containment(orc, samples=24, seed=7):
    """For points x of the source cell the exact probability of landing in
    the labelled cells (a sum of library-CDF products over every labelled
    cell) lies in [R_min, R_max]; the probability of an avoid cell or of
    leaving the domain in [A_min, A_max]. Both modes."""
    rng = np.random.default_rng(seed)
    for prob, tb, ab, rows in region_cases():
        labels = W.region_labels(prob, target=tb, avoid=ab)
        for mode in ("box", "cells"):
            r_lo, r_up, a_lo, a_up = orc.region_vectors(prob, rows, tb, ab, mode)
            for k, row in enumerate(rows):
                cell, j = divmod(int(row), prob.n_inputs)
                bl, bh = cell_box(prob, cell)
                xs = bl + (bh - bl) * rng.random((samples, prob.n))
                corners = np.array([[bh[d] if (c >> d) & 1 else bl[d] for d in range(prob.n)]
                                    for c in range(1 << prob.n)])
                for mu in dynamics(prob, np.concatenate([xs, corners]), prob.inputs[j]):
                    P, out = exact_probs(prob, mu)
                    pr = float(np.sum(P[labels == 1]))
                    pa = float(np.sum(P[labels == 2])) + out
                    assert r_lo[k] - 1e-13 <= pr <= r_up[k] + 1e-13, (prob.name, mode, row, pr)
                    assert a_lo[k] - 1e-13 <= pa <= a_up[k] + 1e-13, (prob.name, mode, row, pa)


def pin_region_box_exact_separable(orc):
    """Separable 2-D system: the box relaxation of a region is the exact
    min / max over the cell of the probability of landing in it (the min at
    a corner, the max the product of numerically maximised 1-D factors)."""
    prob, tb, ab, rows = region_cases()[0]
    labels = W.region_labels(prob, target=tb, avoid=ab).reshape(9, 9)
    ii = np.nonzero(labels == 1)
    span = [(ii[d].min(), ii[d].max()) for d in range(2)]
    r_lo, r_up, _, _ = orc.region_vectors(prob, rows, tb, ab, "box")
    for k, row in enumerate(rows):
        cell, j = divmod(int(row), prob.n_inputs)
        u = prob.inputs[j]
        bl, bh = cell_box(prob, cell)
        mass = []
        for d in range(2):
            e = grid_edges(prob, d)
            a, b = e[span[d][0]], e[span[d][1] + 1]
            mass.append((lambda x, a=a, b=b, d=d: float(interval_mass(a, b, x + u[d],
                                                                      prob.sigma[d]))))
        corners = [(x0, x1) for x0 in (bl[0], bh[0]) for x1 in (bl[1], bh[1])]
        lo_ref = min(mass[0](x0) * mass[1](x1) for x0, x1 in corners)
        up_ref = (_max_over_interval(mass[0], bl[0], bh[0])
                  * _max_over_interval(mass[1], bl[1], bh[1]))
        assert abs(r_lo[k] - lo_ref) <= 1e-14 + 1e-12 * lo_ref, (row, r_lo[k], lo_ref)
        assert r_up[k] >= up_ref - 1e-14 and r_up[k] - up_ref < 1e-9, (row, r_up[k], up_ref)


def pin_region_reductions(orc):
    """One-cell regions equal that cell's own bounds in both modes; the box
    bounds lie inside the paper's sums of per-cell bounds; a region covering
    the whole domain is the complement of the sink."""
    prob = W.robot_2d(cells_per_dim=9)
    rows = [0, 40, 77, 300, 555]
    e0 = grid_edges(prob, 0)
    t = (5, 6)                                           # the cell, as (i0, i1)
    box = ([e0[t[0]] + 0.3, e0[t[1]] + 0.3], [e0[t[0] + 1] - 0.3, e0[t[1] + 1] - 0.3])
    tcell = t[0] * 9 + t[1]
    for mode in ("box", "cells"):
        r_lo, r_up, a_lo, a_up = orc.region_vectors(prob, rows, [box], [], mode)
        for k, row in enumerate(rows):
            up, lo, sl, su = orc.row_dense(prob, row)
            assert abs(r_lo[k] - lo[tcell]) <= 1e-15 * max(1.0, lo[tcell]), (mode, row)
            assert abs(r_up[k] - up[tcell]) <= 1e-15 * max(1.0, up[tcell]), (mode, row)
            assert a_lo[k] == sl and a_up[k] == su
    for prob, tb, ab, rows in region_cases():
        B = orc.region_vectors(prob, rows, tb, ab, "box")
        C = orc.region_vectors(prob, rows, tb, ab, "cells")
        for lo_i, up_i in ((0, 1), (2, 3)):
            assert np.all(C[lo_i] <= B[lo_i] + 1e-15), prob.name
            assert np.all(B[up_i] <= C[up_i] + 1e-15), prob.name
            assert np.all(B[lo_i] <= B[up_i] + 1e-15), prob.name
        whole = (prob.lo, prob.hi)
        r_lo, r_up, _, _ = orc.region_vectors(prob, rows, [whole], [], "box")
        csr = orc.build_rows(prob, rows)
        assert np.all(np.abs(r_lo - (1.0 - csr.sink_up)) < 1e-15), prob.name
        assert np.all(np.abs(r_up - (1.0 - csr.sink_lo)) < 1e-15), prob.name


# --------------------------------------------------------------------------
# sampled noise (Sec. 4.1: Monte-Carlo integration for full covariance or a
# custom distribution)
# --------------------------------------------------------------------------


def _binomial_ok(est, p, S, k=5.0):
    """|est - p| within k binomial standard deviations (plus one count)."""
    sd = np.sqrt(np.maximum(p * (1.0 - p), 0.0) / S)
    return np.abs(est - p) <= k * sd + 1.0 / S


def pin_mc_cell_of(orc):
    """Cell of a coordinate: the library's sorted search over the edges."""
    prob = W.robot_2d(cells_per_dim=9)
    e = grid_edges(prob, 0)
    ys = np.concatenate([e, np.nextafter(e, -np.inf), np.nextafter(e, np.inf), [-50.0, 50.0],
                         np.linspace(-11, 11, 97)])
    for y in ys:
        if y < e[0]:
            ref = -1
        elif y > e[-1]:
            ref = 9
        else:
            ref = min(int(np.searchsorted(e, y, side="right")) - 1, 8)
        assert orc.cell_of(prob, 0, float(y)) == ref, y


def mc_images(prob, seed, width):
    """Images of every row: a random centre per row and the given widths."""
    rng = np.random.default_rng(seed)
    n = prob.n
    mid = prob.lo + (prob.hi - prob.lo) * rng.uniform(0.1, 0.9, (prob.rows, n))
    im = np.stack([mid - 0.5 * np.asarray(width), mid + 0.5 * np.asarray(width)], axis=2)
    return W.with_images(prob, im)


def pin_mc_point_images(orc, S=20000, seed=31):
    """Point images: up == lo for every target, and the fractions agree with
    the closed-form Gaussian cell mass (diagonal noise, library CDF) and with
    the library's bivariate normal CDF (full covariance) within 5 binomial
    standard deviations."""
    from scipy.stats import multivariate_normal
    base = W.robot_2d(cells_per_dim=7)
    prob = mc_images(base, seed, [0.0, 0.0])
    rng = np.random.default_rng(seed)
    rows = [3, 50, 200, 400]
    sig = np.asarray(base.sigma)
    w = rng.normal(0.0, 1.0, (S, 2)) * sig
    csr = orc.build_rows_mc(prob, w, rows)
    for k, row in enumerate(rows):
        cols, lo, up = csr.row(k)
        assert np.array_equal(lo, up)
        mu = prob.images[row][:, 0]
        P, out = exact_probs(base, mu)
        assert np.all(_binomial_ok(up, P[cols], S)), row
        missing = np.setdiff1d(np.arange(P.size), cols)
        assert np.all(P[missing] < 6.0 / np.sqrt(S)), row
        assert _binomial_ok(csr.sink_lo[k], out, S) and csr.sink_lo[k] == csr.sink_up[k]
    # full covariance: w = L z
    cov = np.array([[1.0, 0.6], [0.6, 0.8]]) * 0.6 ** 2
    L = np.linalg.cholesky(cov)
    w = rng.normal(0.0, 1.0, (S, 2)) @ L.T
    csr = orc.build_rows_mc(prob, w, rows)
    e0, e1 = grid_edges(base, 0), grid_edges(base, 1)
    for k, row in enumerate(rows):
        cols, lo, up = csr.row(k)
        mu = prob.images[row][:, 0]
        F = multivariate_normal(mean=mu, cov=cov)
        for t, u in zip(cols[::3], up[::3]):
            i, j = divmod(int(t), 7)
            p = (F.cdf([e0[i + 1], e1[j + 1]]) - F.cdf([e0[i], e1[j + 1]])
                 - F.cdf([e0[i + 1], e1[j]]) + F.cdf([e0[i], e1[j]]))
            assert _binomial_ok(u, max(p, 0.0), S) or abs(u - p) < 2e-4, (row, t, u, p)


def pin_mc_box_images(orc, S=20000, seed=32):
    """Wide images, diagonal noise: the fraction of draws whose moved box
    meets a cell / lies inside it / leaves the domain have product closed
    forms (independent coordinates)."""
    base = W.robot_2d(cells_per_dim=7)
    width = [1.3, 0.4]
    prob = mc_images(base, seed, width)
    rng = np.random.default_rng(seed)
    sig = np.asarray(base.sigma)
    w = rng.normal(0.0, 1.0, (S, 2)) * sig
    rows = [7, 99, 250, 420]
    csr = orc.build_rows_mc(prob, w, rows)
    E = [grid_edges(base, d) for d in range(2)]
    for k, row in enumerate(rows):
        mlo, mhi = prob.images[row][:, 0], prob.images[row][:, 1]
        # P(w in [c - m_hi, e - m_lo]) = mass of [c, e + m_hi - m_lo] around m_hi
        meet = [interval_mass(E[d][:-1], E[d][1:] + (mhi[d] - mlo[d]), mhi[d], sig[d])
                for d in range(2)]
        inside = [np.where(E[d][1:] - E[d][:-1] >= mhi[d] - mlo[d],
                           interval_mass(E[d][:-1] + (mhi[d] - mlo[d]), np.maximum(
                               E[d][1:], E[d][:-1] + (mhi[d] - mlo[d])), mhi[d], sig[d]), 0.0)
                  for d in range(2)]
        Pm = np.multiply.outer(meet[0], meet[1]).reshape(-1)
        Pi = np.multiply.outer(inside[0], inside[1]).reshape(-1)
        cols, lo, up = csr.row(k)
        assert np.all(_binomial_ok(up, Pm[cols], S)), row
        assert np.all(_binomial_ok(lo, Pi[cols], S)), row
        stay = np.prod([float(interval_mass(base.lo[d] + (mhi[d] - mlo[d]), base.hi[d], mhi[d],
                                            sig[d])) for d in range(2)])
        touch = np.prod([float(interval_mass(base.lo[d], base.hi[d] + (mhi[d] - mlo[d]), mhi[d],
                                             sig[d])) for d in range(2)])
        assert _binomial_ok(csr.sink_up[k], 1.0 - stay, S), row
        assert _binomial_ok(csr.sink_lo[k], 1.0 - touch, S), row


def pin_mc_counting(orc, S=3000, seed=33):
    """Exact counting identities: every draw lands in at most one lo cell or
    the sink's lo, and meets at least one cell or the sink's up; and a brute
    force over every cell with the edges searched by the library agrees
    count for count."""
    base = W.robot_2d(cells_per_dim=6)
    prob = mc_images(base, seed, [0.9, 2.1])
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, 1.0, (S, 2)) * np.asarray(base.sigma) * 2.0
    prob.cutoff = 0.02
    rows = [0, 11, 100, 200, 323]
    csr = orc.build_rows_mc(prob, w, rows)
    E = [grid_edges(base, d) for d in range(2)]

    def cell(d, y):
        if y < E[d][0]:
            return -1
        if y > E[d][-1]:
            return 6
        return min(int(np.searchsorted(E[d], y, side="right")) - 1, 5)

    for k, row in enumerate(rows):
        cols, lo, up = csr.row(k)
        mlo, mhi = prob.images[row][:, 0], prob.images[row][:, 1]
        cu = np.zeros(36, np.int64)
        cl = np.zeros(36, np.int64)
        part = whole = 0
        for s in range(S):
            a = [cell(d, w[s, d] + mlo[d]) for d in range(2)]
            b = [cell(d, w[s, d] + mhi[d]) for d in range(2)]
            part += any(a[d] < 0 or b[d] > 5 for d in range(2))
            whole += any(b[d] < 0 or a[d] > 5 for d in range(2))
            for i in range(max(a[0], 0), min(b[0], 5) + 1):
                for j in range(max(a[1], 0), min(b[1], 5) + 1):
                    cu[i * 6 + j] += 1
                    if a == b:
                        cl[i * 6 + j] += 1
        kept = np.nonzero(cu / S >= prob.cutoff)[0]
        assert np.array_equal(cols, kept), row
        assert np.array_equal(np.round(up * S).astype(np.int64), cu[kept]), row
        assert np.array_equal(np.round(lo * S).astype(np.int64), cl[kept]), row
        assert round(csr.trunc[k] * S) == cu.sum() - cu[kept].sum(), row
        assert round(csr.sink_up[k] * S) == part and round(csr.sink_lo[k] * S) == whole, row
        # every draw: at most one lo cell or the sink's lo; at least one cell
        # met or the sink's up
        assert cl.sum() + whole <= S and cu.sum() + part >= S
