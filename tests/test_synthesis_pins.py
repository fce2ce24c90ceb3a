"""Pins of the oracle's interval-iteration synthesis (CPU only).

- the sorting-method LP against a general LP solver (scipy linprog) on random
  interval constraints (Sec. 6.2: the sorting method solves the LP of Sec. 5);
- degenerate intervals (lo == up) turn the IMDP into an MDP: the gambler's
  ruin closed form, and the optimum over every stationary policy by linear
  solves, for reach-avoid and safety;
- the whole iteration with each LP solved by linprog instead of sorting;
- invariants on a real abstraction (2-D robot, reach-avoid).
"""

import itertools

import numpy as np
import pytest

from oracle import synthesis as SY

linprog = pytest.importorskip("scipy.optimize").linprog


class Imdp:
    """A hand-made IMDP in the layout of oracle.build_rows' result."""

    def __init__(self, rows):
        # rows: list of (targets [(col, lo, up)], sink_lo, sink_up, trunc)
        ptr, col, lo, up, sl, su, tr = [0], [], [], [], [], [], []
        for succ, a, b, t in rows:
            for c, l, u in succ:
                col.append(c)
                lo.append(l)
                up.append(u)
            ptr.append(len(col))
            sl.append(a)
            su.append(b)
            tr.append(t)
        self.row_ptr = np.array(ptr, np.int64)
        self.col = np.array(col, np.int32)
        self.lo = np.array(lo, np.float64)
        self.up = np.array(up, np.float64)
        self.sink_lo = np.array(sl, np.float64)
        self.sink_up = np.array(su, np.float64)
        self.trunc = np.array(tr, np.float64)


def lp_general(lo, up, v, maximize):
    c = -np.asarray(v) if maximize else np.asarray(v)
    res = linprog(c, A_eq=np.ones((1, len(lo))), b_eq=[1.0],
                  bounds=list(zip(lo, up)), method="highs")
    assert res.status == 0
    return float(np.dot(res.x, v))


@pytest.mark.parametrize("seed", range(40))
def test_sorting_method_equals_linear_program(seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 9))
    lo = rng.uniform(0, 1, k)
    lo *= rng.uniform(0.2, 1.0) / lo.sum()            # sum lo <= 1
    up = lo + rng.uniform(0, 1, k)
    if up.sum() < 1.0:
        up[0] += 1.0 - up.sum()                      # sum up >= 1
    v = rng.uniform(0, 1, k)
    v[rng.integers(k)] = v[0]                        # a tie
    for maximize in (False, True):
        assert abs(SY.lp_sorted(lo, up, v, maximize) - lp_general(lo, up, v, maximize)) < 1e-9


def chain(N, p, one_input=True):
    """Gambler's ruin on states 0..N: from i, to i+1 with p, to i-1 with 1-p;
    0 is avoid, N target. Degenerate intervals."""
    rows = []
    for i in range(N + 1):
        if 0 < i < N:
            rows.append(([(i + 1, p, p), (i - 1, 1 - p, 1 - p)], 0.0, 0.0, 0.0))
        else:
            rows.append(([(i, 1.0, 1.0)], 0.0, 0.0, 0.0))
    labels = np.zeros(N + 1, np.int8)
    labels[0] = SY.AVOID
    labels[N] = SY.TARGET
    return Imdp(rows), labels


@pytest.mark.parametrize("p", [0.3, 0.5, 0.6])
def test_gamblers_ruin_closed_form(p):
    N = 8
    imdp, labels = chain(N, p)
    res = SY.interval_iteration(imdp, labels, 1, SY.REACH_AVOID, eps=1e-12, max_iters=200000)
    i = np.arange(N + 1)
    if p == 0.5:
        exact = i / N
    else:
        r = (1 - p) / p
        exact = (1 - r ** i) / (1 - r ** N)
    assert res.converged[0] and res.converged[1]
    assert np.max(np.abs(res.p_min - exact)) < 1e-9
    assert np.max(np.abs(res.p_max - exact)) < 1e-9


def random_mdp(seed, S=5, U=2):
    """Random MDP (lo == up) with a sink and one target, one avoid state."""
    rng = np.random.default_rng(seed)
    rows = []
    for s in range(S):
        for u in range(U):
            w = rng.uniform(0, 1, S + 1)
            w /= w.sum()
            rows.append(([(t, w[t], w[t]) for t in range(S)], w[S], w[S], 0.0))
    labels = np.zeros(S, np.int8)
    labels[S - 1] = SY.TARGET
    labels[0] = SY.AVOID
    return Imdp(rows), labels, rng


def policy_values(imdp, labels, U, policy, goal):
    """Probability of reaching `goal` states (1) before the absorbing others
    under a stationary policy, by one linear solve."""
    S = labels.shape[0]
    P = np.zeros((S, S))
    g = np.zeros(S)
    for s in range(S):
        r = s * U + policy[s]
        a, b = imdp.row_ptr[r], imdp.row_ptr[r + 1]
        for c, w in zip(imdp.col[a:b], imdp.lo[a:b]):
            P[s, c] += w
        g[s] = goal[1] * imdp.sink_lo[r]
    A = np.eye(S)
    rhs = np.zeros(S)
    for s in range(S):
        if labels[s] == SY.FREE:
            A[s] -= P[s]
            rhs[s] = g[s]
        else:
            rhs[s] = goal[0][s]
    return np.linalg.solve(A, rhs)


@pytest.mark.parametrize("seed", range(6))
def test_degenerate_imdp_equals_best_policy(seed):
    U = 2
    imdp, labels, _ = random_mdp(seed, U=U)
    S = labels.shape[0]
    free = np.nonzero(labels == SY.FREE)[0]
    # reach-avoid: max over policies of P(target before avoid or sink)
    ra = SY.interval_iteration(imdp, labels, U, SY.REACH_AVOID, eps=1e-12, max_iters=100000)
    # safety: min over policies of P(avoid or sink), reported as 1 - that
    sf = SY.interval_iteration(imdp, labels, U, SY.SAFETY, eps=1e-12, max_iters=100000)
    best_reach = np.full(S, -1.0)
    best_unsafe = np.full(S, 2.0)
    for choice in itertools.product(range(U), repeat=len(free)):
        pol = np.zeros(S, np.int64)
        pol[free] = choice
        reach = policy_values(imdp, labels, U, pol, ((labels == SY.TARGET) * 1.0, 0.0))
        unsafe = policy_values(imdp, labels, U, pol, ((labels == SY.AVOID) * 1.0, 1.0))
        best_reach = np.maximum(best_reach, reach)
        best_unsafe = np.minimum(best_unsafe, unsafe)
    assert np.max(np.abs(ra.p_min - best_reach)) < 1e-8
    assert np.max(np.abs(ra.p_max - best_reach)) < 1e-8
    assert np.max(np.abs(sf.p_min - (1 - best_unsafe))) < 1e-8
    assert np.max(np.abs(sf.p_max - (1 - best_unsafe))) < 1e-8


def interval_iteration_linprog(imdp, labels, U, eps=1e-10, max_iters=5000):
    """Reach-avoid phase 1 with every LP solved by linprog (independent of the
    sorting method)."""
    free = labels == SY.FREE
    fixed = np.where(labels == SY.TARGET, 1.0, 0.0)
    V0 = np.where(free, 0.0, fixed)
    V1 = np.where(free, 1.0, fixed)
    for _ in range(max_iters):
        if np.max(np.abs(V1 - V0)) <= eps:
            break
        N0, N1 = V0.copy(), V1.copy()
        for c in np.nonzero(free)[0]:
            vals0, vals1 = [], []
            for j in range(U):
                r = c * U + j
                a, b = imdp.row_ptr[r], imdp.row_ptr[r + 1]
                lo = np.concatenate([imdp.lo[a:b], [imdp.sink_lo[r], 0.0]])
                up = np.concatenate([imdp.up[a:b], [imdp.sink_up[r], imdp.trunc[r]]])
                col = imdp.col[a:b]
                vals0.append(lp_general(lo, up, np.concatenate([V0[col], [0.0, 0.0]]), False))
                vals1.append(lp_general(lo, up, np.concatenate([V1[col], [0.0, 0.0]]), False))
            N0[c], N1[c] = max(vals0), max(vals1)
        V0, V1 = N0, N1
    return V0


@pytest.mark.parametrize("seed", range(3))
def test_interval_imdp_against_linprog_iteration(seed):
    rng = np.random.default_rng(100 + seed)
    S, U = 5, 2
    rows = []
    for s in range(S):
        for u in range(U):
            w = rng.uniform(0, 1, S + 1)
            w /= w.sum()
            lo = np.maximum(w - rng.uniform(0, 0.1, S + 1), 0.0)
            up = np.minimum(w + rng.uniform(0, 0.1, S + 1), 1.0)
            rows.append(([(t, lo[t], up[t]) for t in range(S)], lo[S], up[S], 0.02))
    imdp = Imdp(rows)
    labels = np.zeros(S, np.int8)
    labels[S - 1] = SY.TARGET
    labels[0] = SY.AVOID
    res = SY.interval_iteration(imdp, labels, U, SY.REACH_AVOID, eps=1e-10, max_iters=5000)
    ref = interval_iteration_linprog(imdp, labels, U)
    assert np.max(np.abs(res.p_min - ref)) < 1e-7
    assert np.all(res.p_min <= res.p_max + 1e-12)


def test_robot_abstraction_invariants():
    import oracle
    from paper_2401_03555_gb300 import workloads as W
    prob = W.robot_2d(cells_per_dim=7)
    csr = oracle.build_rows(prob)
    labels = W.region_labels(prob, target=([3, 3], [7, 7]), avoid=([-7, -7], [-3, -3]))
    res = SY.interval_iteration(csr, labels, prob.n_inputs, SY.REACH_AVOID, eps=1e-6)
    assert res.converged[0]
    assert np.all(res.p_min >= -1e-12) and np.all(res.p_max <= 1 + 1e-12)
    assert np.all(res.p_min <= res.p_max + 1e-9)
    assert np.all(res.p_min[labels == SY.TARGET] == 1.0)
    assert np.all(res.p_max[labels == SY.AVOID] == 0.0)
    assert res.p_min.max() > 0.5
