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


# ---- finite horizon (Remark 5.1) ------------------------------------------


def walk_value(imdp, labels, U, pol, K, goal, sink_goal):
    """Probability of hitting a `goal` state within K steps (absorbing labelled
    states count by `goal`, the sink by `sink_goal`) when pol[t][s] is the
    input at step t; computed by following the policy step by step."""
    S = labels.shape[0]

    def val(s, t):
        if labels[s] != SY.FREE:
            return goal[s]
        if t == K:
            return 0.0
        r = s * U + pol[t][s]
        a, b = imdp.row_ptr[r], imdp.row_ptr[r + 1]
        v = 0.0
        for c, w in zip(imdp.col[a:b], imdp.lo[a:b]):
            v += w * val(c, t + 1)
        return v + imdp.sink_lo[r] * sink_goal

    return np.array([val(s, 0) for s in range(S)])


@pytest.mark.parametrize("seed", range(4))
def test_finite_horizon_equals_the_best_time_varying_policy(seed):
    """Degenerate intervals, K = 3: phase 1 equals the best over every
    time-varying policy (enumerated); phase 2 equals the stationary policy it
    fixes, run for K steps."""
    U, K = 2, 3
    imdp, labels, _ = random_mdp(seed, U=U)
    S = labels.shape[0]
    free = np.nonzero(labels == SY.FREE)[0]
    target = (labels == SY.TARGET) * 1.0
    unsafe = (labels == SY.AVOID) * 1.0
    best_reach = np.full(S, -1.0)
    best_unsafe = np.full(S, 2.0)
    for choice in itertools.product(range(U), repeat=len(free) * K):
        pol = np.zeros((K, S), np.int64)
        pol[:, free] = np.array(choice).reshape(K, len(free))
        best_reach = np.maximum(best_reach, walk_value(imdp, labels, U, pol, K, target, 0.0))
        best_unsafe = np.minimum(best_unsafe, walk_value(imdp, labels, U, pol, K, unsafe, 1.0))
    ra = SY.interval_iteration(imdp, labels, U, SY.REACH_AVOID, horizon=K)
    sf = SY.interval_iteration(imdp, labels, U, SY.SAFETY, horizon=K)
    assert ra.iterations == (K, K) and sf.iterations == (K, K)
    assert np.max(np.abs(ra.p_min - best_reach)) < 1e-12
    assert np.max(np.abs(sf.p_min - (1.0 - best_unsafe))) < 1e-12
    stat = np.tile(ra.policy, (K, 1))
    assert np.max(np.abs(ra.p_max - walk_value(imdp, labels, U, stat, K, target, 0.0))) < 1e-12
    stat = np.tile(sf.policy, (K, 1))
    assert np.max(np.abs(sf.p_max - (1.0 - walk_value(imdp, labels, U, stat, K, unsafe, 1.0)))) \
        < 1e-12


def test_long_horizon_approaches_the_infinite_horizon_value():
    imdp, labels = chain(8, 0.55)
    inf = SY.interval_iteration(imdp, labels, 1, SY.REACH_AVOID, eps=1e-13, max_iters=100000)
    prev = None
    for K in (5, 50, 2000):
        fin = SY.interval_iteration(imdp, labels, 1, SY.REACH_AVOID, horizon=K)
        assert np.all(fin.p_min <= inf.p_min + 1e-12)
        if prev is not None:
            assert np.all(fin.p_min >= prev - 1e-15)     # more steps, more mass reached
        prev = fin.p_min
    assert np.max(np.abs(prev - inf.p_min)) < 1e-10


# ---- disturbances: the adversary's axis ------------------------------------


def random_game(seed, S=5, U=2, Wn=2):
    rng = np.random.default_rng(300 + seed)
    rows = []
    for s in range(S):
        for u in range(U):
            for k in range(Wn):
                w = rng.uniform(0, 1, S + 1)
                w /= w.sum()
                rows.append(([(t, w[t], w[t]) for t in range(S)], w[S], w[S], 0.0))
    labels = np.zeros(S, np.int8)
    labels[S - 1] = SY.TARGET
    labels[0] = SY.AVOID
    return Imdp(rows), labels


def game_policy_values(imdp, labels, U, Wn, sig, tau, goal, sink_goal):
    """Hitting probability of the goal under the input policy sig[s] and the
    disturbance policy tau[s] (one linear solve)."""
    S = labels.shape[0]
    P = np.zeros((S, S))
    g = np.zeros(S)
    for s in range(S):
        r = (s * U + sig[s]) * Wn + tau[s]
        a, b = imdp.row_ptr[r], imdp.row_ptr[r + 1]
        for c, w in zip(imdp.col[a:b], imdp.lo[a:b]):
            P[s, c] += w
        g[s] = sink_goal * imdp.sink_lo[r]
    A = np.eye(S)
    rhs = np.zeros(S)
    for s in range(S):
        if labels[s] == SY.FREE:
            A[s] -= P[s]
            rhs[s] = g[s]
        else:
            rhs[s] = goal[s]
    return np.linalg.solve(A, rhs)


@pytest.mark.parametrize("seed", range(4))
def test_disturbance_game_equals_enumerated_strategies(seed):
    """Degenerate intervals: the input maximises and the disturbance
    minimises satisfaction; the value equals the best input strategy against
    its worst disturbance strategy, both enumerated over stationary choices."""
    U, Wn = 2, 2
    imdp, labels = random_game(seed, U=U, Wn=Wn)
    S = labels.shape[0]
    free = np.nonzero(labels == SY.FREE)[0]
    target = (labels == SY.TARGET) * 1.0
    unsafe = (labels == SY.AVOID) * 1.0
    reach = np.full(S, -1.0)
    safe_unsafe = np.full(S, 2.0)
    for cs in itertools.product(range(U), repeat=len(free)):
        sig = np.zeros(S, np.int64)
        sig[free] = cs
        worst_r = np.full(S, 2.0)
        worst_u = np.full(S, -1.0)
        for ct in itertools.product(range(Wn), repeat=len(free)):
            tau = np.zeros(S, np.int64)
            tau[free] = ct
            worst_r = np.minimum(worst_r, game_policy_values(imdp, labels, U, Wn, sig, tau,
                                                             target, 0.0))
            worst_u = np.maximum(worst_u, game_policy_values(imdp, labels, U, Wn, sig, tau,
                                                             unsafe, 1.0))
        reach = np.maximum(reach, worst_r)
        safe_unsafe = np.minimum(safe_unsafe, worst_u)
    ra = SY.interval_iteration(imdp, labels, U, SY.REACH_AVOID, eps=1e-13, max_iters=100000,
                               n_disturb=Wn)
    sf = SY.interval_iteration(imdp, labels, U, SY.SAFETY, eps=1e-13, max_iters=100000,
                               n_disturb=Wn)
    for got in (ra.p_min, ra.p_max):
        assert np.max(np.abs(got - reach)) < 1e-9
    for got in (sf.p_min, sf.p_max):
        assert np.max(np.abs(got - (1.0 - safe_unsafe))) < 1e-9


# ---- optimistic policy ------------------------------------------------------


def interval_iteration_linprog_max(imdp, labels, U, eps=1e-10, max_iters=5000):
    """Reach-avoid with every LP the max LP (truncated mass valued 1), solved
    by linprog: the optimistic phase 1."""
    free = labels == SY.FREE
    fixed = np.where(labels == SY.TARGET, 1.0, 0.0)
    V = np.where(free, 0.0, fixed)
    for _ in range(max_iters):
        N = V.copy()
        for c in np.nonzero(free)[0]:
            vals = []
            for j in range(U):
                r = c * U + j
                a, b = imdp.row_ptr[r], imdp.row_ptr[r + 1]
                lo = np.concatenate([imdp.lo[a:b], [imdp.sink_lo[r], 0.0]])
                up = np.concatenate([imdp.up[a:b], [imdp.sink_up[r], imdp.trunc[r]]])
                vals.append(lp_general(lo, up, np.concatenate([V[imdp.col[a:b]], [0.0, 1.0]]),
                                       True))
            N[c] = max(vals)
        if np.max(np.abs(N - V)) <= eps:
            return N
        V = N
    return V


@pytest.mark.parametrize("seed", range(2))
def test_optimistic_phase_one_against_linprog(seed):
    rng = np.random.default_rng(500 + seed)
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
    opt = SY.interval_iteration(imdp, labels, U, SY.REACH_AVOID, eps=1e-11, max_iters=5000,
                                optimistic=True)
    pes = SY.interval_iteration(imdp, labels, U, SY.REACH_AVOID, eps=1e-11, max_iters=5000)
    assert np.max(np.abs(opt.p_max - interval_iteration_linprog_max(imdp, labels, U))) < 1e-7
    # the optimistic policy's upper bound is the best possible one, the
    # pessimistic policy's lower bound the best possible one
    assert np.all(opt.p_max >= pes.p_max - 1e-9)
    assert np.all(pes.p_min >= opt.p_min - 1e-9)


@pytest.mark.parametrize("seed", range(3))
def test_optimistic_equals_pessimistic_without_interval_freedom(seed):
    imdp, labels, _ = random_mdp(seed, U=2)
    for spec in (SY.REACH_AVOID, SY.SAFETY):
        a = SY.interval_iteration(imdp, labels, 2, spec, eps=1e-12, max_iters=100000)
        b = SY.interval_iteration(imdp, labels, 2, spec, eps=1e-12, max_iters=100000,
                                  optimistic=True)
        assert np.max(np.abs(a.p_min - b.p_min)) < 1e-9
        assert np.max(np.abs(a.p_max - b.p_max)) < 1e-9


# ---- region vectors in the LP (Sec. 3.1, Sec. 5) ----------------------------


def robot_regions():
    import oracle
    from paper_2401_03555_gb300 import workloads as W
    prob = W.robot_2d(cells_per_dim=7)
    tb = [([2.0, 2.0], [9.0, 9.0])]        # 3 x 3 cells each
    ab = [([-9.0, -9.0], [-2.0, -2.0])]
    return oracle, prob, tb, ab


@pytest.mark.parametrize("spec", [SY.REACH_AVOID, SY.SAFETY])
def test_paper_region_sums_equal_the_labelled_columns(spec):
    """R and A as the paper's sums of per-cell bounds (every cell kept:
    cutoff 0) give the same LPs as the labelled cells kept as columns."""
    oracle, prob, tb, ab = robot_regions()
    csr = oracle.build_rows(prob)
    labels = oracle.region_labels(prob, tb, ab)
    vec = oracle.region_vectors(prob, None, tb, ab, "cells")
    a = SY.interval_iteration(csr, labels, prob.n_inputs, spec, eps=1e-10, max_iters=5000)
    b = SY.interval_iteration(csr, labels, prob.n_inputs, spec, eps=1e-10, max_iters=5000,
                              regions=vec)
    assert np.max(np.abs(a.p_min - b.p_min)) < 1e-11
    assert a.iterations[0] == b.iterations[0]
    if spec == SY.REACH_AVOID:
        assert np.max(np.abs(a.p_max - b.p_max)) < 1e-11
        assert a.iterations == b.iterations
    else:
        # most cells are lost under the pessimistic safety LP (unsafe value
        # ~1 for every input): rounding picks among tied inputs, so compare
        # how good each policy is under the other formulation's phase 1
        V = 1.0 - a.p_min                                   # unsafe values
        U = prob.n_inputs
        for c in np.nonzero(labels == SY.FREE)[0]:
            vals = [SY._row_value(csr, c * U + j, V, 1.0, 1.0, True) for j in range(U)]
            assert vals[b.policy[c]] <= min(vals) + 1e-9


@pytest.mark.parametrize("spec", [SY.REACH_AVOID, SY.SAFETY])
def test_region_boxes_tighten_the_pessimistic_bound(spec):
    """Box relaxations lie inside the per-cell sums, so the optimal
    pessimistic bound can only rise."""
    oracle, prob, tb, ab = robot_regions()
    csr = oracle.build_rows(prob)
    labels = oracle.region_labels(prob, tb, ab)
    cells = SY.interval_iteration(csr, labels, prob.n_inputs, spec, eps=1e-10, max_iters=5000,
                                  regions=oracle.region_vectors(prob, None, tb, ab, "cells"))
    box = SY.interval_iteration(csr, labels, prob.n_inputs, spec, eps=1e-10, max_iters=5000,
                                regions=oracle.region_vectors(prob, None, tb, ab, "box"))
    assert np.all(box.p_min >= cells.p_min - 1e-9)
    assert np.max(box.p_min - cells.p_min) > 1e-6     # and it does, somewhere
