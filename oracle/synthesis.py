"""Plain FP64 interval-iteration synthesis on an IMDP (test infrastructure).

Only ``tests/`` and ``bench.py``'s baseline legs may use this module; the
product path never does. It shares no code with the CUDA library.

What it computes (paper: Sec. 5 and Alg. 3/4 for the serial algorithms, the
linear program of Sec. 5 solved by the sorting method of Sec. 6.2, Lemma 7 of
the cited work):

  states       the grid cells c; labels[c] in {0 free, 1 target, 2 avoid}
  rows         r = c * n_inputs + j  (the IMDP of impact_build)
  successors   of a row: its kept target cells t with [lo_t, up_t], the
               out-of-domain sink with [sink_lo, sink_up], and the truncated
               mass as one more successor with [0, trunc]
  LP (min)     min sum_s T_s v_s  s.t.  lo_s <= T_s <= up_s, sum_s T_s = 1:
               start every T_s at lo_s, then raise the successors in
               ascending order of v_s up to up_s until the sum is 1
  LP (max)     the same in descending order of v_s

  reach-avoid (Alg. 4, pessimistic policy):
    values     target 1, avoid 0, sink 0, truncated mass 0 in the min LP and
               1 in the max LP (its targets are unknown: the worst case)
    phase 1    V0 from 0, V1 from 1 on the free cells;
               V'(c) = max_j LPmin(row(c, j), V), policy(c) = argmax_j of the
               V0 update; until max |V1 - V0| <= eps;  P_min = V0
    phase 2    the policy fixed: V'(c) = LPmax(row(c, policy(c)), V);
               P_max = V1
  safety (Alg. 3, pessimistic): the same on the unsafe set (avoid cells and
               the sink, value 1; truncated mass 1 in the max LP, 0 in the
               min LP), with phase 1 V'(c) = min_j LPmax(row, V) and phase 2
               LPmin under the fixed policy; P_min = 1 - V1 of phase 1,
               P_max = 1 - V0 of phase 2 (the sound ends of each interval).

Ties in the policy take the lowest input index.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

REACH_AVOID, SAFETY = 0, 1
FREE, TARGET, AVOID = 0, 1, 2


def lp_sorted(lo, up, v, maximize: bool) -> float:
    """Optimum of sum T*v over lo <= T <= up, sum T = 1 by the sorting method."""
    lo = np.asarray(lo, np.float64)
    up = np.asarray(up, np.float64)
    v = np.asarray(v, np.float64)
    T = lo.copy()
    rest = 1.0 - T.sum()
    order = np.argsort(-v if maximize else v, kind="stable")
    for s in order:
        if rest <= 0.0:
            break
        add = min(up[s] - lo[s], rest)
        T[s] += add
        rest -= add
    return float(np.dot(T, v))


@dataclass
class SynthResult:
    p_min: np.ndarray      # float64 [cells]
    p_max: np.ndarray      # float64 [cells]
    policy: np.ndarray     # int32 [cells] (input index; 0 on target / avoid cells)
    iterations: tuple      # (phase 1, phase 2)
    converged: tuple


def _row_successors(csr, r):
    s, e = csr.row_ptr[r], csr.row_ptr[r + 1]
    return csr.col[s:e], csr.lo[s:e], csr.up[s:e]


def _row_value(csr, r, V, sink_v, trunc_v, maximize):
    col, lo, up = _row_successors(csr, r)
    lo_all = np.concatenate([lo, [csr.sink_lo[r], 0.0]])
    up_all = np.concatenate([up, [csr.sink_up[r], csr.trunc[r]]])
    v_all = np.concatenate([V[col], [sink_v, trunc_v]])
    return lp_sorted(lo_all, up_all, v_all, maximize)


def interval_iteration(csr, labels, n_inputs: int, spec: int = REACH_AVOID, eps: float = 1e-6,
                       max_iters: int = 10000) -> SynthResult:
    """Alg. 3 / Alg. 4 with the sorting-method LP. `csr` covers every row in
    order (oracle.build_rows(prob) with rows None)."""
    labels = np.asarray(labels, np.int8)
    cells = labels.shape[0]
    assert csr.row_ptr.shape[0] - 1 == cells * n_inputs
    free = labels == FREE
    if spec == REACH_AVOID:
        fixed = np.where(labels == TARGET, 1.0, 0.0)
        sink_v = 0.0
        lp1_max, pick_max = False, True     # phase 1: max_j LPmin
    else:
        fixed = np.where(labels == AVOID, 1.0, 0.0)
        sink_v = 1.0
        lp1_max, pick_max = True, False     # phase 1: min_j LPmax
    lp2_max = not lp1_max

    def trunc_value(maximize):
        return 1.0 if maximize else 0.0

    policy = np.zeros(cells, np.int32)

    def phase(lp_max, choose):
        V0 = np.where(free, 0.0, fixed)
        V1 = np.where(free, 1.0, fixed)
        it = 0
        converged = False
        while it < max_iters:
            if np.max(np.abs(V1 - V0)) <= eps:
                converged = True
                break
            N0, N1 = V0.copy(), V1.copy()
            for c in np.nonzero(free)[0]:
                if choose:
                    best0 = best1 = None
                    arg = 0
                    for j in range(n_inputs):
                        r = c * n_inputs + j
                        a = _row_value(csr, r, V0, sink_v, trunc_value(lp_max), lp_max)
                        b = _row_value(csr, r, V1, sink_v, trunc_value(lp_max), lp_max)
                        if best0 is None or (a > best0 if pick_max else a < best0):
                            best0, arg = a, j
                        if best1 is None or (b > best1 if pick_max else b < best1):
                            best1 = b
                    N0[c], N1[c] = best0, best1
                    policy[c] = arg
                else:
                    r = c * n_inputs + policy[c]
                    N0[c] = _row_value(csr, r, V0, sink_v, trunc_value(lp_max), lp_max)
                    N1[c] = _row_value(csr, r, V1, sink_v, trunc_value(lp_max), lp_max)
            V0, V1 = N0, N1
            it += 1
        return V0, V1, it, converged

    V0a, V1a, it1, ok1 = phase(lp1_max, True)
    V0b, V1b, it2, ok2 = phase(lp2_max, False)
    if spec == REACH_AVOID:
        p_min, p_max = V0a, V1b
    else:
        p_min, p_max = 1.0 - V1a, 1.0 - V0b
    return SynthResult(p_min, p_max, policy, (it1, it2), (ok1, ok2))
