"""Plain FP64 interval-iteration synthesis on an IMDP (test infrastructure).

Only ``tests/`` and ``bench.py``'s baseline legs may use this module; the
product path never does. It shares no code with the CUDA library.

What it computes (paper: Sec. 5 and Alg. 3/4 for the serial algorithms, the
linear program of Sec. 5 solved by the sorting method of Sec. 6.2, Lemma 7 of
the cited work, Remark 5.1 for a finite horizon):

  states       the grid cells c; labels[c] in {0 free, 1 target, 2 avoid}
  rows         r = (c * n_inputs + j) * n_disturb + k  (the IMDP of
               impact_build with the disturbance points as the fastest part
               of the input index)
  successors   of a row: its kept target cells t with [lo_t, up_t], the
               out-of-domain sink with [sink_lo, sink_up], and the truncated
               mass as one more successor with [0, trunc]. With region
               vectors (Sec. 3.1) the labelled cells leave the row, the sink
               too, and two successors take their place: the target region
               with [R_min, R_max] and the avoid region with [A_min, A_max]
               (A includes the sink, Remark 4.1).
  LP (min)     min sum_s T_s v_s  s.t.  lo_s <= T_s <= up_s, sum_s T_s = 1:
               start every T_s at lo_s, then raise the successors in
               ascending order of v_s up to up_s until the sum is 1
  LP (max)     the same in descending order of v_s

  values       reach-avoid (Alg. 4): the probability of satisfying the
               specification; target 1, avoid 0, sink 0.
               safety (Alg. 3): the probability of reaching the unsafe set
               (avoid cells and the sink, value 1; target cells 0); the
               result is its complement.
               The truncated mass is valued at its worst end: 0 in a min LP,
               1 in a max LP (its targets are unknown).
  players      the input maximises satisfaction (reach: max over j, safety:
               min over j of the unsafe value); the disturbance minimises it
               (reach: min over k, safety: max over k), in both phases.
  phases       the LP that bounds satisfaction from below (reach: min LP,
               safety: max LP of the unsafe value) and the one that bounds it
               from above. Phase 1 optimises the inputs with the lower-bound
               LP (pessimistic policy) or the upper-bound LP (optimistic);
               phase 2 runs the other LP with that policy fixed. Each phase
               iterates V0 (from 0 on the free cells) and V1 (from 1) until
               max |V1 - V0| <= eps; with a horizon K > 0 both start from 0
               and take exactly K steps (Remark 5.1: a for loop).
  outputs      reach: P_min = V0 of the min-LP phase, P_max = V1 of the
               max-LP phase; safety: P_min = 1 - V1 of the max-LP phase,
               P_max = 1 - V0 of the min-LP phase (the sound ends of each
               interval). The policy is the choice of phase 1 on the vector
               whose end phase 1 reports.

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


def _row_value(csr, r, V, sink_v, trunc_v, maximize, labels=None, regions=None, vals=None):
    """LP optimum of row r for the value vector V. With ``regions`` (R_min,
    R_max, A_min, A_max per row) the labelled successors are left out and the
    two regions enter with the values ``vals`` = (target, avoid)."""
    s, e = csr.row_ptr[r], csr.row_ptr[r + 1]
    col, lo, up = csr.col[s:e], csr.lo[s:e], csr.up[s:e]
    if regions is None:
        lo_all = np.concatenate([lo, [csr.sink_lo[r], 0.0]])
        up_all = np.concatenate([up, [csr.sink_up[r], csr.trunc[r]]])
        v_all = np.concatenate([V[col], [sink_v, trunc_v]])
    else:
        keep = labels[col] == FREE
        r_lo, r_up, a_lo, a_up = (x[r] for x in regions)
        lo_all = np.concatenate([lo[keep], [r_lo, a_lo, 0.0]])
        up_all = np.concatenate([up[keep], [r_up, a_up, csr.trunc[r]]])
        v_all = np.concatenate([V[col[keep]], [vals[0], vals[1], trunc_v]])
    return lp_sorted(lo_all, up_all, v_all, maximize)


def interval_iteration(csr, labels, n_inputs: int, spec: int = REACH_AVOID, eps: float = 1e-6,
                       max_iters: int = 10000, optimistic: bool = False, horizon: int = 0,
                       n_disturb: int = 1, regions=None, phase2_policy=None) -> SynthResult:
    """Alg. 3 / Alg. 4 with the sorting-method LP. `csr` covers every row in
    order (oracle.build_rows(prob) with rows None); `regions` is None or the
    four region vectors over all rows. `phase2_policy` (cells,) replaces the
    policy of phase 1 in phase 2 (the paper fixes "the" policy for the second
    bound; where inputs tie, another optimal choice is equally valid, and this
    evaluates the second bound under it)."""
    labels = np.asarray(labels, np.int8)
    cells = labels.shape[0]
    W = int(n_disturb)
    assert csr.row_ptr.shape[0] - 1 == cells * n_inputs * W
    free = labels == FREE
    reach = spec == REACH_AVOID
    if reach:
        fixed = np.where(labels == TARGET, 1.0, 0.0)
        sink_v, vals = 0.0, (1.0, 0.0)
        lower_lp_max = False           # the min LP bounds satisfaction from below
        better = lambda a, b: a > b    # inputs maximise satisfaction
        worse = lambda a, b: a < b     # disturbances minimise it
    else:
        fixed = np.where(labels == AVOID, 1.0, 0.0)
        sink_v, vals = 1.0, (0.0, 1.0)
        lower_lp_max = True            # the max LP of the unsafe value
        better = lambda a, b: a < b
        worse = lambda a, b: a > b
    lp1_max = lower_lp_max if not optimistic else not lower_lp_max
    lp2_max = not lp1_max
    # the vector whose end phase 1 reports: reach min LP -> V0, reach max LP
    # -> V1, safety max LP -> V1, safety min LP -> V0
    pol_from_v1 = lp1_max

    def value(r, V, lp_max):
        return _row_value(csr, r, V, sink_v, 1.0 if lp_max else 0.0, lp_max,
                          labels if regions is not None else None, regions, vals)

    def adversary(c, j, V, lp_max):
        best = None
        for k in range(W):
            v = value((c * n_inputs + j) * W + k, V, lp_max)
            if best is None or worse(v, best):
                best = v
        return best

    policy = np.zeros(cells, np.int32)

    def phase(lp_max, choose):
        V0 = np.where(free, 0.0, fixed)
        V1 = np.where(free, 0.0 if horizon > 0 else 1.0, fixed)
        it = 0
        converged = False
        limit = horizon if horizon > 0 else max_iters
        while it < limit:
            if horizon <= 0 and np.max(np.abs(V1 - V0)) <= eps:
                converged = True
                break
            N0, N1 = V0.copy(), V1.copy()
            for c in np.nonzero(free)[0]:
                if choose:
                    best0 = best1 = None
                    arg0 = arg1 = 0
                    for j in range(n_inputs):
                        a = adversary(c, j, V0, lp_max)
                        b = adversary(c, j, V1, lp_max)
                        if best0 is None or better(a, best0):
                            best0, arg0 = a, j
                        if best1 is None or better(b, best1):
                            best1, arg1 = b, j
                    N0[c], N1[c] = best0, best1
                    policy[c] = arg1 if pol_from_v1 else arg0
                else:
                    N0[c] = adversary(c, policy[c], V0, lp_max)
                    N1[c] = adversary(c, policy[c], V1, lp_max)
            V0, V1 = N0, N1
            it += 1
        if horizon > 0:
            converged = True
        return V0, V1, it, converged

    V0a, V1a, it1, ok1 = phase(lp1_max, True)
    if phase2_policy is not None:
        policy[:] = np.where(free, np.asarray(phase2_policy, np.int32), 0)
    V0b, V1b, it2, ok2 = phase(lp2_max, False)
    # (V0, V1) of the min-LP phase and of the max-LP phase
    (mn0, mn1), (mx0, mx1) = ((V0b, V1b), (V0a, V1a)) if lp1_max else ((V0a, V1a), (V0b, V1b))
    if reach:
        p_min, p_max = mn0, mx1
    else:
        p_min, p_max = 1.0 - mx1, 1.0 - mn0
    return SynthResult(p_min, p_max, policy, (it1, it2), (ok1, ok2))
