"""The float identities behind the FP32 walk's pruning, checked with exact
rational arithmetic on the CPU.

The FP32-sound walk keeps a target t of a row iff the upper bound of its
transition probability (Def. 3.1, T_max of the box relaxation), formed as the
left-to-right product of per-dimension factors with every multiplication
rounded up, reaches the cutoff (Sec. 4.4). It never enumerates the pairs it
drops: a node of the prefix tree (the first d + 1 coordinates of t, with its
rounded-up running product P) is expanded only into the children that can
still reach the cutoff. Two claims make that exact and sound:

1. threshold(c, r) = succ(RD(pred(c) / r)) is the least float y with
   RU(y r) >= c, for floats c > 0 and r > 0 (or +inf when no finite y
   reaches c).
2. Growing the rounded-up product R of the later dimensions' largest factors
   by 2^-18 covers the rounding of any chain of up to seven more rounded-up
   multiplications: if RU(...RU(RU(P a_1) a_2)... a_k) >= cut with a_i <= M_i
   <= 1, then P >= threshold(cut, RU(R (1 + 2^-18))).

So no target whose rounded-up product reaches the cutoff is pruned. Neither
claim needs a GPU; the kernels' use of them is covered by the GPU parity
tests (the FP32 kept set contains the FP64 one).
"""

from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32
INF = F32(np.inf)
FMAX = F32(np.finfo(np.float32).max)
GROW18 = F32(1.0000038147)   # the literal the kernel uses for 1 + 2^-18


def ex(x) -> Fraction:
    """Exact value of a float32."""
    return Fraction(float(x))


def ru(q: Fraction):
    """Least float32 >= q (q >= 0), +inf beyond the largest float."""
    if q > ex(FMAX):
        return INF
    f = F32(float(q))
    while ex(f) < q:
        f = np.nextafter(f, INF)
    while True:
        g = np.nextafter(f, -INF)
        if g >= 0 and ex(g) >= q:
            f = g
        else:
            return f


def rd(q: Fraction):
    """Greatest float32 <= q (q >= 0); the largest float beyond it."""
    if q >= ex(FMAX):
        return FMAX
    f = F32(float(q))
    while ex(f) > q:
        f = np.nextafter(f, -INF)
    while True:
        g = np.nextafter(f, INF)
        if ex(g) <= q:
            f = g
        else:
            return f


def pred(x):
    return np.nextafter(F32(x), F32(0.0))


def succ(x):
    with np.errstate(over="ignore"):
        return np.nextafter(F32(x), INF)


def threshold(c, r):
    if not r > 0:
        return INF
    return succ(rd(ex(pred(c)) / ex(r)))


def mul_ru(a, b):
    if np.isinf(a) or np.isinf(b):
        return INF
    return ru(ex(a) * ex(b))


def log_uniform(rng, lo, hi, size):
    return F32(np.exp(rng.uniform(np.log(lo), np.log(hi), size)))


def test_grow_literal_is_one_plus_two_to_minus_18():
    assert ex(GROW18) == 1 + Fraction(1, 2 ** 18)


def threshold_cases():
    rng = np.random.default_rng(11)
    cs = list(log_uniform(rng, 1e-12, 1.0, 300))
    rs = list(log_uniform(rng, 1e-30, 2.0, 300))
    special_c = [F32(1e-8), F32(1.0), F32(np.finfo(np.float32).tiny), F32(0.5), pred(F32(1e-8))]
    special_r = [F32(1.0), pred(F32(1.0)), succ(F32(1.0)), F32(1e-38), F32(2.0 ** -149),
                 F32(0.75), F32(1e-45)]
    out = list(zip(cs, rs))
    out += [(c, r) for c in special_c for r in special_r]
    return out


def test_threshold_is_the_least_float_reaching_c():
    for c, r in threshold_cases():
        y = threshold(c, r)
        if np.isinf(y):
            # no finite float reaches c: even the largest one falls short
            assert mul_ru(FMAX, r) < c, (c, r)
            continue
        assert mul_ru(y, r) >= c, (c, r, y)
        p = pred(y)
        if y > 0:
            assert mul_ru(p, r) < c, (c, r, y)


def test_threshold_of_a_zero_factor_is_infinite():
    assert np.isinf(threshold(F32(1e-8), F32(0.0)))


def chain_ru(P, factors):
    x = P
    for a in factors:
        x = mul_ru(x, a)
    return x


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
def test_grown_product_covers_every_rounding_of_the_chain(k):
    """Whenever some completion's rounded-up product reaches the cutoff, the
    node's product P passes the threshold built from the later maxima."""
    rng = np.random.default_rng(100 + k)
    cut = F32(1e-8)
    checked = 0
    for _ in range(200):
        M = log_uniform(rng, 0.05, 1.0, k)                 # later dimensions' largest factors
        a = F32(M * F32(rng.uniform(0.3, 1.0, k)))          # a completion's factors, a_i <= M_i
        a = np.minimum(a, M)
        if rng.random() < 0.3:
            a = M.copy()                                     # the completion along the maxima
        R = F32(1.0)
        for m in M:
            R = mul_ru(R, m)
        cp = threshold(cut, mul_ru(R, GROW18))
        # node products around the least one whose chain reaches the cutoff
        exact = ex(cut)
        for x in a:
            exact /= ex(x)
        base = ru(exact)
        for step in range(-3, 4):
            P = base
            for _ in range(abs(step)):
                P = succ(P) if step > 0 else pred(P)
            if chain_ru(P, a) >= cut:
                checked += 1
                assert P >= cp, (k, P, cp, a, M)
    assert checked > 100


def test_pruning_threshold_for_the_last_dimension_is_the_cutoff():
    """With no later dimension the child survives iff RU(P U) >= cut, which is
    threshold(cut, U) <= P (claim 1 with c = cut)."""
    rng = np.random.default_rng(5)
    cut = F32(1e-8)
    for U in log_uniform(rng, 1e-9, 1.0, 200):
        th = threshold(cut, U)
        for P in (th, pred(th), succ(th)):
            if np.isinf(P):
                continue
            assert (mul_ru(P, U) >= cut) == (P >= th)


def test_growth_exceeds_seven_roundings():
    """Claim 2's margin: a rounded-up product of normal floats exceeds the
    exact one by a factor below 1 + 2^-23 per multiplication, and seven of
    them stay below the 1 + 2^-18 growth (the chain's products stay at or
    above the cutoff, far above the subnormal range, as every factor is at
    most 1)."""
    assert (1 + Fraction(1, 2 ** 23)) ** 7 < 1 + Fraction(1, 2 ** 18)
