// sound_fp32.cuh -- FP32 arithmetic that rounds outward, for the FP32-sound path.
//
// Every function returns a bound that provably brackets the exact real value
// of the quantity it names, given:
//   * IEEE FP32 directed-rounding intrinsics (__fadd_rd/ru, __fmul_rd/ru, ...)
//     and no flush-to-zero (the library is built without --use_fast_math);
//   * bounds on the error of CUDA's single-precision error functions:
//     erff(x) within K_ERF = 2 ulp and erfcf(x) within K_ERFC = 5 ulp of the
//     exact result over every finite float argument. These are measured, not
//     assumed: the GPU test suite sweeps all 2^32 float arguments against the
//     double-precision functions (largest errors seen with CUDA 13.0 on
//     sm_103a: erff 1.04 ulp, erfcf 4.49 ulp) and fails if a toolkit change
//     ever exceeds them.
//
// Notation: the Gaussian factor of one dimension (Def. 2.2 restricted to a
// coordinate) is written with erf-argument units x = (edge - m) / (sigma*sqrt2):
//   T(x)  = P(w >= x*sigma*sqrt2) = erfc(x)/2          (an upper tail)
//   g     = T(ac) - T(ae)          mass of [c, e] around the mean m
#pragma once
#include <stdint.h>

#define K_ERF 2.0f
#define K_ERFC 5.0f

namespace sound {

// ulp of a non-negative finite float (2^-149 for zero and subnormals).
__device__ __forceinline__ float ulp(float y)
{
    uint32_t e = (__float_as_uint(y) >> 23) & 0xffu;
    if (e >= 24u) return __uint_as_float((e - 23u) << 23);
    if (e >= 1u) return __uint_as_float(1u << (e - 1u));
    return __uint_as_float(1u);
}

// Bound on |y - Y| when y = lib(x) is within K ulp of the exact value Y:
// K ulp of the largest value Y can take (Y may sit one binade above y).
__device__ __forceinline__ float lib_err(float y, float K)
{
    float a = fabsf(y);
    float top = __fmul_ru(a, 1.0f + 2.0f * K * 1.1920929e-7f);
    return K * ulp(top);
}

// Upper and lower bounds of T(x) = erfc(x)/2 at an exactly known float x.
// Three branches keep the absolute error near 2^-24:
//   x >= 1/2 : erfc(x)/2 directly (small tail, relative accuracy)
//   |x| < 1/2: (1 - erf(x))/2 (erf is twice as accurate as erfc near 0)
//   x <= -1/2: 1 - erfc(-x)/2
__device__ __forceinline__ float tail_hi(float x)
{
    float r;
    if (x >= 0.5f) {
        float y = erfcf(x);
        r = __fmul_ru(0.5f, __fadd_ru(y, lib_err(y, K_ERFC)));
    } else if (x > -0.5f) {
        float y = erff(x);
        float ylo = __fsub_rd(y, lib_err(y, K_ERF));
        r = __fmul_ru(0.5f, __fsub_ru(1.0f, ylo));
    } else {
        float y = erfcf(-x);
        float ylo = fmaxf(0.0f, __fsub_rd(y, lib_err(y, K_ERFC)));
        r = __fsub_ru(1.0f, __fmul_rd(0.5f, ylo));
    }
    return fminf(r, 1.0f);
}

__device__ __forceinline__ float tail_lo(float x)
{
    float r;
    if (x >= 0.5f) {
        float y = erfcf(x);
        r = __fmul_rd(0.5f, fmaxf(0.0f, __fsub_rd(y, lib_err(y, K_ERFC))));
    } else if (x > -0.5f) {
        float y = erff(x);
        float yhi = __fadd_ru(y, lib_err(y, K_ERF));
        r = __fmul_rd(0.5f, __fsub_rd(1.0f, yhi));
    } else {
        float y = erfcf(-x);
        float yhi = __fadd_ru(y, lib_err(y, K_ERFC));
        r = __fsub_rd(1.0f, __fmul_ru(0.5f, yhi));
    }
    return fmaxf(r, 0.0f);
}

// Bounds of g = T(ac) - T(ae) for ac in [acl, ach], ae in [ael, aeh], ac <= ae.
// The form is chosen so that every tail argument is (nearly) non-negative:
//   target right of m (ac >= 0):  T(ac) - T(ae)
//   target left of m  (ae <= 0):  T(-ae) - T(-ac)
//   target around m:              1 - T(-ac) - T(ae)
// Any form is a valid bound for any arguments; the choice only affects width.
__device__ __forceinline__ float mass_hi(float acl, float ach, float ael, float aeh)
{
    float r;
    if (acl >= 0.0f)
        r = __fsub_ru(tail_hi(acl), tail_lo(aeh));
    else if (aeh <= 0.0f)
        r = __fsub_ru(tail_hi(-aeh), tail_lo(-acl));
    else
        r = __fsub_ru(__fsub_ru(1.0f, tail_lo(-acl)), tail_lo(aeh));
    return fminf(fmaxf(r, 0.0f), 1.0f);
}

__device__ __forceinline__ float mass_lo(float acl, float ach, float ael, float aeh)
{
    float r;
    if (acl >= 0.0f)
        r = __fsub_rd(tail_lo(ach), tail_hi(ael));
    else if (aeh <= 0.0f)
        r = __fsub_rd(tail_lo(-ael), tail_hi(-ach));
    else
        r = __fsub_rd(__fsub_rd(1.0f, tail_hi(-ach)), tail_hi(ael));
    return fminf(fmaxf(r, 0.0f), 1.0f);
}

// Interval of alpha_i = (E_i - m) / (sigma sqrt2) for edge i = a + k of a
// dimension, from rho = (E_a - m)/(sigma sqrt2) given as an FP32 pair
// (r_hi + r_lo, from an FP64 value) and kappa = h/(sigma sqrt2) as an FP32
// pair. Small integers k make k*kappa_hi's rounding error exact (fma), the
// sum that cancels (k*kappa + rho near 0) is formed in FP32 with its rounding
// error accounted for, and edge_err covers the gap between the grid's FP64
// edges and a + k cells of width h. Result: [al, ah] contains alpha_i.
__device__ __forceinline__ void alpha_interval(int k, float kappa_hi, float kappa_lo,
                                               float edge_err, float r_hi, float r_lo,
                                               float &al, float &ah)
{
    float kf = (float)k;
    float p = __fmul_rn(kf, kappa_hi);
    float pe = __fmaf_rn(kf, kappa_hi, -p);
    float s = __fadd_rn(p, r_hi);
    float t = __fadd_rn(pe, __fmaf_rn(kf, kappa_lo, r_lo));
    float a = __fadd_rn(s, t);
    float err = __fadd_ru(__fmul_ru(__fadd_ru(fabsf(a), fabsf(s)), 1.1920929e-7f),
                          __fadd_ru(__fmul_ru(__fadd_ru(fabsf(p), fabsf(r_hi)), 5.6843419e-14f),
                                    edge_err));
    al = __fsub_rd(a, err);
    ah = __fadd_ru(a, err);
}

// Bounds of T(x) and T(-x) over an argument interval [xm - dx, xm + dx] from
// ONE library evaluation at xm, widened by a bound on the derivative:
//   |xm| < 1/2 : erf branch, |d erf/dx| <= 2/sqrt(pi) < 1.1284
//   |xm| >= 1/2: erfc(|xm|) (the small tail) with the relative bound
//                erfc(x - dx) <= erfc(x) exp(dx (2x + 2dx + sqrt2)) for x >= 0
//                (from erfc(x) >= 2/sqrt(pi) e^{-x^2} / (x + sqrt(x^2 + 2))), and
//                exp(z) - 1 <= z (1 + z) for 0 <= z <= 1; outside z <= 1 and
//                dx < |xm| the bounds are the trivial [0, 1].
// The tail that is small keeps its relative accuracy; the other is 1 minus it.
struct TailPair {
    float p_lo, p_hi;   // T(x)
    float m_lo, m_hi;   // T(-x)
};

static __device__ __noinline__ TailPair tails(float xm, float dx)
{
    TailPair r;
    float ax = fabsf(xm);
    if (ax < 0.5f) {
        float y = erff(xm);
        float w = __fadd_ru(lib_err(y, K_ERF), __fmul_ru(1.1284f, dx));
        float ylo = fmaxf(__fsub_rd(y, w), -1.0f), yhi = fminf(__fadd_ru(y, w), 1.0f);
        r.p_hi = __fmul_ru(0.5f, __fsub_ru(1.0f, ylo));
        r.p_lo = __fmul_rd(0.5f, __fsub_rd(1.0f, yhi));
        r.m_hi = __fmul_ru(0.5f, __fadd_ru(1.0f, yhi));
        r.m_lo = __fmul_rd(0.5f, __fadd_rd(1.0f, ylo));
        return r;
    }
    float z = __fmul_ru(dx, __fadd_ru(__fmul_ru(2.0f, __fadd_ru(ax, dx)), 1.4143f));
    if (!(z <= 1.0f) || !(dx < ax)) {
        // the relative bound needs z <= 1 and an interval that stays on one
        // side of 0; wider argument intervals (never met by the callers,
        // whose dx is a few ulp) get the trivial bracket
        r.p_lo = r.m_lo = 0.0f;
        r.p_hi = r.m_hi = 1.0f;
        return r;
    }
    float y = erfcf(ax);
    float le = lib_err(y, K_ERFC);
    float rho = __fmul_ru(z, __fadd_ru(1.0f, z));
    float shi = __fmul_ru(0.5f, __fmul_ru(__fadd_ru(y, le), __fadd_ru(1.0f, rho)));
    float slo = __fmul_rd(0.5f, __fmul_rd(fmaxf(__fsub_rd(y, le), 0.0f), __fsub_rd(1.0f, rho)));
    shi = fminf(shi, 0.5f);
    float bhi = __fsub_ru(1.0f, slo), blo = __fsub_rd(1.0f, shi);
    if (xm >= 0.0f) {
        r.p_lo = slo; r.p_hi = shi; r.m_lo = blo; r.m_hi = bhi;
    } else {
        r.m_lo = slo; r.m_hi = shi; r.p_lo = blo; r.p_hi = bhi;
    }
    return r;
}

// Mass g = T(ac) - T(ae) of a target cell [c, e] from the tails of its two
// edges (c left of e), upper and lower bounds, in the form whose terms are
// the small tails: c right of the mean, e left of it, or the mean inside.
__device__ __forceinline__ float cell_hi(float ac, const TailPair &c, float ae, const TailPair &e)
{
    float r;
    if (ac >= 0.0f) r = __fsub_ru(c.p_hi, e.p_lo);
    else if (ae <= 0.0f) r = __fsub_ru(e.m_hi, c.m_lo);
    else r = __fsub_ru(__fsub_ru(1.0f, c.m_lo), e.p_lo);
    return fminf(fmaxf(r, 0.0f), 1.0f);
}

__device__ __forceinline__ float cell_lo(float ac, const TailPair &c, float ae, const TailPair &e)
{
    float r;
    if (ac >= 0.0f) r = __fsub_rd(c.p_lo, e.p_hi);
    else if (ae <= 0.0f) r = __fsub_rd(e.m_lo, c.m_hi);
    else r = __fsub_rd(__fsub_rd(1.0f, c.m_hi), e.p_hi);
    return fminf(fmaxf(r, 0.0f), 1.0f);
}

// Point estimate and half-width of alpha_i (see alpha_interval).
__device__ __forceinline__ void alpha_point(int k, float kappa_hi, float kappa_lo, float edge_err,
                                            float r_hi, float r_lo, float &a, float &err)
{
    float kf = (float)k;
    float p = __fmul_rn(kf, kappa_hi);
    float pe = __fmaf_rn(kf, kappa_hi, -p);
    float s = __fadd_rn(p, r_hi);
    float t = __fadd_rn(pe, __fmaf_rn(kf, kappa_lo, r_lo));
    a = __fadd_rn(s, t);
    err = __fadd_ru(__fmul_ru(__fadd_ru(fabsf(a), fabsf(s)), 1.1920929e-7f),
                    __fadd_ru(__fmul_ru(__fadd_ru(fabsf(p), fabsf(r_hi)), 5.6843419e-14f),
                              edge_err));
}

// Split an FP64 value into an FP32 pair hi + lo (|hi + lo - v| <= 2^-48 |v|).
__device__ __forceinline__ void split_pair(double v, float &hi, float &lo)
{
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
}

}  // namespace sound
