// tree_fp32.cu -- FP32-sound construction (Def. 3.1 with outward rounding,
// Sec. 4.4 cutoff, Remark 4.1 sink) in two kernels plus the row scan:
//
//   setup_fp32  one lane per (row, dimension), the rows of a warp aligned to
//               it. From the interval image of the cell each lane finds the
//               window of target cells that can pass the cutoff and the factor
//               table of the window: U[t], an upper bound of the largest
//               Gaussian mass of target t over the image (T_max of Def. 3.1,
//               relaxed to the image box) and L[t], a lower bound of the
//               smallest (T_min). Each window edge needs one erf/erfc
//               evaluation at the image's lower end and one at its upper end;
//               neighbouring targets share them. The lanes of a row then
//               exchange their window maxima and sums by shuffles: each turns
//               its table into exact pruning thresholds, and the lane of the
//               first dimension writes the row's sink bounds and the mass of
//               the targets outside the window box.
//   tree_fp32   one warp per row. It walks the prefix tree of target cells in
//               C order: a node at depth d is a prefix (t_0..t_d) with the
//               RU-rounded running product P of its upper factors, and its
//               children that can still reach the cutoff are exactly
//               {t : TH_{d+1}[t] <= P}, a contiguous run. Nodes wait in one
//               ring buffer per level; every step works on up to 32 of them
//               (one per lane). Count pass: pairs per row, truncated mass and
//               row checks. Emit pass: the same walk, each batch's pairs
//               spread over the lanes for warp-contiguous stores.
//
// Products run left to right over the dimensions with directed rounding
// (up: round up, lo: round down) whatever the enumeration order, so every
// pair's value depends only on its own row.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "impact_desc.h"
#include "kernels.h"
#include "sound_fp32.cuh"

namespace {

constexpr int kSetupThreads = 256;
constexpr int kTreeThreadsMax = IMPACT_TREE_WARPS_MAX * 32;
constexpr int kSeg = IMPACT_TREE_SEG;      // pairs staged per leaf batch
constexpr int kHdr = IMPACT_TREE_HDR;      // bytes of per-row scalars per warp
constexpr float kTwoM44 = 5.6843419e-14f;  // 2^-44
constexpr float kGrow18 = 1.0000038147f;   // 1 + 2^-18

__device__ __forceinline__ uint32_t fastdiv(uint32_t x, uint32_t m, int s)
{
    return (__umulhi(x, m) + x) >> s;   // exact for x < 2^31 (host-built m, s)
}

// (sh, sl) += p, exactly in sh (TwoSum) with the rounding error kept in sl.
__device__ __forceinline__ void acc_pair(float &sh, float &sl, float2 p)
{
    float s = __fadd_rn(sh, p.x);
    float bb = __fsub_rn(s, sh);
    float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p.x, bb));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(e, p.y));
}

// (rh, rl) = a - (bh, bl)
__device__ __forceinline__ void sub_pair(float2 a, float bh, float bl, float &rh, float &rl)
{
    float s = __fsub_rn(a.x, bh);
    float bb = __fsub_rn(s, a.x);
    float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(-bh, bb));
    rh = s;
    rl = __fadd_rn(__fsub_rn(a.y, bl), e);
}

// Row sums of the count pass are accumulated in fixed point (units of 2^-44,
// each term rounded outward), so the totals do not depend on which lane took
// which node nor on the order: every launch shape gives the same bits. Terms
// are capped at 2^18 and sums saturate at 2^62 (2^18 in value): the sums
// bound probability masses (at most 1) or only ever prove a row sum too
// small, so a capped value keeps every use sound.
constexpr float kFix = 17592186044416.0f;            // 2^44
constexpr double kUnfix = 5.684341886080802e-14;     // 2^-44
constexpr float kTermCap = 262144.0f;                // 2^18
constexpr unsigned long long kFixMax = 1ull << 62;
__device__ __forceinline__ unsigned long long fix_up(float x)
{
    return __float2ull_ru(__fmul_ru(fminf(x, kTermCap), kFix));
}
__device__ __forceinline__ unsigned long long fix_dn(float x)
{
    return __float2ull_rd(__fmul_rd(fminf(x, kTermCap), kFix));
}
__device__ __forceinline__ void fix_add(unsigned long long &s, unsigned long long t)
{
    s = (s > kFixMax - t) ? kFixMax : s + t;
}

__device__ __forceinline__ float fpred(float x) { return nextafterf(x, 0.0f); }
__device__ __forceinline__ float fsucc(float x) { return nextafterf(x, INFINITY); }

// Smallest float y with RU(y * r) >= c (c > 0 a float, r >= 0): RU(y r) >= c
// iff y r > pred(c), and the smallest float above pred(c)/r is
// succ(RD(pred(c)/r)) whether or not that quotient is a float.
__device__ __forceinline__ float threshold(float c, float r)
{
    if (!(r > 0.0f)) return INFINITY;
    return fsucc(__fdiv_rd(fpred(c), r));
}

// Problem of a batch that owns global index x: begin[q] <= x < begin[q + 1].
__device__ __forceinline__ int find_problem(const int64_t *__restrict__ begin, int count,
                                            int64_t x)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Edge point: alpha = (E - m)/(sigma sqrt2) at one image end, and its tails.
struct EdgePt {
    float a, da;
    sound::TailPair t;
};

struct RhoPair {
    float kh, kl, err, rh, rl;
    __device__ __forceinline__ EdgePt at(int k) const
    {
        EdgePt e;
        sound::alpha_point(k, kh, kl, err, rh, rl, e.a, e.da);
        e.t = sound::tails(e.a, e.da);
        return e;
    }
};

// The target midpoint lies at or below / at or above the mean, certainly.
__device__ __forceinline__ bool mid_below(const EdgePt &c, const EdgePt &e)
{
    return __fadd_ru(__fadd_ru(c.a, c.da), __fadd_ru(e.a, e.da)) <= 0.0f;
}
__device__ __forceinline__ bool mid_above(const EdgePt &c, const EdgePt &e)
{
    return __fadd_rd(__fsub_rd(c.a, c.da), __fsub_rd(e.a, e.da)) >= 0.0f;
}

// Everything of one (row, dimension) that needs no other dimension: the
// window and its factor tables U, L (written to the row record, trimmed to
// the targets that pass on their own, U made unimodal there: a running
// maximum from each end towards the peak, which only raises upper bounds),
// the mass outside the trimmed window and the out-of-domain bounds.
struct DimOut {
    int a = 0;          // first window cell
    int tw = 0, f0 = 0, pk = 0;   // trimmed width, its first index, peak index
    float M = 0.0f;     // largest U
    float SW = 0.0f;    // sum of U over the trimmed window (rounded up)
    float O = 0.0f;     // mass outside the trimmed window (rounded up)
    float qlo = 0.0f, qhi = 0.0f;   // out-of-domain mass bounds
};

__device__ DimOut dim_table(const ImpactDesc &D, unsigned char *rr, int64_t row, int d,
                            uint32_t *status)
{
    DimOut o;
    const int n = D.n;
    const float cut = D.cutoff32;
    // row -> (cell digits, input)
    int64_t cell;
    int j;
    if (row < ((int64_t)1 << 31)) {
        uint32_t c = fastdiv((uint32_t)row, D.inp_div_m, D.inp_div_s);
        cell = c;
        j = (int)((uint32_t)row - c * (uint32_t)D.n_inputs);
    } else {
        cell = row / D.n_inputs;
        j = (int)(row - cell * D.n_inputs);
    }
    int idx[IMPACT_MAX_DIM];
    {
        uint32_t c = (uint32_t)cell;
#pragma unroll
        for (int k = IMPACT_MAX_DIM - 1; k >= 0; --k) {
            if (k < n) {
                uint32_t q = fastdiv(c, D.dim[k].div_m, D.dim[k].div_s);
                idx[k] = (int)(c - q * (uint32_t)D.dim[k].N);
                c = q;
            }
        }
    }
    int my_idx = 0;
#pragma unroll
    for (int k = 0; k < IMPACT_MAX_DIM; ++k)
        if (k == d) my_idx = idx[k];
    const ImpactDim &g = D.dim[d];

    // image of dimension d: window estimate (cells) and, in erf units,
    // rho = (E_a - m)/(sigma sqrt2) at m_lo and m_hi as FP32 pairs
    float mulo = 0.0f, muhi = 0.0f;
    float m0h = 0.0f, m0l = 0.0f, m1h = 0.0f, m1l = 0.0f, mag = 0.0f;
    double dmlo = 0.0, dmhi = 0.0;
    if (D.kind == KIND_AFFINE) {
#pragma unroll
        for (int k = 0; k < IMPACT_MAX_DIM; ++k) {
            if (k < n) {
                int t = (d * n + k) * D.n_max + idx[k];
                mulo += D.mu_lo[t];
                muhi += D.mu_hi[t];
                float2 pl = D.ta_lo[t], ph = D.ta_hi[t];
                acc_pair(m0h, m0l, pl);
                acc_pair(m1h, m1l, ph);
                mag += fabsf(pl.x) + fabsf(ph.x);
            }
        }
        float2 o = D.oa[j * n + d];
        acc_pair(m0h, m0l, o);
        acc_pair(m1h, m1l, o);
        mag += 2.0f * fabsf(o.x);
        float mo = D.mo[j * n + d];
        mulo += mo;
        muhi += mo;
    } else if (D.kind == KIND_UNICYCLE) {
        const float2 *ea = D.ea + g.edge_off;
        float2 xlo = ea[my_idx], xhi = ea[my_idx + 1];
        acc_pair(m0h, m0l, xlo);
        acc_pair(m1h, m1l, xhi);
        float2 vl, vh;
        float cl, ch;
        if (d == 2) {
            vl = vh = D.oma[j];
            cl = ch = D.omm[j];
        } else {
            int t = (idx[2] * D.n_inputs + j) * 4 + 2 * d;
            vl = D.ua[t];
            vh = D.ua[t + 1];
            cl = D.um[t];
            ch = D.um[t + 1];
        }
        acc_pair(m0h, m0l, vl);
        acc_pair(m1h, m1l, vh);
        mag += fabsf(xlo.x) + fabsf(xhi.x) + fabsf(vl.x) + fabsf(vh.x);
        mulo = (float)my_idx + cl;
        muhi = (float)(my_idx + 1) + ch;
    } else {
        const double *im = D.images + (row * n + d) * 2;
        dmlo = im[0];
        dmhi = im[1];
        mulo = (float)((dmlo - g.lo) * g.inv_h);
        muhi = (float)((dmhi - g.lo) * g.inv_h);
    }
    // conservative window [a, a + W): every target outside has U below
    // the cutoff (its cell lies more than delta beyond the image)
    const float dc = g.delta_cells;
    float xa = floorf(mulo - dc - 1e-3f - 1e-5f * fabsf(mulo));
    float xb = floorf(muhi + dc + 1e-3f + 1e-5f * fabsf(muhi));
    const float top = (float)(g.N - 1);
    xa = fminf(fmaxf(xa, 0.0f), top);
    xb = fminf(fmaxf(xb, 0.0f), top);
    const int a = (int)xa;
    const int W = max((int)xb - a + 1, 1);
    o.a = a;
    if (W > g.wcap) {
        atomicOr(status, IMPACT_STATUS_TABLE_OVERFLOW);
        return o;
    }
    RhoPair R0, R1;
    {
        float2 ea = D.ea[g.edge_off + a];
        if (D.kind == KIND_IMAGES) {
            const double Ea = D.edges[g.edge_off + a];
            sound::split_pair((Ea - dmlo) * g.inv_s, R0.rh, R0.rl);
            sound::split_pair((Ea - dmhi) * g.inv_s, R1.rh, R1.rl);
            mag = (float)((fabs(Ea) + fabs(dmlo) + fabs(dmhi)) * g.inv_s);
        } else {
            sub_pair(ea, m0h, m0l, R0.rh, R0.rl);
            sub_pair(ea, m1h, m1l, R1.rh, R1.rl);
            mag += fabsf(ea.x);
        }
        R0.kh = R1.kh = g.kappa_hi;
        R0.kl = R1.kl = g.kappa_lo;
        R0.err = R1.err = __fadd_ru(g.edge_err, __fmul_ru(__fmul_ru(mag, 4.0f), kTwoM44));
    }

    // factor table of the window: U[k], L[k] for target a + k
    float *RU = reinterpret_cast<float *>(rr + 48 * n) + g.rec_off;
    float *RL = RU + D.tsum_cap;
    EdgePt c0 = R0.at(0), c1 = R1.at(0);
    const EdgePt w0 = c0;   // edge a at m_lo (left tail below)
    int first = -1, last = -1;
    float pre = 0.0f, mid = 0.0f, post = 0.0f;
    for (int k = 0; k < W; ++k) {
        EdgePt e0 = R0.at(k + 1), e1 = R1.at(k + 1);
        float U, L;
        if (mid_below(c0, e0)) {            // target midpoint <= m_lo
            U = sound::cell_hi(c0.a, c0.t, e0.a, e0.t);
            L = sound::cell_lo(c1.a, c1.t, e1.a, e1.t);
        } else if (mid_above(c1, e1)) {     // target midpoint >= m_hi
            U = sound::cell_hi(c1.a, c1.t, e1.a, e1.t);
            L = sound::cell_lo(c0.a, c0.t, e0.a, e0.t);
        } else {                            // midpoint may be inside
            U = g.plateau_hi;
            L = fminf(sound::cell_lo(c0.a, c0.t, e0.a, e0.t),
                      sound::cell_lo(c1.a, c1.t, e1.a, e1.t));
        }
        RU[k] = U;
        RL[k] = L;
        if (U >= cut) {
            if (first < 0) {
                first = k;
                mid = U;
            } else {
                mid = __fadd_ru(mid, __fadd_ru(post, U));
                post = 0.0f;
            }
            last = k;
        } else if (first < 0) {
            pre = __fadd_ru(pre, U);
        } else {
            post = __fadd_ru(post, U);
        }
        c0 = e0;
        c1 = e1;
    }
    // c1 is now edge a + W at m_hi
    float O = __fadd_ru(pre, post);
    const EdgePt lo0 = R0.at(-a), hi0 = R0.at(g.N - a);   // domain edges at m_lo
    const EdgePt lo1 = R1.at(-a), hi1 = R1.at(g.N - a);   // domain edges at m_hi
    if (a > 0)   // cells 0..a-1 lie left of the image: their mass at m_lo
        O = __fadd_ru(O, sound::cell_hi(lo0.a, lo0.t, w0.a, w0.t));
    if (a + W < g.N)   // cells right of the window: their mass at m_hi
        O = __fadd_ru(O, sound::cell_hi(c1.a, c1.t, hi1.a, hi1.t));
    // out-of-domain mass Q(m) = T(-alpha(lo_D)) + T(alpha(hi_D))
    float q0 = __fadd_ru(lo0.t.m_hi, hi0.t.p_hi);
    float q1 = __fadd_ru(lo1.t.m_hi, hi1.t.p_hi);
    float qhi = fminf(fmaxf(q0, q1), 1.0f);
    float qlo;
    if (mid_below(lo0, hi0))
        qlo = __fadd_rd(lo0.t.m_lo, hi0.t.p_lo);
    else if (mid_above(lo1, hi1))
        qlo = __fadd_rd(lo1.t.m_lo, hi1.t.p_lo);
    else
        qlo = g.qmin_lo;
    qlo = fminf(qlo, 1.0f);
    const int tw = first >= 0 ? last - first + 1 : 0;
    const int f0 = first >= 0 ? first : 0;
    // unimodal envelope of U on the trimmed window (running maximum from
    // each end towards the peak); raw U is unimodal up to rounding, so
    // this rarely changes a value, and it only raises upper bounds
    int pk = 0;
    float M = 0.0f;
    if (tw > 0) {
        float *u = RU + f0;
        for (int t = 0; t < tw; ++t)
            if (u[t] > M) { M = u[t]; pk = t; }
        float run = u[0];
        for (int t = 1; t < pk; ++t) {
            float v = u[t];
            if (v < run) u[t] = run; else run = v;
        }
        run = u[tw - 1];
        for (int t = tw - 2; t > pk; --t) {
            float v = u[t];
            if (v < run) u[t] = run; else run = v;
        }
    }
    o.tw = tw;
    o.f0 = f0;
    o.pk = pk;
    o.M = M;
    o.SW = mid;
    o.O = O;
    o.qlo = qlo;
    o.qhi = qhi;
    return o;
}

// setup_fp32: one warp per 32/n rows of one build, one lane per (row,
// dimension). Each lane builds its dimension's tables (dim_table); the lanes
// of a row then exchange their maxima and window sums by shuffles and each
// finishes its dimension: the pruning thresholds (a child t of a node with
// product P survives iff RU(RU(P U_d[t]) R') >= cutoff, R' bounding the
// product of the later dimensions' largest factors; TH_d[t] is the least such
// P) and the header. The lane of dimension 0 also writes the row's sink
// bounds and the mass of the targets outside the window box (FP64, outward
// rounding), unless the row outputs are null (records rebuilt for an emit).
__global__ void __launch_bounds__(kSetupThreads, 3)
setup_fp32(const BatchIndex *__restrict__ B, uint32_t *__restrict__ status,
           double *__restrict__ sink_lo, double *__restrict__ sink_up, double *__restrict__ trunc)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp0; u < B->units; u += nwarps) {
        const int q = find_problem(B->unit_begin, B->count, u);
        const ImpactDesc &D = *B->desc[q];
        const int n = D.n;
        const int rpw = 32 / n;
        const int slot = lane / n, d = lane - slot * n;
        const int64_t rows_q = B->row_begin[q + 1] - B->row_begin[q];
        const int64_t rl = (u - B->unit_begin[q]) * rpw + slot;
        const bool act = slot < rpw && rl < rows_q;
        unsigned char *rr = act ? B->rec[q] + rl * (int64_t)D.rec_stride : nullptr;
        DimOut o;
        if (act) o = dim_table(D, rr, rl, d, status);
        // the row's other dimensions, in order k = 0..n-1 (lanes base + k)
        const int base = slot * n;
        float R = 1.0f, SR = 1.0f;
        double pin_up = 1.0, pin_dn = 1.0, acc = 0.0, pre = 1.0;
#pragma unroll
        for (int k = 0; k < IMPACT_MAX_DIM; ++k) {
            if (k < n) {   // n is the same for the whole warp
                const int src = (base + k) & 31;
                const float Mk = __shfl_sync(0xffffffffu, o.M, src);
                const float SWk = __shfl_sync(0xffffffffu, o.SW, src);
                const float Ok = __shfl_sync(0xffffffffu, o.O, src);
                const float qlk = __shfl_sync(0xffffffffu, o.qlo, src);
                const float qhk = __shfl_sync(0xffffffffu, o.qhi, src);
                if (k > d) {
                    R = __fmul_ru(R, Mk);
                    SR = __fmul_ru(SR, SWk);
                }
                // sink: 1 - prod_k (1 - Q_k)
                pin_up = __dmul_ru(pin_up, __dsub_ru(1.0, (double)qlk));
                pin_dn = __dmul_rd(pin_dn, __dsub_rd(1.0, (double)qhk));
                // mass outside the window box, partitioned by the first
                // dimension that leaves its window:
                // sum_k prod_{i<k} SW_i * O_k * prod_{i>k} (SW_i + O_i)
                acc = acc * ((double)SWk + (double)Ok) + pre * (double)Ok;
                pre *= (double)SWk;
            }
        }
        if (!act) continue;
        const float cut = D.cutoff32;
        float cp = 0.0f;
        if (cut > 0.0f) cp = (d == n - 1) ? cut : threshold(cut, __fmul_ru(R, kGrow18));
        const float *RUt = reinterpret_cast<const float *>(rr + 48 * n) + D.dim[d].rec_off + o.f0;
        float *RT = reinterpret_cast<float *>(rr + 48 * n) + 2 * D.tsum_cap + D.dim[d].rec_off + o.f0;
        for (int t = 0; t < o.tw; ++t) RT[t] = cp > 0.0f ? threshold(cp, RUt[t]) : 0.0f;
        reinterpret_cast<int4 *>(rr)[3 * d] = make_int4(o.a + o.f0, o.tw, o.f0, o.pk);
        reinterpret_cast<float4 *>(rr)[3 * d + 1] = make_float4(o.SW, o.O, o.qlo, o.qhi);
        reinterpret_cast<float4 *>(rr)[3 * d + 2] = make_float4(o.M, cp, SR, 0.0f);
        if (d == 0 && trunc) {
            const int64_t row = B->row_begin[q] + rl;   // global row
            sink_lo[row] = fmax(__dsub_rd(1.0, pin_up), 0.0);
            sink_up[row] = fmin(__dsub_ru(1.0, pin_dn), 1.0);
            trunc[row] = acc * (1.0 + 1e-12);
        }
    }
}

// ---------------------------------------------------------------------------
// the prefix-tree walk
// ---------------------------------------------------------------------------

// Per-warp shared memory: a header of per-row scalars, then (entries)
//   U, L, T                      3 * tcap      factor tables, thresholds
//   npu, npl, ncol               3 * pool      node rings of all levels
// and, count pass:
//   pu_up, pu_dn, pl_up, pl_dn   4 * (tcap+8)  prefix sums
//   su_up                        (tcap+8)      suffix sums of U
// or, emit pass:
//   bq (32 float4) + seg (kSeg bytes)          leaf runs of one batch
struct Hdr {
    int ta[IMPACT_MAX_DIM], tw[IMPACT_MAX_DIM], pk[IMPACT_MAX_DIM], toff[IMPACT_MAX_DIM];
    float swr[IMPACT_MAX_DIM];
};
static_assert(sizeof(Hdr) <= kHdr, "row header does not fit");

constexpr int kEmitStageBytes = 32 * 16 + kSeg;

struct Smem {
    Hdr *h;
    float *U, *L, *T, *pu_up, *pu_dn, *pl_up, *pl_dn, *su_up, *npu, *npl;
    int *ncol;
    float4 *bq;
    unsigned char *seg;
};

template <bool EMIT>
__device__ __forceinline__ Smem carve(unsigned char *base, int tcap, int pool)
{
    Smem S;
    S.h = reinterpret_cast<Hdr *>(base);
    float *f = reinterpret_cast<float *>(base + kHdr);
    S.U = f; f += tcap;
    S.L = f; f += tcap;
    S.T = f; f += tcap;
    S.npu = f; f += pool;
    S.npl = f; f += pool;
    S.ncol = reinterpret_cast<int *>(f); f += pool;
    S.pu_up = S.pu_dn = S.pl_up = S.pl_dn = S.su_up = nullptr;
    S.bq = nullptr;
    S.seg = nullptr;
    if (!EMIT) {
        const int tp = tcap + IMPACT_MAX_DIM;
        S.pu_up = f; f += tp;
        S.pu_dn = f; f += tp;
        S.pl_up = f; f += tp;
        S.pl_dn = f; f += tp;
        S.su_up = f; f += tp;
    } else {
        unsigned char *q = reinterpret_cast<unsigned char *>(((uintptr_t)f + 15) & ~(uintptr_t)15);
        S.bq = reinterpret_cast<float4 *>(q);
        S.seg = q + 32 * 16;
    }
    return S;
}

__device__ __forceinline__ int warp_excl_scan(int v, int &total)
{
    const int lane = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// Run of dimension `dim` kept under a node with product P: [l, l + c).
// TH is non-increasing up to the peak and non-decreasing after it.
// Both ends by binary lifting (the trip counts depend on the row only, so the
// lanes stay converged): the left end is the first t <= pk with T[t] <= P, the
// right end the last t > pk with T[t] <= P.
__device__ __forceinline__ void run_of(const Smem &S, int dim, float P, int &l, int &c)
{
    const int off = S.h->toff[dim], pk = S.h->pk[dim], tw = S.h->tw[dim];
    const float *T = S.T + off;
    int a = pk + 1;
    for (int st = 1 << (31 - __clz(pk + 1)); st > 0; st >>= 1)
        if (a - st >= 0 && T[a - st] <= P) a -= st;
    int b = pk;
    if (tw - pk - 1 > 0)
        for (int st = 1 << (31 - __clz(tw - pk - 1)); st > 0; st >>= 1)
            if (b + st < tw && T[b + st] <= P) b += st;
    c = a <= pk ? b - a + 1 : 0;
    l = a;
}

// The same run, moved from the previous run [l, r) of the dimension under
// another product: the boundaries only step outwards while they still pass
// and inwards while they fail (T is monotone on each side of the peak), so a
// sequence of products that rises and falls costs O(window) steps in all.
// An empty run is l = r = pk + 1.
__device__ __forceinline__ void run_step(const Smem &S, int dim, float P, int &l, int &r)
{
    const int off = S.h->toff[dim], pk = S.h->pk[dim], tw = S.h->tw[dim];
    const float *T = S.T + off;
    while (l > 0 && T[l - 1] <= P) --l;
    while (l <= pk && T[l] > P) ++l;
    while (r < tw && T[r] <= P) ++r;
    while (r > pk + 1 && T[r - 1] > P) --r;
    if (l > pk) r = pk + 1;
}

// Upper bound of the sum of U over the window of `dim` outside [l, l + c):
// a prefix sum plus a suffix sum, both rounded up (no cancellation).
__device__ __forceinline__ float outside_sum(const Smem &S, int dim, int l, int c)
{
    const int po = S.h->toff[dim] + dim, tw = S.h->tw[dim];
    if (c == 0) return S.pu_up[po + tw];
    return __fadd_ru(S.pu_up[po + l], S.su_up[po + l + c]);
}

template <bool EMIT>
__global__ void __launch_bounds__(kTreeThreadsMax)
tree_fp32(const BatchIndex *__restrict__ B, int warp_smem, int64_t *__restrict__ row_ptr,
          int32_t *__restrict__ out_col, float *__restrict__ out_lo, float *__restrict__ out_up,
          double *__restrict__ sink_lo, double *__restrict__ sink_up,
          double *__restrict__ trunc, uint32_t *__restrict__ flags, uint32_t *__restrict__ status,
          int64_t capacity, int64_t total_at)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    unsigned char *const smem_warp = smem_raw + (size_t)(threadIdx.x >> 5) * warp_smem;
    if (EMIT && capacity >= 0 && row_ptr[total_at] > capacity) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(status, IMPACT_STATUS_CAPACITY);
        return;
    }
    unsigned long long *const next_row = B->next_row + (EMIT ? 1 : 0);

    // persistent: each warp takes the next row of the batch until none is left
    while (true) {
        unsigned long long taken = 0;
        if (lane == 0) taken = atomicAdd(next_row, 1ull);
        taken = __shfl_sync(0xffffffffu, taken, 0);
        if (taken >= (unsigned long long)B->rows) break;
        const int64_t row = (int64_t)taken;   // global row of the batch
        const int q = find_problem(B->row_begin, B->count, row);
        const ImpactDesc &D = *B->desc[q];
        const int n = D.n;
        const int tcap = D.tsum_cap;
        const int pool = D.pool_cap[EMIT ? 1 : 0];
        const Smem S = carve<EMIT>(smem_warp, tcap, pool);
        Hdr &H = *S.h;
        // the last dimensions: 1 leaf batches, 2 two dimensions serially per
        // lane (count pass), 3 two dimensions lane-parallel
        const int K = D.tree_k[EMIT ? 1 : 0];
        const int Lp = n - 1 - (K == 1 ? 1 : 2);   // level of the batch parents (-1: the root)
        const unsigned char *rr = B->rec[q] + (row - B->row_begin[q]) * (int64_t)D.rec_stride;
        // 1. the row record: per-dimension scalars, and the U, L, T tables
        // copied whole in the record's own layout (U, L, T of tcap entries
        // each, dimension k at rec_off[k]), so that every load of the row is
        // issued at once; dimension k's trimmed window starts at
        // rec_off[k] + first[k]. The record is 16-byte aligned (the workspace
        // is 256-byte aligned and the stride a multiple of 16).
        if (lane < n) {
            const int4 hi = reinterpret_cast<const int4 *>(rr)[3 * lane];
            const float4 hc = reinterpret_cast<const float4 *>(rr)[3 * lane + 2];
            H.ta[lane] = hi.x;
            H.tw[lane] = hi.y;
            H.toff[lane] = D.dim[lane].rec_off + hi.z;
            H.pk[lane] = hi.w;
            H.swr[lane] = hc.z;
        }
        {
            const int nf = 3 * tcap, n4 = nf >> 2;
            const float4 *src4 = reinterpret_cast<const float4 *>(rr + 48 * n);
            float4 *dst4 = reinterpret_cast<float4 *>(S.U);
            for (int i = lane; i < n4; i += 32) dst4[i] = src4[i];
            const float *src = reinterpret_cast<const float *>(rr + 48 * n);
            for (int i = 4 * n4 + lane; i < nf; i += 32) S.U[i] = src[i];
        }
        __syncwarp();
        bool empty = false;
        for (int k = 0; k < n; ++k) empty |= (H.tw[k] == 0);
        if (!EMIT && lane < n) {   // prefix and suffix sums of U and L per dimension
            const int off = H.toff[lane], po = off + lane, tw = H.tw[lane];
            float a = 0.0f, b = 0.0f, c = 0.0f, e = 0.0f;
            S.pu_up[po] = 0.0f;
            S.pu_dn[po] = 0.0f;
            S.pl_up[po] = 0.0f;
            S.pl_dn[po] = 0.0f;
            for (int t = 0; t < tw; ++t) {
                const float ut = S.U[off + t], lt = S.L[off + t];
                a = __fadd_ru(a, ut);
                b = __fadd_rd(b, ut);
                c = __fadd_ru(c, lt);
                e = __fadd_rd(e, lt);
                S.pu_up[po + t + 1] = a;
                S.pu_dn[po + t + 1] = b;
                S.pl_up[po + t + 1] = c;
                S.pl_dn[po + t + 1] = e;
            }
            float z = 0.0f;
            S.su_up[po + tw] = 0.0f;
            for (int t = tw - 1; t >= 0; --t) {
                z = __fadd_ru(z, S.U[off + t]);
                S.su_up[po + t] = z;
            }
        }
        __syncwarp();

        unsigned long long drop = 0, sup = 0, slo = 0;   // count pass, per lane (fixed point)
        int cnt = 0;
        int64_t out_base = 0, out_end = 0, written = 0;
        if (EMIT) {
            out_base = row_ptr[row];
            out_end = row_ptr[row + 1];
        }
        // count-pass bookkeeping of one leaf run [l, l + c) under P (dim dl)
        auto leaf_sums = [&](int dl, float P, float Pl, int l, int c) {
            const int po = H.toff[dl] + dl;
            cnt += c;
            if (c > 0) {
                float su = fmaxf(__fsub_ru(S.pu_up[po + l + c], S.pu_dn[po + l]), 0.0f);
                float sl = fmaxf(__fsub_rd(S.pl_dn[po + l + c], S.pl_up[po + l]), 0.0f);
                fix_add(sup, fix_up(__fmul_ru(P, su)));
                fix_add(slo, fix_dn(__fmul_rd(Pl, sl)));
            }
            fix_add(drop, fix_up(__fmul_ru(P, outside_sum(S, dl, l, c))));
        };

        // K = 1: each active lane's parent (P, Pl, cb) owns one run of the
        // last dimension; emit spreads the batch's pairs over the lanes
        auto leaf_batch = [&](bool act, float P, float Pl, int cb) {
            const int dl = n - 1;
            int l = 0, c = 0;
            if (act) run_of(S, dl, P, l, c);
            if (!EMIT) {
                if (act) leaf_sums(dl, P, Pl, l, c);
            } else {
                int C;
                const int o = warp_excl_scan(c, C);
                S.bq[lane] = make_float4(P, Pl, __int_as_float(cb + H.ta[dl]),
                                         __int_as_float(l - o));
                for (int k = 0; k < c; ++k) S.seg[o + k] = (unsigned char)lane;
                __syncwarp();
                const float *U = S.U + H.toff[dl];
                const float *L = S.L + H.toff[dl];
                for (int e = lane; e < C; e += 32) {
                    const float4 q = S.bq[S.seg[e]];
                    const int t = e + __float_as_int(q.w);
                    const int64_t pos = out_base + written + e;
                    if (pos < out_end) {
                        out_col[pos] = __float_as_int(q.z) + t;
                        out_lo[pos] = __fmul_rd(q.y, L[t]);
                        out_up[pos] = __fmul_ru(q.x, U[t]);
                    }
                }
                written += C;
                __syncwarp();
            }
        };

        // K = 2 (count pass): each active lane's parent owns the subtree of
        // the last two dimensions, a run of the middle dimension with a leaf
        // run under each of its nodes, walked serially by the lane
        auto block_batch = [&](bool act, float P, float Pl) {
            const int dm = n - 2, dl = n - 1;
            const int offm = H.toff[dm];
            int lm = 0, cm = 0;
            if (act) run_of(S, dm, P, lm, cm);
            if (act) {
                fix_add(drop, fix_up(__fmul_ru(__fmul_ru(P, outside_sum(S, dm, lm, cm)), H.swr[dm])));
                // the middle run's products rise to its peak and fall after it:
                // the leaf runs follow them incrementally
                int l1 = H.pk[dl] + 1, r1 = l1;
                for (int i = 0; i < cm; ++i) {
                    const int m = lm + i;
                    const float P2 = __fmul_ru(P, S.U[offm + m]);
                    const float Pl2 = __fmul_rd(Pl, S.L[offm + m]);
                    run_step(S, dl, P2, l1, r1);
                    leaf_sums(dl, P2, Pl2, l1, r1 - l1);
                }
            }
        };

        // K = 3: the last two dimensions lane-parallel. Each active lane's
        // parent owns a run of the middle dimension; the runs' nodes are
        // numbered across the warp and taken in groups of one per lane (the
        // owner of node e is the last lane whose first node is at or before
        // e), and each group is a leaf batch. Same terms as K = 1, without
        // queueing the middle nodes in a ring.
        auto pair_batch = [&](bool act, float P, float Pl, int cb, int LB) {
            const int dm = n - 2;
            const int offm = H.toff[dm], stm = D.dim[dm].stride, tam = H.ta[dm];
            int lm = 0, cm = 0;
            if (act) run_of(S, dm, P, lm, cm);
            if (!EMIT && act)
                fix_add(drop, fix_up(__fmul_ru(__fmul_ru(P, outside_sum(S, dm, lm, cm)), H.swr[dm])));
            int C1;
            const int o = warp_excl_scan(cm, C1);
            for (int base = 0; base < C1; base += LB) {
                const int e = base + lane;
                const bool a2 = lane < LB && e < C1;
                int owner = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int oc = __shfl_sync(0xffffffffu, o, owner + step);
                    if (oc <= e) owner += step;
                }
                const float Po = __shfl_sync(0xffffffffu, P, owner);
                const float Plo = __shfl_sync(0xffffffffu, Pl, owner);
                const int cbo = __shfl_sync(0xffffffffu, cb, owner);
                const int lmo = __shfl_sync(0xffffffffu, lm, owner);
                const int oo = __shfl_sync(0xffffffffu, o, owner);
                float P2 = 0.0f, Pl2 = 0.0f;
                int cb2 = 0;
                if (a2) {
                    const int m = lmo + (e - oo);
                    P2 = __fmul_ru(Po, S.U[offm + m]);
                    Pl2 = __fmul_rd(Plo, S.L[offm + m]);
                    cb2 = cbo + (tam + m) * stm;
                }
                leaf_batch(a2, P2, Pl2, cb2);
            }
        };

        // The walk keeps one ring buffer of nodes per level 0..Lp (level k
        // holds prefixes of k + 1 dimensions, in C order). Lane k keeps the
        // head and size of ring k. A step either consumes a batch of the
        // deepest ring (Lp) or expands a batch of parents of the deepest
        // other ring that has room below it; the parents taken are the
        // longest prefix of the batch whose children fit. Rings are FIFOs and
        // expansions append in order, so pairs leave in C order.
        const int pass = EMIT ? 1 : 0;
        int my_head = 0, my_size = 0;   // ring `lane`
        const int my_cap = lane < n ? (1 << D.ring_log2[pass][lane]) : 0;
        const int my_off = lane < n ? D.ring_off[pass][lane] : 0;
        const int LB = EMIT ? min(32, kSeg / max(H.tw[n - 1], 1)) : 32;
        if (!empty) {
            // every step takes at least one node off a ring (or is the root
            // step), so the nodes of levels 0..Lp bound the steps; the guard
            // only turns a broken invariant into an error instead of a hang
            int64_t guard = 2, prod = 1;
            for (int k = 0; k <= Lp; ++k) {
                prod = min(prod * H.tw[k], (int64_t)1 << 40);
                guard += 2 * prod;
            }
            bool root_pending = true;
            while (true) {
                if (--guard < 0) {
                    if (lane == 0) atomicOr(status, IMPACT_STATUS_TABLE_OVERFLOW);
                    break;
                }
                const int nxt_size = __shfl_down_sync(0xffffffffu, my_size, 1);
                const int nxt_cap = __shfl_down_sync(0xffffffffu, my_cap, 1);
                const int nxt_tw = (lane + 1 < n) ? H.tw[lane + 1] : 0;
                const unsigned up_any = __ballot_sync(0xffffffffu, lane < Lp && my_size > 0);
                const unsigned can = __ballot_sync(
                    0xffffffffu, lane < Lp && my_size > 0 && nxt_cap - nxt_size >= nxt_tw);
                const int szL = Lp >= 0 ? __shfl_sync(0xffffffffu, my_size, Lp) : 0;
                const bool more_above = up_any != 0u || root_pending;
                if (Lp >= 0 && (szL >= LB || (szL > 0 && !more_above))) {
                    // consume a batch of the deepest ring
                    const int np = min(LB, szL);
                    const int hd = __shfl_sync(0xffffffffu, my_head, Lp);
                    const int cap = __shfl_sync(0xffffffffu, my_cap, Lp);
                    const int off = __shfl_sync(0xffffffffu, my_off, Lp);
                    const bool act = lane < np;
                    const int ix = off + ((hd + lane) & (cap - 1));
                    const float P = act ? S.npu[ix] : 0.0f;
                    const float Pl = act ? S.npl[ix] : 0.0f;
                    const int cb = act ? S.ncol[ix] : 0;
                    if (K == 1)
                        leaf_batch(act, P, Pl, cb);
                    else if (K == 3)
                        pair_batch(act, P, Pl, cb, LB);
                    else
                        block_batch(act, P, Pl);
                    if (lane == Lp) {
                        my_head = (my_head + np) & (cap - 1);
                        my_size -= np;
                    }
                    continue;
                }
                int src;   // level of the parents to expand (-1: the root)
                if (can != 0u) {
                    src = 31 - __clz(can);
                } else if (root_pending) {
                    src = -1;
                    root_pending = false;
                } else {
                    break;
                }
                const int dim = src + 1;
                if (dim > Lp) {   // Lp < 0: the root is the only parent
                    if (K == 1)
                        leaf_batch(lane == 0, 1.0f, 1.0f, 0);
                    else if (K == 3)
                        pair_batch(lane == 0, 1.0f, 1.0f, 0, LB);
                    else
                        block_batch(lane == 0, 1.0f, 1.0f);
                    continue;
                }
                int np, hd = 0, scap = 1, soff = 0;
                if (src >= 0) {
                    np = min(32, __shfl_sync(0xffffffffu, my_size, src));
                    hd = __shfl_sync(0xffffffffu, my_head, src);
                    scap = __shfl_sync(0xffffffffu, my_cap, src);
                    soff = __shfl_sync(0xffffffffu, my_off, src);
                } else {
                    np = 1;
                }
                const int dsize = __shfl_sync(0xffffffffu, my_size, dim);
                const int dhead = __shfl_sync(0xffffffffu, my_head, dim);
                const int dcap = __shfl_sync(0xffffffffu, my_cap, dim);
                const int doff = __shfl_sync(0xffffffffu, my_off, dim);
                const bool act = lane < np;
                float P = 1.0f, Pl = 1.0f;
                int cb = 0;
                if (src >= 0 && act) {
                    const int ix = soff + ((hd + lane) & (scap - 1));
                    P = S.npu[ix];
                    Pl = S.npl[ix];
                    cb = S.ncol[ix];
                }
                int l = 0, c = 0;
                if (act) run_of(S, dim, P, l, c);
                int C;
                const int o = warp_excl_scan(c, C);
                const bool take = act && o + c <= dcap - dsize;
                const unsigned tk = __ballot_sync(0xffffffffu, take);
                const int nt = __popc(tk);
                if (take) {
                    const int off = H.toff[dim], st = D.dim[dim].stride, ta = H.ta[dim];
                    const int base = dhead + dsize + o;
                    for (int k = 0; k < c; ++k) {
                        const int t = l + k;
                        const int ix = doff + ((base + k) & (dcap - 1));
                        S.npu[ix] = __fmul_ru(P, S.U[off + t]);
                        S.npl[ix] = __fmul_rd(Pl, S.L[off + t]);
                        S.ncol[ix] = cb + (ta + t) * st;
                    }
                    if (!EMIT)
                        fix_add(drop, fix_up(__fmul_ru(__fmul_ru(P, outside_sum(S, dim, l, c)),
                                                       H.swr[dim])));
                }
                // children appended: the sum of the taken lanes' runs
                int added = take ? c : 0;
#pragma unroll
                for (int s2 = 16; s2 > 0; s2 >>= 1) added += __shfl_xor_sync(0xffffffffu, added, s2);
                if (lane == dim) my_size += added;
                if (src >= 0 && lane == src) {
                    my_head = (my_head + nt) & (scap - 1);
                    my_size -= nt;
                }
                __syncwarp();
            }
        }

        if (EMIT) {
            if (lane == 0 && out_base + written != out_end)
                atomicOr(status, IMPACT_STATUS_EMIT_MISMATCH);
        } else {
            unsigned long long dsum = drop, usum = sup, lsum = slo;
            long long csum = cnt;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                fix_add(dsum, __shfl_xor_sync(0xffffffffu, dsum, o));
                fix_add(usum, __shfl_xor_sync(0xffffffffu, usum, o));
                fix_add(lsum, __shfl_xor_sync(0xffffffffu, lsum, o));
                csum += __shfl_xor_sync(0xffffffffu, csum, o);
            }
            if (lane == 0) {
                const double tr = __dadd_ru(trunc[row], __ull2double_ru(dsum) * kUnfix);
                row_ptr[row] = csum;
                trunc[row] = tr;
                if (flags) {
                    // the emitted values are RU / RD products of the factors:
                    // widen the run sums by their rounding before testing
                    const double lo_sum = __ull2double_rd(lsum) * kUnfix * (1.0 - 1e-6);
                    const double up_sum = __ull2double_ru(usum) * kUnfix * (1.0 + 1e-6);
                    uint32_t f = 0;
                    if (__dadd_rd(lo_sum, sink_lo[row]) > 1.0) f |= 0x1u;
                    if (__dadd_ru(__dadd_ru(up_sum, sink_up[row]), tr) < 1.0) f |= 0x2u;
                    flags[row] = f;
                    if (f) atomicOr(status, IMPACT_STATUS_UNSOUND);
                }
            }
        }
        __syncwarp();
    }
}

int occupancy_grid(const void *kernel, int threads, size_t smem, int64_t work_items,
                   int items_per_block)
{
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem);
    if (occ < 1) occ = 1;
    int64_t want = (work_items + items_per_block - 1) / items_per_block;
    int64_t cap = (int64_t)sms * occ;
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

}  // namespace

namespace impact {

int64_t record_stride(int n, int tsum_cap)
{
    return ((int64_t)48 * n + (int64_t)12 * tsum_cap + 15) / 16 * 16;
}

int tree_smem_bytes(int tsum_cap, int pool_cap, bool emit)
{
    int64_t b = kHdr + 4 * (int64_t)(3 * tsum_cap + 3 * pool_cap);
    if (emit)
        b = (b + 15) / 16 * 16 + kEmitStageBytes;
    else
        b += 4 * (int64_t)5 * (tsum_cap + IMPACT_MAX_DIM);
    return (int)((b + 15) / 16 * 16);
}

cudaError_t launch_setup_fp32(const BatchIndex *d_index, int64_t units, uint32_t *status,
                              double *sink_lo, double *sink_up, double *trunc, cudaStream_t stream)
{
    if (units <= 0) return cudaSuccess;
    int g = occupancy_grid((const void *)setup_fp32, kSetupThreads, 0, units, kSetupThreads / 32);
    setup_fp32<<<g, kSetupThreads, 0, stream>>>(d_index, status, sink_lo, sink_up, trunc);
    return cudaGetLastError();
}

cudaError_t launch_tree_fp32(const BatchIndex *d_index, int64_t rows, int warp_smem, int warps,
                             bool emit, const RowOutputs &o, cudaStream_t stream)
{
    if (rows <= 0) return cudaSuccess;
    warps = std::max(1, std::min(warps, IMPACT_TREE_WARPS_MAX));
    const int threads = warps * 32;
    const size_t smem = (size_t)warp_smem * warps;
    const void *k = emit ? (const void *)tree_fp32<true> : (const void *)tree_fp32<false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // persistent grid: as many blocks as fit at once (rows are taken dynamically)
    int g = occupancy_grid(k, threads, smem, rows, warps);
    if (emit)
        tree_fp32<true><<<g, threads, smem, stream>>>(
            d_index, warp_smem, o.row_ptr, o.col, (float *)o.lo, (float *)o.up, o.sink_lo,
            o.sink_up, o.trunc, o.flags, o.status, o.capacity, o.total_at);
    else
        tree_fp32<false><<<g, threads, smem, stream>>>(
            d_index, warp_smem, o.row_ptr, o.col, (float *)o.lo, (float *)o.up, o.sink_lo,
            o.sink_up, o.trunc, o.flags, o.status, o.capacity, o.total_at);
    return cudaGetLastError();
}

}  // namespace impact
