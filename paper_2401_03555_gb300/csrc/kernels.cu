// kernels.cu -- the FP64-plain path and the row-pointer scan.
//
// FP64 plain: one warp builds one row (source cell x input) at a time (Alg. 2:
// rows are independent) and evaluates every factor of every candidate pair in
// FP64 (the comparison baseline; the FP32-sound path is in tree_fp32.cu).
// Per row:
//   1. interval image [m_lo, m_hi] of f over the cell (table lookups + sums)
//   2. per dimension, a window of target cells outside of which every upper
//      factor is below cutoff/2 (Sec. 4.4: entries whose upper bound is
//      negligible are not stored), then the per-dimension factor table
//      U_d[t] (upper, Def. 3.1 T_max relaxed) and L_d[t] (lower, T_min)
//   3. the window box is enumerated in C order: an outer prefix of
//      dimensions is pruned as a whole when even the largest remaining
//      factors cannot lift it to the cutoff, the surviving prefixes are
//      expanded over the inner dimensions, lanes test up >= cutoff and the
//      warp compacts the kept targets with ballot/popc
//   4. per-row terms: the out-of-domain sink bounds (Remark 4.1), the
//      truncated mass and the row-sum checks of Def. 3.1, combined in FP64.
// The count pass runs 1-4 without storing pairs; a scan turns the counts into
// row pointers; the emit pass repeats 1-3 and writes the CSR pairs.
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>
#include <stdint.h>

#include "impact_desc.h"
#include "kernels.h"
#include "sound_fp32.cuh"

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kThreads = kWarpsPerBlock * 32;
constexpr int kTab = IMPACT_TABLE_MAX;   // staged factor entries per row (all dims)

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Cell digits (C order) of a row, and the input index.
__device__ __forceinline__ void decode_row(const ImpactDesc &D, int64_t row, int *idx, int &j)
{
    int64_t cell = row / D.n_inputs;
    j = (int)(row - cell * D.n_inputs);
    uint32_t c = (uint32_t)cell;
#pragma unroll
    for (int d = IMPACT_MAX_DIM - 1; d >= 0; --d) {
        if (d < D.n) {
            uint32_t N = (uint32_t)D.dim[d].N;
            uint32_t q = c / N;
            idx[d] = (int)(c - q * N);
            c = q;
        }
    }
}

// Interval image of f(., u_j) over the cell in dimension d.
//   SOUND: outward-rounded bounds of the exact image.
//   plain: round-to-nearest in the same operation order as the definition
//          (sum over k of the per-term range, then the input offset).
template <bool SOUND>
__device__ __forceinline__ void image_dim(const ImpactDesc &D, int64_t row, const int *idx, int j,
                                          int d, double &mlo, double &mhi)
{
    const int n = D.n;
    if (D.kind == KIND_AFFINE) {
        const int NM = D.n_max;
        if (SOUND) {
            double slo = 0.0, shi = 0.0;
            for (int k = 0; k < n; ++k) {
                int t = (d * n + k) * NM + idx[k];
                slo = __dadd_rd(slo, D.term_dn[t]);
                shi = __dadd_ru(shi, D.term_up[t]);
            }
            mlo = __dadd_rd(slo, D.off_dn[j * n + d]);
            mhi = __dadd_ru(shi, D.off_up[j * n + d]);
        } else {
            double slo = 0.0, shi = 0.0;
            for (int k = 0; k < n; ++k) {
                int t = ((d * n + k) * NM + idx[k]) * 2;
                slo = __dadd_rn(slo, D.term_rn[t]);
                shi = __dadd_rn(shi, D.term_rn[t + 1]);
            }
            mlo = __dadd_rn(slo, D.off_rn[j * n + d]);
            mhi = __dadd_rn(shi, D.off_rn[j * n + d]);
        }
    } else if (D.kind == KIND_UNICYCLE) {
        const double *E = D.edges + D.dim[d].edge_off;
        double xlo = E[idx[d]], xhi = E[idx[d] + 1];
        if (d == 2) {
            double om = D.inputs[j * D.m + 1];
            if (SOUND) { mlo = __dadd_rd(xlo, om); mhi = __dadd_ru(xhi, om); }
            else { mlo = __dadd_rn(xlo, om); mhi = __dadd_rn(xhi, om); }
        } else {
            const double *u = (SOUND ? D.uni_sd : D.uni_rn) + ((int64_t)idx[2] * D.n_inputs + j) * 4;
            double vlo = u[d * 2 + 0], vhi = u[d * 2 + 1];
            if (SOUND) { mlo = __dadd_rd(xlo, vlo); mhi = __dadd_ru(xhi, vhi); }
            else { mlo = __dadd_rn(xlo, vlo); mhi = __dadd_rn(xhi, vhi); }
        }
    } else {
        const double *im = D.images + (row * n + d) * 2;
        mlo = im[0];
        mhi = im[1];
    }
}

// Conservative window [a, b] of target cells in dimension d: any target whose
// cell lies entirely more than delta beyond the image has every upper factor
// below cutoff/2. One extra cell of slack on each side absorbs rounding.
__device__ __forceinline__ void window_dim(const ImpactDim &g, double mlo, double mhi, int &a,
                                           int &b)
{
    if (!(g.delta < INFINITY)) {
        a = 0;
        b = g.N - 1;
        return;
    }
    double xa = floor((mlo - g.delta - g.lo) * g.inv_h) - 1.0;
    double xb = floor((mhi + g.delta - g.lo) * g.inv_h) + 1.0;
    xa = fmin(fmax(xa, 0.0), (double)(g.N - 1));
    xb = fmin(fmax(xb, 0.0), (double)(g.N - 1));
    a = (int)xa;
    b = (int)xb;
    if (b < a) b = a - 1;   // empty
}

// ---------------------------------------------------------------------------
// FP64 plain row kernel: every factor of every candidate pair in FP64
// ---------------------------------------------------------------------------

// g(c, e; m) = Phi((e-m)/sigma) - Phi((c-m)/sigma), inv_s = 1/(sigma sqrt 2).
__device__ __forceinline__ double g64(double c, double e, double m, double inv_s)
{
    double a = (c - m) * inv_s;
    double b = (e - m) * inv_s;
    if (a >= 0.0) return 0.5 * (erfc(a) - erfc(b));
    if (b <= 0.0) return 0.5 * (erfc(-b) - erfc(-a));
    return 1.0 - 0.5 * erfc(-a) - 0.5 * erfc(b);
}

__device__ __forceinline__ double clampd(double x, double lo, double hi)
{
    return x < lo ? lo : (x > hi ? hi : x);
}

// Upper factor of target cell t of dimension d.
__device__ __forceinline__ double up64(const ImpactDim &g, const double *E, int t, double mlo,
                                       double mhi)
{
    double c = E[t], e = E[t + 1];
    return g64(c, e, clampd(0.5 * (c + e), mlo, mhi), g.inv_s);
}

__device__ __forceinline__ double lo64(const ImpactDim &g, const double *E, int t, double mlo,
                                       double mhi)
{
    double c = E[t], e = E[t + 1];
    return fmin(g64(c, e, mlo, g.inv_s), g64(c, e, mhi, g.inv_s));
}

struct WarpSm64 {
    double U[kTab];
    double mlo[IMPACT_MAX_DIM], mhi[IMPACT_MAX_DIM];
    double SW[IMPACT_MAX_DIM], O[IMPACT_MAX_DIM];
    double gin_max[IMPACT_MAX_DIM], gin_min[IMPACT_MAX_DIM];
    int a[IMPACT_MAX_DIM], w[IMPACT_MAX_DIM], cum[IMPACT_MAX_DIM];
    int ta[IMPACT_MAX_DIM], tw[IMPACT_MAX_DIM];
};

template <bool EMIT>
__global__ void __launch_bounds__(kThreads)
rows_fp64(const ImpactDesc *__restrict__ Dp, int64_t row_begin, int64_t row_end,
          int64_t *__restrict__ row_ptr, int32_t *__restrict__ out_col,
          double *__restrict__ out_lo, double *__restrict__ out_up,
          double *__restrict__ sink_lo, double *__restrict__ sink_up,
          double *__restrict__ trunc, uint32_t *__restrict__ flags,
          uint32_t *__restrict__ status, int64_t capacity, int64_t total_at)
{
    __shared__ WarpSm64 sm_all[kWarpsPerBlock];
    const ImpactDesc &D = *Dp;
    const int lane = threadIdx.x & 31;
    WarpSm64 &S = sm_all[threadIdx.x >> 5];
    const int n = D.n;
    const double cut = D.cutoff;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned lt = lanemask_lt();
    if (EMIT && capacity >= 0 && row_ptr[total_at] > capacity) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(status, IMPACT_STATUS_CAPACITY);
        return;
    }

    for (int64_t row = row_begin + warp0; row < row_end; row += nwarps) {
        int idx[IMPACT_MAX_DIM];
        int j;
        decode_row(D, row, idx, j);
        if (lane < n) {
            const ImpactDim &g = D.dim[lane];
            double mlo, mhi;
            image_dim<false>(D, row, idx, j, lane, mlo, mhi);
            int a, b;
            window_dim(g, mlo, mhi, a, b);
            S.mlo[lane] = mlo;
            S.mhi[lane] = mhi;
            S.a[lane] = a;
            S.w[lane] = b - a + 1;
            if (!EMIT) {   // in-domain mass at the three points (sink)
                double mid = 0.5 * (g.lo + g.hi);
                S.gin_max[lane] = g64(g.lo, g.hi, clampd(mid, mlo, mhi), g.inv_s);
                S.gin_min[lane] = fmin(g64(g.lo, g.hi, mlo, g.inv_s), g64(g.lo, g.hi, mhi, g.inv_s));
            }
        }
        __syncwarp();
        int total = 0;
        for (int d = 0; d < n; ++d) {
            if (lane == 0) S.cum[d] = total;
            total += S.w[d];
        }
        __syncwarp();
        // upper factors of the window (used only to trim the windows and for
        // the truncated-mass sums; the pairs below recompute every factor),
        // staged when they fit, else evaluated again where they are read
        const bool staged = total <= kTab;
        if (staged) {
            for (int e = lane; e < total; e += 32) {
                int d = 0;
                while (d + 1 < n && e >= S.cum[d + 1]) ++d;
                const ImpactDim &g = D.dim[d];
                S.U[e] = up64(g, D.edges + g.edge_off, S.a[d] + e - S.cum[d], S.mlo[d], S.mhi[d]);
            }
        }
        __syncwarp();
        bool empty = false;
        for (int d = 0; d < n; ++d) {
            const int base = S.cum[d], W = S.w[d];
            const ImpactDim &gd = D.dim[d];
            auto Uw = [&](int t) {
                return staged ? S.U[base + t]
                              : up64(gd, D.edges + gd.edge_off, S.a[d] + t, S.mlo[d], S.mhi[d]);
            };
            int first = -1, last = -1;
            for (int c0 = 0; c0 < W; c0 += 32) {
                int t = c0 + lane;
                bool pass = t < W && Uw(t) >= cut;
                unsigned bal = __ballot_sync(0xffffffffu, pass);
                if (bal) {
                    if (first < 0) first = c0 + __ffs(bal) - 1;
                    last = c0 + 31 - __clz(bal);
                }
            }
            double sw = 0.0, ow = 0.0;
            for (int c0 = 0; c0 < W; c0 += 32) {
                int t = c0 + lane;
                if (t < W) {
                    double v = Uw(t);
                    if (first >= 0 && t >= first && t <= last) sw += v;
                    else ow += v;
                }
            }
            sw = warp_sum_d(sw);
            ow = warp_sum_d(ow);
            if (lane == 0) {
                const ImpactDim &g = D.dim[d];
                const double *E = D.edges + g.edge_off;
                const int a = S.a[d], b = a + W - 1;
                double O = ow;
                if (a > 0) O += g64(E[0], E[a], S.mlo[d], g.inv_s);
                if (b < g.N - 1) O += g64(E[b + 1], E[g.N], S.mhi[d], g.inv_s);
                S.O[d] = O;
                S.SW[d] = sw;
                S.ta[d] = first < 0 ? a : a + first;
                S.tw[d] = first < 0 ? 0 : last - first + 1;
            }
            empty |= (first < 0);
        }
        __syncwarp();

        double drop = 0.0, slo = 0.0, sup = 0.0;
        int64_t cnt = 0, out_base = 0, out_end = 0, written = 0;
        if (EMIT) {
            out_base = row_ptr[row];
            out_end = row_ptr[row + 1];
        }
        if (!empty) {
            int64_t K = 1;
            for (int d = 0; d < n; ++d) K *= S.tw[d];
            int tt[IMPACT_MAX_DIM], sd[IMPACT_MAX_DIM];
            uint32_t q = (uint32_t)lane, qs = 32u;
            for (int d = n - 1; d >= 0; --d) {
                uint32_t W = (uint32_t)S.tw[d];
                tt[d] = (int)(q % W);
                q /= W;
                sd[d] = (int)(qs % W);
                qs /= W;
            }
            for (int64_t kb = 0; kb < K; kb += 32) {
                bool valid = (kb + lane < K);
                bool keep = false;
                double uv = 1.0, lv = 1.0;
                int cv = 0;
                if (valid) {
                    for (int d = 0; d < n; ++d) {
                        const ImpactDim &g = D.dim[d];
                        int t = S.ta[d] + tt[d];
                        uv *= up64(g, D.edges + g.edge_off, t, S.mlo[d], S.mhi[d]);
                        cv += t * g.stride;
                    }
                    keep = uv >= cut;
                    if (keep) {
                        for (int d = 0; d < n; ++d) {
                            const ImpactDim &g = D.dim[d];
                            lv *= lo64(g, D.edges + g.edge_off, S.ta[d] + tt[d], S.mlo[d], S.mhi[d]);
                        }
                    }
                }
                unsigned bal = __ballot_sync(0xffffffffu, keep);
                if (EMIT) {
                    if (keep) {
                        int64_t p = out_base + written + __popc(bal & lt);
                        if (p < out_end) {
                            out_col[p] = cv;
                            out_lo[p] = lv;
                            out_up[p] = uv;
                        }
                    }
                    written += __popc(bal);
                } else {
                    cnt += __popc(bal);
                    if (keep) {
                        slo += lv;
                        sup += uv;
                    } else if (valid) {
                        drop += uv;
                    }
                }
                int carry = 0;
                for (int d = n - 1; d >= 0; --d) {
                    int t = tt[d] + sd[d] + carry;
                    carry = t >= S.tw[d];
                    tt[d] = carry ? t - S.tw[d] : t;
                }
            }
        }
        if (EMIT && lane == 0 && out_base + written != out_end)
            atomicOr(status, IMPACT_STATUS_EMIT_MISMATCH);
        if (!EMIT) {
            double dsum = warp_sum_d(drop);
            double lsum = warp_sum_d(slo);
            double usum = warp_sum_d(sup);
            if (lane == 0) {
                double outside = 0.0;
                for (int d = 0; d < n; ++d) {
                    double t = S.O[d];
                    for (int k = 0; k < d; ++k) t *= S.SW[k];
                    for (int k = d + 1; k < n; ++k) t *= S.SW[k] + S.O[k];
                    outside += t;
                }
                double pmax = 1.0, pmin = 1.0;
                for (int d = 0; d < n; ++d) {
                    pmax *= S.gin_max[d];
                    pmin *= S.gin_min[d];
                }
                double sl = 1.0 - pmax, su = 1.0 - pmin;
                double tr = outside + dsum;
                row_ptr[row] = cnt;
                sink_lo[row] = sl;
                sink_up[row] = su;
                trunc[row] = tr;
                if (flags) {
                    uint32_t f = 0;
                    if (lsum + sl > 1.0 + 1e-12) f |= 0x1u;
                    if (usum + su + tr < 1.0 - 1e-12) f |= 0x2u;
                    flags[row] = f;
                    if (f) atomicOr(status, IMPACT_STATUS_UNSOUND);
                }
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Exclusive scan of the per-row counts (in place in row_ptr), 3 passes.
// ---------------------------------------------------------------------------

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *sh, int64_t &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    int64_t before = (w > 0 ? sh[w - 1] : 0) + x - v;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanThreads) scan_tiles(const int64_t *__restrict__ v,
                                                           int64_t n, int64_t *__restrict__ tsum)
{
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += v[base + k];
    int64_t total;
    block_excl_scan(s, sh, total);
    if (threadIdx.x == 0) tsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_sums(int64_t *__restrict__ tsum, int64_t nt,
                                                          int64_t *__restrict__ grand)
{
    __shared__ int64_t sh[32];
    int64_t carry = 0;
    for (int64_t b = 0; b < nt; b += kScanThreads) {
        int64_t i = b + threadIdx.x;
        int64_t v = i < nt ? tsum[i] : 0;
        int64_t total;
        int64_t ex = block_excl_scan(v, sh, total);
        if (i < nt) tsum[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply(int64_t *__restrict__ v, int64_t n,
                                                           const int64_t *__restrict__ toff)
{
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t loc[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = (base + k < n) ? v[base + k] : 0;
        s += loc[k];
    }
    int64_t total;
    int64_t ex = block_excl_scan(s, sh, total) + toff[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) v[base + k] = ex;
        ex += loc[k];
    }
}

// ---------------------------------------------------------------------------
// target / avoid regions (Sec. 3.1, Alg. 1, Remark 4.1)
// ---------------------------------------------------------------------------

using impact::RegionBoxes;
using impact::RowOutputs;

__global__ void __launch_bounds__(256)
label_cells(RegionBoxes B, int64_t total, uint8_t *__restrict__ labels)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
         c += (int64_t)gridDim.x * blockDim.x) {
        int idx[IMPACT_MAX_DIM];
        int64_t rest = c;
        for (int d = B.n - 1; d >= 0; --d) {
            idx[d] = (int)(rest % B.cells[d]);
            rest /= B.cells[d];
        }
        uint8_t lab = 0;
        for (int b = 0; b < B.count; ++b) {
            bool in = true;
            for (int d = 0; d < B.n; ++d)
                in = in && idx[d] >= B.first[b][d] && idx[d] <= B.last[b][d];
            if (in) lab = b >= B.n_target ? 2 : (lab == 0 ? 1 : lab);
        }
        labels[c] = lab;
    }
}

// FP32 interval of (p - m') / (sigma sqrt2) for every m' within dm of m: the
// FP64 evaluation (relative error below 2^-49 with the rounded 1/(sigma
// sqrt2)) widened by that error and by dm, then rounded outward to FP32.
__device__ __forceinline__ void arg_iv(double p, double m, double dm, double inv_s, float &lo,
                                       float &hi)
{
    const double x = (p - m) * inv_s;
    const double w = dm * inv_s;
    const double e = (fabs(x) + w) * 0x1p-49 + w;
    lo = __double2float_rd(x - e);
    hi = __double2float_ru(x + e);
}

// Bounds of one factor g(c, e; m), the mass of [c, e] around a mean m known
// to within dm: FP64 round-to-nearest (plain), or the FP32 outward bounds of
// sound_fp32.cuh (sound).
template <bool SOUND>
__device__ __forceinline__ double g_up(double c, double e, double m, double dm, double inv_s)
{
    if (!SOUND) return g64(c, e, m, inv_s);
    float acl, ach, ael, aeh;
    arg_iv(c, m, dm, inv_s, acl, ach);
    arg_iv(e, m, dm, inv_s, ael, aeh);
    return (double)sound::mass_hi(acl, ach, ael, aeh);
}
template <bool SOUND>
__device__ __forceinline__ double g_dn(double c, double e, double m, double inv_s)
{
    if (!SOUND) return g64(c, e, m, inv_s);
    float acl, ach, ael, aeh;
    arg_iv(c, m, 0.0, inv_s, acl, ach);
    arg_iv(e, m, 0.0, inv_s, ael, aeh);
    return (double)sound::mass_lo(acl, ach, ael, aeh);
}

// Largest factor over m in [mlo, mhi] (at the clamped midpoint of [c, e],
// whose rounding dm the sound bound covers) and the smallest (at an end).
template <bool SOUND>
__device__ __forceinline__ double f_max(double c, double e, double mlo, double mhi, double inv_s)
{
    const double mid = 0.5 * (c + e);
    const double m = clampd(mid, mlo, mhi);
    const double dm = (m == mid) ? fabs(mid) * 0x1p-52 : 0.0;
    return g_up<SOUND>(c, e, m, dm, inv_s);
}
template <bool SOUND>
__device__ __forceinline__ double f_min(double c, double e, double mlo, double mhi, double inv_s)
{
    return fmin(g_dn<SOUND>(c, e, mlo, inv_s), g_dn<SOUND>(c, e, mhi, inv_s));
}

template <bool SOUND>
__device__ __forceinline__ double mul_up(double a, double b) { return SOUND ? __dmul_ru(a, b) : a * b; }
template <bool SOUND>
__device__ __forceinline__ double mul_dn(double a, double b) { return SOUND ? __dmul_rd(a, b) : a * b; }
template <bool SOUND>
__device__ __forceinline__ double add_up(double a, double b) { return SOUND ? __dadd_ru(a, b) : a + b; }
template <bool SOUND>
__device__ __forceinline__ double add_dn(double a, double b) { return SOUND ? __dadd_rd(a, b) : a + b; }

// One thread per row: the interval image, the sink (the domain box, Remark
// 4.1), then per region box the product over dimensions of either the box's
// own factor (one relaxation per box) or the sum of the per-cell factors
// over the box's cells (the paper's sums: sum over the cells of a product
// of per-dimension factors equals the product of per-dimension sums).
template <bool SOUND>
__global__ void __launch_bounds__(128)
region_rows(const ImpactDesc *__restrict__ Dp, int64_t rows, RegionBoxes B, bool cell_sum,
            double *__restrict__ r_lo, double *__restrict__ r_up, double *__restrict__ a_lo,
            double *__restrict__ a_up)
{
    const ImpactDesc &D = *Dp;
    const int n = D.n;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
         row += (int64_t)gridDim.x * blockDim.x) {
        int idx[IMPACT_MAX_DIM];
        int j;
        decode_row(D, row, idx, j);
        double mlo[IMPACT_MAX_DIM], mhi[IMPACT_MAX_DIM];
        double in_max = 1.0, in_min = 1.0;
        for (int d = 0; d < n; ++d) {
            image_dim<SOUND>(D, row, idx, j, d, mlo[d], mhi[d]);
            const ImpactDim &g = D.dim[d];
            in_max = mul_up<SOUND>(in_max, f_max<SOUND>(g.lo, g.hi, mlo[d], mhi[d], g.inv_s));
            in_min = mul_dn<SOUND>(in_min, f_min<SOUND>(g.lo, g.hi, mlo[d], mhi[d], g.inv_s));
        }
        double rl = 0.0, ru = 0.0;
        double xl = SOUND ? fmax(__dsub_rd(1.0, in_max), 0.0) : 1.0 - in_max;
        double xu = SOUND ? fmin(__dsub_ru(1.0, in_min), 1.0) : 1.0 - in_min;
        for (int b = 0; b < B.count; ++b) {
            double pu = 1.0, pl = 1.0;
            for (int d = 0; d < n; ++d) {
                const ImpactDim &g = D.dim[d];
                const double *E = D.edges + g.edge_off;
                double fu, fl;
                if (cell_sum) {
                    fu = 0.0;
                    fl = 0.0;
                    for (int i = B.first[b][d]; i <= B.last[b][d]; ++i) {
                        fu = add_up<SOUND>(fu, f_max<SOUND>(E[i], E[i + 1], mlo[d], mhi[d], g.inv_s));
                        fl = add_dn<SOUND>(fl, f_min<SOUND>(E[i], E[i + 1], mlo[d], mhi[d], g.inv_s));
                    }
                } else {
                    const double c = E[B.first[b][d]], e = E[B.last[b][d] + 1];
                    fu = f_max<SOUND>(c, e, mlo[d], mhi[d], g.inv_s);
                    fl = f_min<SOUND>(c, e, mlo[d], mhi[d], g.inv_s);
                }
                pu = mul_up<SOUND>(pu, fu);
                pl = mul_dn<SOUND>(pl, fl);
            }
            if (b < B.n_target) {
                rl = add_dn<SOUND>(rl, pl);
                ru = add_up<SOUND>(ru, pu);
            } else {
                xl = add_dn<SOUND>(xl, pl);
                xu = add_up<SOUND>(xu, pu);
            }
        }
        r_lo[row] = rl;
        r_up[row] = ru;
        a_lo[row] = xl;
        a_up[row] = xu;
    }
}

// ---------------------------------------------------------------------------
// sampled noise: Monte-Carlo integration of the cell masses (Sec. 4.1)
// ---------------------------------------------------------------------------

constexpr int kMcThreads = 256;
constexpr int kMcThr = IMPACT_MC_EDGES_MAX + 1;   // thresholds per (row, dimension, end)

// Order-preserving integer key of a finite double (-0 and +0 share key 0):
// x < y exactly when key(x) < key(y). Comparisons of keys are integer work,
// which matters here: FP64 issue is scarce on this part.
__device__ __forceinline__ long long dkey(double x)
{
    if (x == 0.0) return 0;
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}

// Per-call tables: the draws' keys (dimension-major, like the draws), the
// per-dimension least and largest draw, the values u / S for every count u
// (FP64, and FP32 rounded down / up) and a flag for non-finite draws.
__global__ void __launch_bounds__(kMcThreads)
mc_prep(const double *__restrict__ samples, int n, int64_t S, long long *__restrict__ keys,
        double *__restrict__ val, float *__restrict__ val_dn, float *__restrict__ val_up,
        unsigned *__restrict__ bad)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)n * S;
         i += stride) {
        const double w = samples[i];
        if (!isfinite(w)) atomicOr(bad, 1u);
        keys[i] = dkey(w);
    }
    const double dS = (double)S;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= S; u += stride) {
        const double v = (double)u / dS;
        val[u] = v;
        val_dn[u] = __double2float_rd(v);
        val_up[u] = __double2float_ru(v);
    }
}

// Per-dimension least and largest draw: range[2d], range[2d + 1].
__global__ void __launch_bounds__(kMcThreads)
mc_range(const double *__restrict__ samples, int64_t S, double *__restrict__ range)
{
    __shared__ double smin[kMcThreads], smax[kMcThreads];
    const int d = blockIdx.x;
    double a = INFINITY, b = -INFINITY;
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
        const double w = samples[(int64_t)d * S + s];
        a = fmin(a, w);
        b = fmax(b, w);
    }
    smin[threadIdx.x] = a;
    smax[threadIdx.x] = b;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + k]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + k]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        range[2 * d] = smin[0];
        range[2 * d + 1] = smax[0];
    }
}

// Cell of a coordinate: -1 below the domain, N above it, else the i with
// E_i <= y < E_{i+1} (the last cell also holds y == E_N). A first guess from
// the nominal width, corrected against the edges themselves.
__device__ __forceinline__ int cell_of(const double *__restrict__ E, int N, double inv_h, double y)
{
    if (y < E[0]) return -1;
    if (y > E[N]) return N;
    int i = (int)fmin(fmax(floor((y - E[0]) * inv_h), 0.0), (double)(N - 1));
    while (i > 0 && y < E[i]) --i;
    while (i < N - 1 && y >= E[i + 1]) ++i;
    return i;
}

// Neighbouring doubles of a finite x (bit arithmetic; 0 steps to the least
// subnormal of either sign).
__device__ __forceinline__ double step_up(double x)
{
    if (x == 0.0) return __longlong_as_double(1ll);
    const long long b = __double_as_longlong(x);
    return __longlong_as_double(x > 0.0 ? b + 1 : b - 1);
}
__device__ __forceinline__ double step_down(double x)
{
    if (x == 0.0) return -__longlong_as_double(1ll);
    const long long b = __double_as_longlong(x);
    return __longlong_as_double(x > 0.0 ? b - 1 : b + 1);
}

// The least double w whose rounded sum w + m reaches the edge E (gt: passes
// it). RN addition is monotone in w, so these w form an up-set; the guess
// E - m is moved a few ulps, and bisection over the keys' order finishes the
// rare case where the guess is far off (|m| much larger than |E - m|).
__device__ double threshold_of(double m, double E, bool gt)
{
    auto ok = [&](double w) {
        const double y = w + m;
        return gt ? y > E : y >= E;
    };
    double w = E - m;
    for (int k = 0; k < 2; ++k) {
        if (ok(w)) {
            const double p = step_down(w);
            if (!ok(p)) return w;
            w = p;
        } else {
            w = step_up(w);
        }
    }
    // bracket [lo, hi] with ok(hi) and not ok(lo), then bisection on the
    // order of doubles (the sign is handled by the keys' order)
    double span = fmax(fabs(m), fabs(E)) * 0x1p-50 + 0x1p-1000;
    double lo = w - span, hi = w + span;
    for (int k = 0; k < 64 && ok(lo); ++k) lo -= (span *= 2.0);
    for (int k = 0; k < 64 && !ok(hi); ++k) hi += (span *= 2.0);
    for (int k = 0; k < 128; ++k) {
        const long long kl = dkey(lo), kh = dkey(hi);
        if (kh - kl <= 1) break;
        // midpoint in key order, back to a double
        const long long km = kl + (kh - kl) / 2;
        const double mid = km >= 0 ? __longlong_as_double(km)
                                   : __longlong_as_double(km ^ 0x7fffffffffffffffll);
        if (ok(mid)) hi = mid; else lo = mid;
    }
    return hi;
}

struct McRow {
    double mlo[IMPACT_MAX_DIM], mhi[IMPACT_MAX_DIM];
    int o[IMPACT_MAX_DIM], e[IMPACT_MAX_DIM];   // window: first cell and extent per dimension
    int ws[IMPACT_MAX_DIM];                      // window strides (C order)
    int H;                                       // window cells (0: the draws all leave)
    unsigned sink_lo, sink_up;
    unsigned long long kept, dropped;
    int scan[kMcThreads / 32];
    // keys of the thresholds of edges o .. o + e, for the low and the high
    // end of the image: the draw's cell is o - 1 + #{k: key(w) >= thr[k]}
    long long thr_lo[IMPACT_MAX_DIM][kMcThr], thr_hi[IMPACT_MAX_DIM][kMcThr];
};

// #{k < cnt: t[k] <= key}, t ascending (binary search).
__device__ __forceinline__ int count_le(const long long *t, int cnt, long long key)
{
    int lo = 0, hi = cnt;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (t[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// One block per row (grid-stride over the rows). The draws move the row's
// image box; a block-wide histogram in shared memory counts, for every cell
// of the row's window, the draws whose moved box meets it (hu) and lies in it
// (hl). The cell of a moved end is found by integer comparisons of the draw's
// key with per-row thresholds (the FP64 decision of the definition, made
// exactly once per row and edge). The count pass writes the row's kept count,
// sink and dropped mass; the emit pass repeats the histogram and writes the
// kept cells in ascending order (cutoff 0 keeps every cell of the grid, as the
// dense definition does).
template <bool EMIT>
__global__ void __launch_bounds__(kMcThreads)
mc_rows(const ImpactDesc *__restrict__ Dp, int64_t rows, const long long *__restrict__ keys,
        int64_t S, const double *__restrict__ range, const double *__restrict__ val,
        const float *__restrict__ val_dn, const float *__restrict__ val_up, unsigned kmin,
        int hist_cap, RowOutputs o)
{
    extern __shared__ __align__(16) unsigned char mc_smem[];
    __shared__ McRow R;
    unsigned *hu = reinterpret_cast<unsigned *>(mc_smem);
    unsigned *hl = hu + hist_cap;
    const ImpactDesc &D = *Dp;
    const int n = D.n;
    const double dS = (double)S;
    const bool dense = D.cutoff <= 0.0;   // cutoff 0: every cell is kept
    const int64_t T = D.cells;
    if (EMIT && o.capacity >= 0 && o.row_ptr[o.total_at] > o.capacity) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(o.status, IMPACT_STATUS_CAPACITY);
        return;
    }
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        // the row's image and window: one thread per dimension
        if (threadIdx.x < (unsigned)n) {
            const int d = threadIdx.x;
            int idx[IMPACT_MAX_DIM];
            int j;
            decode_row(D, row, idx, j);
            double lo, hi;
            image_dim<false>(D, row, idx, j, d, lo, hi);
            const double mlo = fmin(lo, hi), mhi = fmax(lo, hi);   // ordered ends
            R.mlo[d] = mlo;
            R.mhi[d] = mhi;
            const ImpactDim &g = D.dim[d];
            const double *E = D.edges + g.edge_off;
            const int a = max(cell_of(E, g.N, g.inv_h, range[2 * d] + mlo), 0);
            const int b = min(cell_of(E, g.N, g.inv_h, range[2 * d + 1] + mhi), g.N - 1);
            R.o[d] = a;
            R.e[d] = b >= a ? b - a + 1 : 0;
        }
        __syncthreads();
        // the thresholds of every (dimension, edge, end), one per thread
        for (int q = threadIdx.x; q < n * 2 * kMcThr; q += blockDim.x) {
            const int d = q / (2 * kMcThr), r = q - d * (2 * kMcThr);
            const int end = r / kMcThr, k = r - end * kMcThr;
            const int ext = R.e[d];
            if (ext == 0 || ext > IMPACT_MC_EDGES_MAX || k > ext) continue;
            const ImpactDim &g = D.dim[d];
            const int edge = R.o[d] + k;
            const bool gt = edge == g.N;   // beyond the last edge: leaves the domain
            const long long t = dkey(threshold_of(end ? R.mhi[d] : R.mlo[d],
                                                  D.edges[g.edge_off + edge], gt));
            if (end) R.thr_hi[d][k] = t; else R.thr_lo[d][k] = t;
        }
        if (threadIdx.x == 0) {
            int64_t Hw = 1;
            bool wide = false;
            for (int d = 0; d < n; ++d) {
                Hw *= R.e[d];   // at most the grid's cell count
                wide = wide || R.e[d] > IMPACT_MC_EDGES_MAX;
            }
            int H = Hw < (int64_t)hist_cap ? (int)Hw : hist_cap;
            if (Hw > hist_cap || wide) {
                atomicOr(o.status, IMPACT_STATUS_MC_WINDOW);
                H = -1;
            }
            int st = 1;
            for (int d = n - 1; d >= 0; --d) {
                R.ws[d] = st;
                st *= R.e[d] > 0 ? R.e[d] : 1;
            }
            R.H = H;
            R.sink_lo = 0;
            R.sink_up = 0;
            R.kept = 0;
            R.dropped = 0;
        }
        __syncthreads();
        const int H = R.H;
        if (H < 0) {   // window too large: counted as empty, the call fails
            if (!EMIT && threadIdx.x == 0) o.row_ptr[row] = 0;
            __syncthreads();
            continue;
        }
        for (int h = threadIdx.x; h < H; h += blockDim.x) {
            hu[h] = 0;
            hl[h] = 0;
        }
        __syncthreads();
        unsigned my_sl = 0, my_su = 0;
        if (H > 0)
            for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
                // per dimension: the cells of the moved ends (integer
                // comparisons with the row's thresholds), the met range
                // relative to the window, and whether it spans two cells
                bool inside = true, outside = false, single = true, wide = false;
                int hb = 0, m2 = 0;
                unsigned pk = 0;   // dims whose met range spans two cells, 3 bits each
                int A[IMPACT_MAX_DIM], Bd[IMPACT_MAX_DIM];
#pragma unroll
                for (int d = 0; d < IMPACT_MAX_DIM; ++d) {
                    if (d < n) {
                        const long long kw = keys[(int64_t)d * S + s];
                        const int ext = R.e[d], N = D.dim[d].N;
                        const int a = R.o[d] - 1 + count_le(R.thr_lo[d], ext + 1, kw);
                        const int b = R.o[d] - 1 + count_le(R.thr_hi[d], ext + 1, kw);
                        inside = inside && a >= 0 && b <= N - 1;
                        outside = outside || b < 0 || a > N - 1;
                        single = single && a == b;
                        // relative to the window (inside it by construction;
                        // the clamps only bound malformed input)
                        const int top = ext - 1;
                        const int ad = min(max(max(a, 0) - R.o[d], 0), top);
                        const int bd = min(max(min(b, N - 1) - R.o[d], ad), top);
                        A[d] = ad;
                        Bd[d] = bd;
                        hb += ad * R.ws[d];
                        if (bd - ad == 1) {
                            pk |= (unsigned)d << (3 * m2);
                            ++m2;
                        } else if (bd - ad > 1) {
                            wide = true;
                        }
                    }
                }
                my_su += inside ? 0u : 1u;
                if (outside) {
                    ++my_sl;
                    continue;
                }
                if (single) atomicAdd(&hl[hb], 1u);
                atomicAdd(&hu[hb], 1u);
                if (!wide) {
                    // the other cells of a box of 2^m2 cells, in Gray-code
                    // order: one stride added or taken away per cell
                    int h = hb;
                    unsigned gray = 0;
                    for (unsigned k = 1; k < (1u << m2); ++k) {
                        const int j = __ffs(k) - 1;
                        const int dim = (pk >> (3 * j)) & 7;
                        const unsigned bit = 1u << j;
                        h += (gray & bit) ? -R.ws[dim] : R.ws[dim];
                        gray ^= bit;
                        atomicAdd(&hu[h], 1u);
                    }
                } else {
                    // a range of three or more cells somewhere: odometer walk
                    int c[IMPACT_MAX_DIM];
                    for (int d = 0; d < n; ++d) c[d] = A[d];
                    int h = hb;
                    while (true) {
                        int d = n - 1;
                        while (d >= 0 && c[d] == Bd[d]) {
                            h -= (c[d] - A[d]) * R.ws[d];
                            c[d] = A[d];
                            --d;
                        }
                        if (d < 0) break;
                        ++c[d];
                        h += R.ws[d];
                        atomicAdd(&hu[h], 1u);
                    }
                }
            }
        else   // every draw leaves the domain whole
            for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
                ++my_sl;
                ++my_su;
            }
        // block totals: a warp reduction, then one shared atomic per warp
        // (all threads on one shared word would serialise)
        my_sl = __reduce_add_sync(0xffffffffu, my_sl);
        my_su = __reduce_add_sync(0xffffffffu, my_su);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&R.sink_lo, my_sl);
            atomicAdd(&R.sink_up, my_su);
        }
        __syncthreads();

        if (!EMIT) {
            unsigned kept = 0;
            unsigned long long dropped = 0;
            if (!dense) {
                for (int h = threadIdx.x; h < H; h += blockDim.x) {
                    const unsigned u = hu[h];
                    if (u >= kmin) ++kept; else dropped += u;
                }
                kept = __reduce_add_sync(0xffffffffu, kept);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    dropped += __shfl_xor_sync(0xffffffffu, dropped, off);
                if ((threadIdx.x & 31) == 0) {
                    atomicAdd(&R.kept, (unsigned long long)kept);
                    atomicAdd(&R.dropped, dropped);
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                o.row_ptr[row] = dense ? T : (int64_t)R.kept;
                o.sink_lo[row] = (double)R.sink_lo / dS;
                o.sink_up[row] = (double)R.sink_up / dS;
                o.trunc[row] = (double)R.dropped / dS;
                if (o.flags) o.flags[row] = 0u;
            }
        } else {
            const int64_t base = o.row_ptr[row], end = o.row_ptr[row + 1];
            const bool f64 = D.prec == PREC_FP64_PLAIN;
            auto put = [&](int64_t pos, int64_t t, unsigned u, unsigned l) {
                o.col[pos] = (int32_t)t;
                if (f64) {
                    ((double *)o.up)[pos] = val[u];
                    ((double *)o.lo)[pos] = val[l];
                } else {
                    ((float *)o.up)[pos] = val_up[u];
                    ((float *)o.lo)[pos] = val_dn[l];
                }
            };
            if (dense) {
                // every cell of the grid, in order; outside the window the counts are 0
                for (int64_t t = threadIdx.x; t < T; t += blockDim.x) {
                    int64_t rest = t;
                    int h = 0;
                    bool in = H > 0;
                    for (int d = n - 1; d >= 0; --d) {
                        const int N = D.dim[d].N;
                        const int i = (int)(rest % N) - R.o[d];
                        rest /= N;
                        in = in && i >= 0 && i < R.e[d];
                        h += i * R.ws[d];
                    }
                    if (base + t < end) put(base + t, t, in ? hu[h] : 0u, in ? hl[h] : 0u);
                }
            } else {
                // the kept cells of the window in C order (ascending cell ids)
                const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
                int64_t at = 0;
                for (int h0 = 0; h0 < H; h0 += blockDim.x) {
                    const int h = h0 + threadIdx.x;
                    const bool keep = h < H && hu[h] >= kmin;
                    const unsigned m = __ballot_sync(0xffffffffu, keep);
                    if (lane == 0) R.scan[wid] = __popc(m);
                    __syncthreads();
                    int before = 0, total = 0;
                    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
                        if (k < wid) before += R.scan[k];
                        total += R.scan[k];
                    }
                    if (keep) {
                        int64_t t = 0;
                        int rest = h;
                        for (int d = 0; d < n; ++d) {
                            const int i = rest / R.ws[d];
                            rest -= i * R.ws[d];
                            t += (int64_t)(i + R.o[d]) * D.dim[d].stride;
                        }
                        const int64_t pos =
                            base + at + before + __popc(m & ((1u << lane) - 1u));
                        if (pos < end) put(pos, t, hu[h], hl[h]);
                    }
                    at += total;
                    __syncthreads();
                }
            }
        }
        __syncthreads();
    }
}

int grid_for(const void *kernel, int64_t rows)
{
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, 0);
    if (occ < 1) occ = 1;
    int64_t want = (rows + kWarpsPerBlock - 1) / kWarpsPerBlock;
    int64_t cap = (int64_t)sms * occ;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

}  // namespace

namespace impact {

cudaError_t launch_rows(const ImpactDesc *d_desc, int prec, bool emit, int64_t row_begin,
                        int64_t row_end, const RowOutputs &o, cudaStream_t stream)
{
    int64_t rows = row_end - row_begin;
    if (rows <= 0) return cudaSuccess;
    if (prec != PREC_FP64_PLAIN) return cudaErrorInvalidValue;
    {
        if (emit) {
            int g = grid_for((const void *)rows_fp64<true>, rows);
            rows_fp64<true><<<g, kThreads, 0, stream>>>(
                d_desc, row_begin, row_end, o.row_ptr, o.col, (double *)o.lo, (double *)o.up,
                o.sink_lo, o.sink_up, o.trunc, o.flags, o.status, o.capacity, o.total_at);
        } else {
            int g = grid_for((const void *)rows_fp64<false>, rows);
            rows_fp64<false><<<g, kThreads, 0, stream>>>(
                d_desc, row_begin, row_end, o.row_ptr, o.col, (double *)o.lo, (double *)o.up,
                o.sink_lo, o.sink_up, o.trunc, o.flags, o.status, o.capacity, o.total_at);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_labels(const RegionBoxes &boxes, int64_t total_cells, uint8_t *labels,
                          cudaStream_t stream)
{
    if (total_cells <= 0) return cudaSuccess;
    const int64_t g = std::min<int64_t>((total_cells + 255) / 256, 152 * 16);
    label_cells<<<(unsigned)g, 256, 0, stream>>>(boxes, total_cells, labels);
    return cudaGetLastError();
}

cudaError_t launch_regions(const ImpactDesc *d_desc, int64_t rows, const RegionBoxes &boxes,
                           bool cell_sum, bool sound, double *r_lo, double *r_up, double *a_lo,
                           double *a_up, cudaStream_t stream)
{
    if (rows <= 0) return cudaSuccess;
    const int64_t g = std::min<int64_t>((rows + 127) / 128, 152 * 32);
    if (sound)
        region_rows<true><<<(unsigned)g, 128, 0, stream>>>(d_desc, rows, boxes, cell_sum, r_lo,
                                                           r_up, a_lo, a_up);
    else
        region_rows<false><<<(unsigned)g, 128, 0, stream>>>(d_desc, rows, boxes, cell_sum, r_lo,
                                                            r_up, a_lo, a_up);
    return cudaGetLastError();
}

cudaError_t launch_mc_prep(const double *samples, int n, int64_t S, long long *keys,
                           double *val, float *val_dn, float *val_up, unsigned *bad,
                           double *range, cudaStream_t stream)
{
    const int64_t items = std::max<int64_t>((int64_t)n * S, S + 1);
    const int64_t g = std::min<int64_t>((items + kMcThreads - 1) / kMcThreads, 152 * 16);
    mc_prep<<<(unsigned)g, kMcThreads, 0, stream>>>(samples, n, S, keys, val, val_dn, val_up,
                                                     bad);
    mc_range<<<n, kMcThreads, 0, stream>>>(samples, S, range);
    return cudaGetLastError();
}

cudaError_t launch_mc_rows(const ImpactDesc *d_desc, bool emit, int64_t rows,
                           const long long *keys, int64_t S, const double *range,
                           const double *val, const float *val_dn, const float *val_up,
                           unsigned kmin, const RowOutputs &o, cudaStream_t stream)
{
    if (rows <= 0) return cudaSuccess;
    const int cap = IMPACT_MC_HIST_MAX;
    const size_t smem = (size_t)cap * 2 * sizeof(unsigned);
    const void *k = emit ? (const void *)mc_rows<true> : (const void *)mc_rows<false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kMcThreads, smem);
    const int64_t g = std::min<int64_t>(rows, (int64_t)sms * std::max(occ, 1));
    if (emit)
        mc_rows<true><<<(unsigned)g, kMcThreads, smem, stream>>>(
            d_desc, rows, keys, S, range, val, val_dn, val_up, kmin, cap, o);
    else
        mc_rows<false><<<(unsigned)g, kMcThreads, smem, stream>>>(
            d_desc, rows, keys, S, range, val, val_dn, val_up, kmin, cap, o);
    return cudaGetLastError();
}

int64_t scan_scratch_elems(int64_t n)
{
    return (n + kScanTile - 1) / kScanTile + 1;
}

cudaError_t launch_scan(int64_t *row_ptr, int64_t n, int64_t *scratch, cudaStream_t stream)
{
    int64_t nt = (n + kScanTile - 1) / kScanTile;
    if (nt < 1) nt = 1;
    scan_tiles<<<(unsigned)nt, kScanThreads, 0, stream>>>(row_ptr, n, scratch);
    scan_sums<<<1, kScanThreads, 0, stream>>>(scratch, nt, row_ptr + n);
    scan_apply<<<(unsigned)nt, kScanThreads, 0, stream>>>(row_ptr, n, scratch);
    return cudaGetLastError();
}

}  // namespace impact
