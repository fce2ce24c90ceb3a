// tree_fp32.cu -- FP32-sound construction (Def. 3.1 with outward rounding,
// Sec. 4.4 cutoff, Remark 4.1 sink) in three kernels:
//
//   setup_fp32  8 threads per row, thread d owns dimension d. From the
//               interval image of the cell it computes the window of target
//               cells that can pass the cutoff, the factor table U_d[t]
//               (upper bound of the largest Gaussian mass over the image) and
//               L_d[t] (lower bound of the smallest), trims the window to the
//               targets whose U passes, makes U unimodal (a running maximum
//               from each end: only raises upper bounds), and turns U into
//               exact pruning thresholds TH_d[t]. The row's sink bounds and
//               the mass of every target outside the window box are finished
//               here in FP64. Output: one fixed-size record per row.
//   tree_fp32   one warp per row walks the prefix tree of target cells in C
//               order. A node at depth d is a prefix (t_0..t_d) with the
//               RU-rounded running product P of its upper factors; its
//               children that can still reach the cutoff are exactly
//               {t : TH_{d+1}[t] <= P}, a contiguous run because U is
//               unimodal. Count pass: pairs per row, the in-box truncated
//               mass and the row checks, from per-node run sums. Emit pass:
//               the same walk, leaves written with warp-contiguous stores.
//
// Products run left to right over the dimensions with directed rounding
// (up: round up, lo: round down) whatever the enumeration order, so every
// pair's value depends only on its own row.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "impact_desc.h"
#include "kernels.h"
#include "sound_fp32.cuh"

namespace {

constexpr int kSetupThreads = 256;
constexpr int kWin = IMPACT_WINDOW_MAX;   // window entries per (row, dim) in setup
constexpr int kTsum = IMPACT_TSUM_MAX;    // factor entries per row record (all dims)
constexpr int kPool = 384;                // prefix nodes staged per warp
constexpr int kSeg = 512;                 // pairs staged per leaf batch
constexpr int kTreeWarps = 4;
constexpr int kTreeThreads = kTreeWarps * 32;
constexpr float kTwoM44 = 5.6843419e-14f;    // 2^-44
constexpr float kGrow18 = 1.0000038147f;     // 1 + 2^-18

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

struct Alpha {
    float kh, kl, err, rh, rl;
    __device__ __forceinline__ void at(int k, float &lo, float &hi) const
    {
        sound::alpha_interval(k, kh, kl, err, rh, rl, lo, hi);
    }
};

__global__ void __launch_bounds__(kSetupThreads)
setup_fp32(const ImpactDesc *__restrict__ Dp, int64_t row_begin, int64_t row_end,
           unsigned char *__restrict__ rec, double *__restrict__ sink_lo,
           double *__restrict__ sink_up, double *__restrict__ trunc,
           uint32_t *__restrict__ status)
{
    const ImpactDesc &D = *Dp;
    const int n = D.n;
    const int lane = threadIdx.x & 31;
    const int d = lane & 7;
    const unsigned gmask = 0xffu << (lane & 24);
    const bool act = d < n;
    const float cut = D.cutoff32;
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int64_t ng = ((int64_t)gridDim.x * blockDim.x) >> 3;
    float u[kWin], l[kWin];

    for (int64_t row = row_begin + g0; row < row_end; row += ng) {
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
        const ImpactDim &g = D.dim[act ? d : 0];

        // image of dimension d: window estimate (cells) and, in erf units,
        // rho = (E_a - m)/(sigma sqrt2) at m_lo and m_hi as FP32 pairs
        float mulo = 0.0f, muhi = 0.0f;
        float m0h = 0.0f, m0l = 0.0f, m1h = 0.0f, m1l = 0.0f, mag = 0.0f;
        double dmlo = 0.0, dmhi = 0.0;
        if (act) {
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
                float2 xlo = ea[idx[d]], xhi = ea[idx[d] + 1];
                acc_pair(m0h, m0l, xlo);
                acc_pair(m1h, m1l, xhi);
                float2 vl, vh;
                float cl, ch;
                if (d == 2) {
                    vl = vh = D.oma[j];
                    cl = ch = D.omm[j];
                } else {
                    int t = ((int)idx[2] * D.n_inputs + j) * 4 + 2 * d;
                    vl = D.ua[t];
                    vh = D.ua[t + 1];
                    cl = D.um[t];
                    ch = D.um[t + 1];
                }
                acc_pair(m0h, m0l, vl);
                acc_pair(m1h, m1l, vh);
                mag += fabsf(xlo.x) + fabsf(xhi.x) + fabsf(vl.x) + fabsf(vh.x);
                mulo = (float)idx[d] + cl;
                muhi = (float)(idx[d] + 1) + ch;
            } else {
                const double *im = D.images + (row * n + d) * 2;
                dmlo = im[0];
                dmhi = im[1];
                mulo = (float)((dmlo - g.lo) * g.inv_h);
                muhi = (float)((dmhi - g.lo) * g.inv_h);
            }
        }
        // conservative window [a, b]
        int a = 0, W = 0;
        bool bad = false;
        if (act) {
            float dc = g.delta_cells;
            float xa = floorf(mulo - dc - 1e-3f - 1e-5f * fabsf(mulo));
            float xb = floorf(muhi + dc + 1e-3f + 1e-5f * fabsf(muhi));
            float top = (float)(g.N - 1);
            xa = fminf(fmaxf(xa, 0.0f), top);
            xb = fminf(fmaxf(xb, 0.0f), top);
            a = (int)xa;
            int b = (int)xb;
            W = b - a + 1;
            if (W < 1) W = 1;
            if (W > kWin || W > g.wcap) bad = true;
        }
        Alpha A0, A1;
        if (act && !bad) {
            float2 ea = D.ea[g.edge_off + a];
            if (D.kind == KIND_IMAGES) {
                const double Ea = D.edges[g.edge_off + a];
                sound::split_pair((Ea - dmlo) * g.inv_s, A0.rh, A0.rl);
                sound::split_pair((Ea - dmhi) * g.inv_s, A1.rh, A1.rl);
                mag = (float)((fabs(Ea) + fabs(dmlo) + fabs(dmhi)) * g.inv_s);
            } else {
                sub_pair(ea, m0h, m0l, A0.rh, A0.rl);
                sub_pair(ea, m1h, m1l, A1.rh, A1.rl);
                mag += fabsf(ea.x);
            }
            A0.kh = A1.kh = g.kappa_hi;
            A0.kl = A1.kl = g.kappa_lo;
            A0.err = A1.err = __fadd_ru(g.edge_err, __fmul_ru(__fmul_ru(mag, 4.0f), kTwoM44));
        }

        // factor table of the window
        float M = 0.0f, SW = 0.0f, O = 0.0f, qlo = 0.0f, qhi = 0.0f;
        int first = -1, last = -1, pk = 0;
        if (act && !bad) {
            float c0l, c0h, c1l, c1h;
            A0.at(0, c0l, c0h);
            A1.at(0, c1l, c1h);
            for (int k = 0; k < W; ++k) {
                float e0l, e0h, e1l, e1h;
                A0.at(k + 1, e0l, e0h);
                A1.at(k + 1, e1l, e1h);
                float U;
                if (__fadd_ru(c0h, e0h) <= 0.0f)          // target midpoint <= m_lo
                    U = sound::mass_hi(c0l, c0h, e0l, e0h);
                else if (__fadd_rd(c1l, e1l) >= 0.0f)     // target midpoint >= m_hi
                    U = sound::mass_hi(c1l, c1h, e1l, e1h);
                else                                       // midpoint may be inside
                    U = g.plateau_hi;
                float L = fminf(sound::mass_lo(c0l, c0h, e0l, e0h),
                                sound::mass_lo(c1l, c1h, e1l, e1h));
                u[k] = U;
                l[k] = L;
                if (U >= cut) {
                    if (first < 0) first = k;
                    last = k;
                }
                c0l = e0l; c0h = e0h; c1l = e1l; c1h = e1h;
            }
            // unimodal envelope of U on the trimmed window, its max and sums
            if (first >= 0) {
                pk = first;
                for (int k = first + 1; k <= last; ++k)
                    if (u[k] > u[pk]) pk = k;
                for (int k = first + 1; k < pk; ++k) u[k] = fmaxf(u[k], u[k - 1]);
                for (int k = last - 1; k > pk; --k) u[k] = fmaxf(u[k], u[k + 1]);
                M = u[pk];
                for (int k = first; k <= last; ++k) SW = __fadd_ru(SW, u[k]);
            }
            for (int k = 0; k < W; ++k)
                if (first < 0 || k < first || k > last) O = __fadd_ru(O, u[k]);
            // cells left of the window (all left of the image): mass at m_lo;
            // cells right of it: mass at m_hi (telescoped over the cells)
            float al, ah, bl, bh;
            if (a > 0) {
                A0.at(-a, al, ah);
                A0.at(0, bl, bh);
                O = __fadd_ru(O, sound::mass_hi(al, ah, bl, bh));
            }
            if (a + W < g.N) {
                A1.at(W, al, ah);
                A1.at(g.N - a, bl, bh);
                O = __fadd_ru(O, sound::mass_hi(al, ah, bl, bh));
            }
            // out-of-domain mass Q(m) = T(-alpha(lo_D)) + T(alpha(hi_D))
            float l0l, l0h, h0l, h0h, l1l, l1h, h1l, h1h;
            A0.at(-a, l0l, l0h);
            A0.at(g.N - a, h0l, h0h);
            A1.at(-a, l1l, l1h);
            A1.at(g.N - a, h1l, h1h);
            float q0 = __fadd_ru(sound::tail_hi(-l0h), sound::tail_hi(h0l));
            float q1 = __fadd_ru(sound::tail_hi(-l1h), sound::tail_hi(h1l));
            qhi = fminf(fmaxf(q0, q1), 1.0f);
            if (__fadd_ru(l0h, h0h) <= 0.0f)
                qlo = __fadd_rd(sound::tail_lo(-l0l), sound::tail_lo(h0h));
            else if (__fadd_rd(l1l, h1l) >= 0.0f)
                qlo = __fadd_rd(sound::tail_lo(-l1l), sound::tail_lo(h1h));
            else
                qlo = g.qmin_lo;
            qlo = fminf(qlo, 1.0f);
        }
        int tw = (act && !bad && first >= 0) ? last - first + 1 : 0;
        bool any_bad = __any_sync(gmask, bad);

        // cross-dimension terms within the row's 8 threads
        float R = 1.0f, SWR = 1.0f;
        int toff = 0, tsum = 0;
        for (int k = 0; k < n; ++k) {
            float Mk = __shfl_sync(gmask, M, k, 8);
            float SWk = __shfl_sync(gmask, SW, k, 8);
            int twk = __shfl_sync(gmask, tw, k, 8);
            if (k > d) {
                R = __fmul_ru(R, Mk);
                SWR = __fmul_ru(SWR, SWk);
            }
            if (k < d) toff += twk;
            tsum += twk;
        }
        if (tsum > D.tsum_cap) any_bad = true;
        if (any_bad) {
            tw = 0;
            tsum = 0;
            toff = 0;
        }
        // thresholds: a child t of a depth-(d-1) node with product P is kept
        // iff TH_d[t] <= P, i.e. RU(RU(P U_d[t]) R') >= cutoff, R' bounding the
        // product of the remaining dimensions' largest factors
        float cp = 0.0f;
        if (cut > 0.0f) cp = (d == n - 1) ? cut : threshold(cut, __fmul_ru(R, kGrow18));

        unsigned char *rr = rec + (row - row_begin) * (int64_t)D.rec_stride;
        if (act) {
            int4 h = make_int4(a + (first >= 0 ? first : 0), tw, pk - (first >= 0 ? first : 0),
                               __float_as_int(SWR));
            reinterpret_cast<int4 *>(rr)[d] = h;
            float *RU = reinterpret_cast<float *>(rr + 16 * n) + toff;
            float *RL = RU + D.tsum_cap;
            float *RT = RL + D.tsum_cap;
            for (int k = 0; k < tw; ++k) {
                float uk = u[first + k];
                RU[k] = uk;
                RL[k] = l[first + k];
                RT[k] = (cp > 0.0f) ? threshold(cp, uk) : 0.0f;
            }
        }

        // row terms (thread 0 of the row): sink bounds and the mass outside
        // the window box, combined in FP64 with outward rounding
        float gq_lo[IMPACT_MAX_DIM], gq_hi[IMPACT_MAX_DIM], gsw[IMPACT_MAX_DIM], go[IMPACT_MAX_DIM];
#pragma unroll
        for (int k = 0; k < IMPACT_MAX_DIM; ++k) {
            gq_lo[k] = __shfl_sync(gmask, qlo, k, 8);
            gq_hi[k] = __shfl_sync(gmask, qhi, k, 8);
            gsw[k] = __shfl_sync(gmask, SW, k, 8);
            go[k] = __shfl_sync(gmask, O, k, 8);
        }
        if (d == 0) {
            double pin_up = 1.0, pin_dn = 1.0, outside = 0.0, pre = 1.0;
#pragma unroll
            for (int k = 0; k < IMPACT_MAX_DIM; ++k) {
                if (k < n) {
                    pin_up = __dmul_ru(pin_up, __dsub_ru(1.0, (double)gq_lo[k]));
                    pin_dn = __dmul_rd(pin_dn, __dsub_rd(1.0, (double)gq_hi[k]));
                }
            }
            // partition the targets outside the box by the first dimension whose
            // index leaves the window: prod_{k<d} SW_k * O_d * prod_{k>d} (SW_k + O_k)
#pragma unroll
            for (int k = 0; k < IMPACT_MAX_DIM; ++k) {
                if (k < n) {
                    double post = 1.0;
#pragma unroll
                    for (int q = k + 1; q < IMPACT_MAX_DIM; ++q)
                        if (q < n) post *= (double)gsw[q] + (double)go[q];
                    outside += pre * (double)go[k] * post;
                    pre *= (double)gsw[k];
                }
            }
            if (sink_lo) {
                sink_lo[row] = fmax(__dsub_rd(1.0, pin_up), 0.0);
                sink_up[row] = fmin(__dsub_ru(1.0, pin_dn), 1.0);
                trunc[row] = outside * (1.0 + 1e-12);
            }
            if (any_bad) atomicOr(status, IMPACT_STATUS_TABLE_OVERFLOW);
        }
    }
}

// ---------------------------------------------------------------------------
// the prefix-tree walk
// ---------------------------------------------------------------------------

struct TreeSm {
    float U[kTsum], L[kTsum], T[kTsum];
    float pu_up[kTsum + IMPACT_MAX_DIM], pu_dn[kTsum + IMPACT_MAX_DIM];   // prefix sums of U
    float pl_up[kTsum + IMPACT_MAX_DIM], pl_dn[kTsum + IMPACT_MAX_DIM];   // prefix sums of L
    float su_up[kTsum + IMPACT_MAX_DIM];                                   // suffix sums of U
    float npu[kPool], npl[kPool];
    int ncol[kPool];
    float bpu[32], bpl[32];
    int bcol[32], bl[32], bo[32];
    unsigned char seg[kSeg];
    int ta[IMPACT_MAX_DIM], tw[IMPACT_MAX_DIM], pk[IMPACT_MAX_DIM], toff[IMPACT_MAX_DIM];
    float swr[IMPACT_MAX_DIM];
    int cnt[IMPACT_MAX_DIM], cur[IMPACT_MAX_DIM], base[IMPACT_MAX_DIM];
};

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
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
__device__ __forceinline__ void run_of(const TreeSm &S, int dim, float P, int &l, int &c)
{
    const int off = S.toff[dim], pk = S.pk[dim], tw = S.tw[dim];
    int cl = 0, cr = 0;
    for (int t = 0; t <= pk; ++t) cl += (S.T[off + t] <= P) ? 1 : 0;
    for (int t = pk + 1; t < tw; ++t) cr += (S.T[off + t] <= P) ? 1 : 0;
    c = cl > 0 ? cl + cr : 0;
    l = pk + 1 - cl;
}

// Upper bound of the sum of U over the window of `dim` outside [l, l + c):
// a prefix sum plus a suffix sum, both rounded up (no cancellation).
__device__ __forceinline__ float outside_sum(const TreeSm &S, int dim, int l, int c)
{
    const int po = S.toff[dim] + dim, tw = S.tw[dim];
    if (c == 0) return S.pu_up[po + tw];
    return __fadd_ru(S.pu_up[po + l], S.su_up[po + l + c]);
}

template <bool EMIT>
__global__ void __launch_bounds__(kTreeThreads)
tree_fp32(const ImpactDesc *__restrict__ Dp, int64_t row_begin, int64_t row_end,
          const unsigned char *__restrict__ rec, int64_t *__restrict__ row_ptr,
          int32_t *__restrict__ out_col, float *__restrict__ out_lo, float *__restrict__ out_up,
          const double *__restrict__ sink_lo, const double *__restrict__ sink_up,
          double *__restrict__ trunc, uint32_t *__restrict__ flags, uint32_t *__restrict__ status,
          int64_t capacity, int64_t total_at)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const ImpactDesc &D = *Dp;
    const int lane = threadIdx.x & 31;
    TreeSm &S = reinterpret_cast<TreeSm *>(smem_raw)[threadIdx.x >> 5];
    const int n = D.n;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned lt = lanemask_lt();
    if (EMIT && capacity >= 0 && row_ptr[total_at] > capacity) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(status, IMPACT_STATUS_CAPACITY);
        return;
    }

    for (int64_t row = row_begin + warp0; row < row_end; row += nwarps) {
        const unsigned char *rr = rec + (row - row_begin) * (int64_t)D.rec_stride;
        // load the row record
        if (lane < n) {
            int4 h = reinterpret_cast<const int4 *>(rr)[lane];
            S.ta[lane] = h.x;
            S.tw[lane] = h.y;
            S.pk[lane] = h.z;
            S.swr[lane] = __int_as_float(h.w);
        }
        __syncwarp();
        int tsum = 0;
        bool empty = false;
        for (int k = 0; k < n; ++k) {
            if (lane == 0) S.toff[k] = tsum;
            tsum += S.tw[k];
            empty |= (S.tw[k] == 0);
        }
        {
            const float *RU = reinterpret_cast<const float *>(rr + 16 * n);
            for (int i = lane; i < tsum; i += 32) {
                S.U[i] = RU[i];
                S.L[i] = RU[D.tsum_cap + i];
                S.T[i] = RU[2 * D.tsum_cap + i];
            }
        }
        __syncwarp();
        if (!EMIT && lane < n) {   // prefix sums of U and L per dimension
            const int off = S.toff[lane], po = off + lane, tw = S.tw[lane];
            float a = 0.0f, b = 0.0f, c = 0.0f, e = 0.0f;
            S.pu_up[po] = 0.0f; S.pu_dn[po] = 0.0f; S.pl_up[po] = 0.0f; S.pl_dn[po] = 0.0f;
            for (int t = 0; t < tw; ++t) {
                a = __fadd_ru(a, S.U[off + t]);
                b = __fadd_rd(b, S.U[off + t]);
                c = __fadd_ru(c, S.L[off + t]);
                e = __fadd_rd(e, S.L[off + t]);
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

        float drop = 0.0f, sup = 0.0f, slo = 0.0f;   // count pass, per lane
        int cnt = 0;
        int64_t out_base = 0, out_end = 0, written = 0;
        if (EMIT) {
            out_base = row_ptr[row];
            out_end = row_ptr[row + 1];
        }
        bool overflow = false;
        if (!empty) {
            const int leaf = n - 1;
            // node buffers: level 0 holds the children of the root (<= tw_0);
            // a deeper level holds the children of one batch of B parents
            int B = 32;
            if (n >= 3) {
                int s = 0;
                for (int k = 1; k <= n - 2; ++k) s += S.tw[k];
                B = min(32, (kPool - S.tw[0]) / max(s, 1));
            }
            if (lane == 0) {
                int bse = 0;
                for (int k = 0; k <= n - 2; ++k) {
                    S.base[k] = bse;
                    bse += (k == 0) ? S.tw[0] : B * S.tw[k];
                }
            }
            __syncwarp();
            if (B < 1) overflow = true;
            const int LB = min(32, kSeg / max(S.tw[leaf], 1));   // leaf parents per batch

            // leaf processing of parents [p0, p0 + np) of a parent array
            auto leaf_batch = [&](const float *ppu, const float *ppl, const int *pcol, int p0,
                                  int np) {
                bool act = lane < np;
                float P = act ? ppu[p0 + lane] : 0.0f;
                float Pl = act ? ppl[p0 + lane] : 0.0f;
                int cb = act ? pcol[p0 + lane] : 0;
                int l = 0, c = 0;
                if (act) run_of(S, leaf, P, l, c);
                if (!EMIT) {
                    if (act) {
                        const int po = S.toff[leaf] + leaf;
                        cnt += c;
                        if (c > 0) {
                            float su = fmaxf(__fsub_ru(S.pu_up[po + l + c], S.pu_dn[po + l]), 0.0f);
                            float sl = fmaxf(__fsub_rd(S.pl_dn[po + l + c], S.pl_up[po + l]), 0.0f);
                            sup = __fadd_ru(sup, __fmul_ru(P, su));
                            slo = __fadd_rd(slo, __fmul_rd(Pl, sl));
                        }
                        drop = __fadd_ru(drop, __fmul_ru(P, outside_sum(S, leaf, l, c)));
                    }
                } else {
                    int C;
                    int o = warp_excl_scan(c, C);
                    S.bpu[lane] = P;
                    S.bpl[lane] = Pl;
                    S.bcol[lane] = cb + S.ta[leaf];
                    S.bl[lane] = l;
                    S.bo[lane] = o;
                    for (int k = 0; k < c; ++k) S.seg[o + k] = (unsigned char)lane;
                    __syncwarp();
                    const int off = S.toff[leaf];
                    for (int e = lane; e < C; e += 32) {
                        int p = S.seg[e];
                        int t = S.bl[p] + e - S.bo[p];
                        float uv = __fmul_ru(S.bpu[p], S.U[off + t]);
                        float lv = __fmul_rd(S.bpl[p], S.L[off + t]);
                        int64_t pos = out_base + written + e;
                        if (pos < out_end) {
                            out_col[pos] = S.bcol[p] + t;
                            out_lo[pos] = lv;
                            out_up[pos] = uv;
                        }
                    }
                    written += C;
                    __syncwarp();
                }
            };

            // expansion of parents [p0, p0 + np) into the children on `dim`
            auto expand = [&](const float *ppu, const float *ppl, const int *pcol, int p0, int np,
                              int dim) -> int {
                bool act = lane < np;
                float P = act ? ppu[p0 + lane] : 0.0f;
                float Pl = act ? ppl[p0 + lane] : 0.0f;
                int cb = act ? pcol[p0 + lane] : 0;
                int l = 0, c = 0;
                if (act) run_of(S, dim, P, l, c);
                int C;
                int o = warp_excl_scan(c, C);
                const int off = S.toff[dim], st = D.dim[dim].stride, ta = S.ta[dim];
                const int bse = S.base[dim];
                for (int k = 0; k < c; ++k) {
                    int t = l + k;
                    S.npu[bse + o + k] = (dim == 0) ? S.U[off + t] : __fmul_ru(P, S.U[off + t]);
                    S.npl[bse + o + k] = (dim == 0) ? S.L[off + t] : __fmul_rd(Pl, S.L[off + t]);
                    S.ncol[bse + o + k] = cb + (ta + t) * st;
                }
                if (!EMIT && act)
                    drop = __fadd_ru(drop, __fmul_ru(__fmul_ru(P, outside_sum(S, dim, l, c)),
                                                     S.swr[dim]));
                __syncwarp();
                return C;
            };

            if (!overflow) {
                if (n == 1) {
                    if (lane == 0) {
                        S.bpu[0] = 1.0f;   // the root: empty product
                        S.bpl[0] = 1.0f;
                        S.bcol[0] = 0;
                    }
                    __syncwarp();
                    leaf_batch(S.bpu, S.bpl, S.bcol, 0, 1);
                } else {
                    float one_u = 1.0f, one_l = 1.0f;
                    int zero = 0;
                    int c0 = expand(&one_u, &one_l, &zero, 0, 1, 0);
                    if (lane == 0) {
                        S.cnt[0] = c0;
                        S.cur[0] = 0;
                    }
                    __syncwarp();
                    int lev = 0;
                    while (true) {
                        if (lev == n - 2) {
                            const int bse = S.base[lev];
                            for (int p = 0; p < S.cnt[lev]; p += LB)
                                leaf_batch(S.npu + bse, S.npl + bse, S.ncol + bse, p,
                                           min(LB, S.cnt[lev] - p));
                            if (lev == 0) break;
                            --lev;
                            continue;
                        }
                        if (S.cur[lev] >= S.cnt[lev]) {
                            if (lev == 0) break;
                            --lev;
                            continue;
                        }
                        const int bse = S.base[lev];
                        int p0 = S.cur[lev];
                        int np = min(B, S.cnt[lev] - p0);
                        int cc = expand(S.npu + bse, S.npl + bse, S.ncol + bse, p0, np, lev + 1);
                        if (lane == 0) {
                            S.cur[lev] = p0 + np;
                            S.cnt[lev + 1] = cc;
                            S.cur[lev + 1] = 0;
                        }
                        __syncwarp();
                        ++lev;
                    }
                }
            }
        }

        if (EMIT) {
            if (lane == 0 && (overflow || out_base + written != out_end))
                atomicOr(status, overflow ? IMPACT_STATUS_TABLE_OVERFLOW
                                          : IMPACT_STATUS_EMIT_MISMATCH);
        } else {
            double dsum = (double)drop, usum = (double)sup, lsum = (double)slo;
            long long csum = cnt;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
                usum += __shfl_xor_sync(0xffffffffu, usum, o);
                lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
                csum += __shfl_xor_sync(0xffffffffu, csum, o);
            }
            if (lane == 0) {
                row_ptr[row] = overflow ? 0 : csum;
                double tr = trunc[row] + dsum * (1.0 + 1e-12);
                trunc[row] = tr;
                if (overflow) atomicOr(status, IMPACT_STATUS_TABLE_OVERFLOW);
                if (flags) {
                    // the emitted values are RU / RD products of the factors:
                    // widen the run sums by their rounding before testing
                    double lo_sum = lsum * (1.0 - 1e-6);
                    double up_sum = usum * (1.0 + 1e-6);
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
    return ((int64_t)16 * n + (int64_t)12 * tsum_cap + 15) / 16 * 16;
}

cudaError_t launch_setup_fp32(const ImpactDesc *d_desc, int64_t row_begin, int64_t row_end,
                              unsigned char *rec, double *sink_lo, double *sink_up, double *trunc,
                              uint32_t *status, cudaStream_t stream)
{
    int64_t rows = row_end - row_begin;
    if (rows <= 0) return cudaSuccess;
    int g = occupancy_grid((const void *)setup_fp32, kSetupThreads, 0, rows, kSetupThreads / 8);
    setup_fp32<<<g, kSetupThreads, 0, stream>>>(d_desc, row_begin, row_end, rec, sink_lo,
                                                sink_up, trunc, status);
    return cudaGetLastError();
}

cudaError_t launch_tree_fp32(const ImpactDesc *d_desc, bool emit, int64_t row_begin,
                             int64_t row_end, const unsigned char *rec, const RowOutputs &o,
                             cudaStream_t stream)
{
    int64_t rows = row_end - row_begin;
    if (rows <= 0) return cudaSuccess;
    const size_t smem = sizeof(TreeSm) * kTreeWarps;
    const void *k = emit ? (const void *)tree_fp32<true> : (const void *)tree_fp32<false>;
    static bool attr_set[2] = {false, false};
    if (!attr_set[emit]) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set[emit] = true;
    }
    int g = occupancy_grid(k, kTreeThreads, smem, rows, kTreeWarps);
    if (emit)
        tree_fp32<true><<<g, kTreeThreads, smem, stream>>>(
            d_desc, row_begin, row_end, rec, o.row_ptr, o.col, (float *)o.lo, (float *)o.up,
            o.sink_lo, o.sink_up, o.trunc, o.flags, o.status, o.capacity, o.total_at);
    else
        tree_fp32<false><<<g, kTreeThreads, smem, stream>>>(
            d_desc, row_begin, row_end, rec, o.row_ptr, o.col, (float *)o.lo, (float *)o.up,
            o.sink_lo, o.sink_up, o.trunc, o.flags, o.status, o.capacity, o.total_at);
    return cudaGetLastError();
}

}  // namespace impact
