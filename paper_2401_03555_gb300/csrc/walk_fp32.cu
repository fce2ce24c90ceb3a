// walk_fp32.cu -- FP32-sound construction (Def. 3.1 with outward rounding,
// Sec. 4.4 cutoff, Remark 4.1 sink) in two steps.
//
//   setup_fp32  one lane per (row, dimension), the 32/n rows of a warp
//               aligned to it (Alg. 2: rows are independent). From the
//               interval image of the source cell the lane finds the window
//               of target cells that can pass the cutoff, evaluates erf/erfc
//               once per window edge at the image's lower and upper end, and
//               writes the window's factor table to the row's record: U[t] >=
//               the largest Gaussian mass of target t over the image (T_max of
//               Def. 3.1 relaxed to the image box) and L[t] <= the smallest
//               (T_min), trimmed to the targets that pass on their own. The
//               lanes of a row then exchange their window maxima and sums by
//               shuffles: each finishes its dimension's pruning threshold, and
//               the lane of dimension 0 writes the row's sink bounds and the
//               mass of the targets outside the window box (FP64, outward).
//   walk_fp32   one warp per row, persistent (rows from an atomic counter in
//               ascending order). It walks the prefix tree of target cells
//               level by level in C order over the first n - 2 dimensions: a
//               node at level k is a prefix (t_0..t_k) with the RU-rounded
//               product P of its upper factors; the children of a list of
//               nodes are enumerated as candidates, one lane each, a child is
//               kept iff RU(P U[t]) can still reach the cutoff under the
//               largest factors of the later dimensions, and the warp compacts
//               the kept ones (ballot + popc) into the next level's list (lists
//               hold kCap nodes; longer expansions are taken in chunks, depth
//               first, so leaves come out in C order). The last two dimensions
//               form one leaf table per row, B[a, b] = RU(U[a] U[b]) (and the
//               RD product of the lower factors), so a pair's bound is one more
//               product RU(P B[a, b]). The count pass finds how many entries of
//               B pass under each parent by a binary search in B sorted by
//               value, with prefix sums for the row sums; the emit pass tests
//               every entry of B under each parent, one lane each, and stores
//               the kept pairs warp-contiguously.
//
// Kernel modes: COUNT (pairs per row, truncated mass, row checks), EMIT
// (pairs at given row offsets) and FUSED (both: each row publishes its pair
// count, finds its offset by a decoupled look-back over the rows before it,
// and writes its pairs).
//
// Upper bounds are products rounded up, lower bounds products rounded down,
// associated as ((..(U_0 U_1) ..) U_{n-3}) (U_{n-2} U_{n-1}) whatever the
// enumeration order, so a pair's value depends only on its row. Every
// lane-to-candidate assignment is a function of the row alone, so per-lane
// partial sums and their fixed reduction tree give the same bits under every
// launch shape and in every batch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/impact.h"
#include "impact_desc.h"
#include "kernels.h"
#include "sound_fp32.cuh"

namespace {

constexpr float kTwoM44 = 5.6843419e-14f;       // 2^-44
constexpr float kGrow18 = 1.0000038147f;        // 1 + 2^-18

__device__ __forceinline__ uint32_t fastdiv(uint32_t x, uint32_t m, int s)
{
    return (__umulhi(x, m) + x) >> s;   // exact for x < 2^31 (host-built m, s)
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
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

// Problem of a batch that owns global row x: begin[q] <= x < begin[q + 1].
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

// Edge point: alpha = (E - m)/(sigma sqrt2) at one image end, its half-width
// and its tails.
struct EdgePt {
    float a, da;
    sound::TailPair t;
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

// One dimension of a row: the window [a, a + W) of target cells that can
// pass the cutoff and, in erf units, rho = (E_a - m)/(sigma sqrt2) at both
// image ends as FP32 pairs (edge a + k is then rho + k kappa).
struct Win {
    int a, W;
    float kh, kl, err;          // kappa (cell width in erf units) pair, edge error
    float rh0, rl0, rh1, rl1;   // rho at m_lo and m_hi, pairs
};

__device__ __forceinline__ EdgePt edge_at(const Win &h, int k, bool hi_end)
{
    EdgePt e;
    sound::alpha_point(k, h.kh, h.kl, h.err, hi_end ? h.rh1 : h.rh0, hi_end ? h.rl1 : h.rl0, e.a,
                       e.da);
    e.t = sound::tails(e.a, e.da);
    return e;
}

// The interval image of the source cell in dimension d (affine sign
// split or unicycle trig ranges from host tables, or the caller's images),
// the window [a, a + W) of targets that can pass the cutoff (every target
// outside lies more than delta beyond the image), and rho = (E_a - m) /
// (sigma sqrt2) at both image ends as FP32 pairs. False if the window
// exceeds the planner's bound wcap.
__device__ bool dim_window(const ImpactDesc &D, int64_t row, int d, Win &h)
{
    const int n = D.n;
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
            idx[k] = 0;
            if (k < n) {
                uint32_t q = fastdiv(c, D.dim[k].div_m, D.dim[k].div_s);
                idx[k] = (int)(c - q * (uint32_t)D.dim[k].N);
                c = q;
            }
        }
    }
    int my_idx = 0, idx2 = idx[2 < IMPACT_MAX_DIM ? 2 : 0];
#pragma unroll
    for (int k = 0; k < IMPACT_MAX_DIM; ++k)
        if (k == d) my_idx = idx[k];
    const ImpactDim &g = D.dim[d];

    float mulo = 0.0f, muhi = 0.0f;   // image ends in cells (window placement only)
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
            int t = (idx2 * D.n_inputs + j) * 4 + 2 * d;
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
    // conservative window [a, a + W): every target outside has U below the
    // cutoff (its cell lies more than delta beyond the image)
    const float dc = g.delta_cells;
    float xa = floorf(mulo - dc - 1e-3f - 1e-5f * fabsf(mulo));
    float xb = floorf(muhi + dc + 1e-3f + 1e-5f * fabsf(muhi));
    const float top = (float)(g.N - 1);
    xa = fminf(fmaxf(xa, 0.0f), top);
    xb = fminf(fmaxf(xb, 0.0f), top);
    const int a = (int)xa;
    const int W = max((int)xb - a + 1, 1);
    h.a = a;
    h.W = W;
    if (W > g.wcap) return false;
    float2 ea = D.ea[g.edge_off + a];
    if (D.kind == KIND_IMAGES) {
        const double Ea = D.edges[g.edge_off + a];
        sound::split_pair((Ea - dmlo) * g.inv_s, h.rh0, h.rl0);
        sound::split_pair((Ea - dmhi) * g.inv_s, h.rh1, h.rl1);
        mag = (float)((fabs(Ea) + fabs(dmlo) + fabs(dmhi)) * g.inv_s);
    } else {
        sub_pair(ea, m0h, m0l, h.rh0, h.rl0);
        sub_pair(ea, m1h, m1l, h.rh1, h.rl1);
        mag += fabsf(ea.x);
    }
    h.kh = g.kappa_hi;
    h.kl = g.kappa_lo;
    h.err = __fadd_ru(g.edge_err, __fmul_ru(__fmul_ru(mag, 4.0f), kTwoM44));
    return true;
}


// ---------------------------------------------------------------------------
// setup: one record per row
// ---------------------------------------------------------------------------

// Per (row, dimension) entry of a row record. The record is RecDim[n], then
// the window tables, (U, L) pairs, dimension d's at entry rec_off[d].
struct RecDim {
    int tw;          // trimmed width: targets first..last that pass on their own
    int tb;          // table entry of the first trimmed target
    int cb;          // column of the first trimmed target: (a + first) * stride
    uint32_t magic;  // ceil(2^32 / tw) when tw > 1: e / tw = umulhi(e, magic)
    float cp;        // least child product whose subtree can still reach the cutoff
    float SR;        // RU product of the later dimensions' window sums
    int stride;      // column stride of the dimension (C order)
    int lay;         // the walk's layout (tw <= 32): lanes hold floor(32 / tw) parents
                     // (bits 0-15), a chunk is floor(kCap / tw) whole parents of
                     // candidates (bits 16-31); wider windows: 0
};
static_assert(sizeof(RecDim) == 32, "RecDim layout");

// Everything of one (row, dimension) that needs no other dimension.
struct DimOut {
    int tw = 0, f0 = 0, a = 0;
    float M = 0.0f;     // largest U
    float SW = 0.0f;    // sum of U over the trimmed window (rounded up)
    float O = 0.0f;     // mass outside the trimmed window (rounded up)
    float qlo = 0.0f, qhi = 0.0f;   // out-of-domain mass bounds
};

// The window of dimension d of a row and its factor table, written to `ul`
// (the record's entries of dimension d): U[k], L[k] for target a + k from the
// tails of its two edges at both image ends (neighbouring targets share an
// edge), then the trimmed window, its sums and the out-of-domain bounds.
__device__ DimOut setup_dim(const ImpactDesc &D, int64_t row, int d, float2 *ul, uint32_t *status)
{
    DimOut o;
    Win h;
    if (!dim_window(D, row, d, h)) {
        atomicOr(status, IMPACT_STATUS_TABLE_OVERFLOW);
        return o;
    }
    const ImpactDim &g = D.dim[d];
    const float cut = D.cutoff32;
    o.a = h.a;
    EdgePt c0 = edge_at(h, 0, false), c1 = edge_at(h, 0, true);
    const EdgePt w0 = c0;   // edge a at m_lo (left tail below)
    int first = -1, last = -1;
    float pre = 0.0f, mid = 0.0f, post = 0.0f, M = 0.0f;
    for (int k = 0; k < h.W; ++k) {
        const EdgePt e0 = edge_at(h, k + 1, false), e1 = edge_at(h, k + 1, true);
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
        ul[k] = make_float2(U, L);
        if (U >= cut) {
            if (first < 0) {
                first = k;
                mid = U;
            } else {
                mid = __fadd_ru(mid, __fadd_ru(post, U));
                post = 0.0f;
            }
            last = k;
            M = fmaxf(M, U);
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
    const EdgePt lo0 = edge_at(h, -h.a, false), hi0 = edge_at(h, g.N - h.a, false);
    const EdgePt lo1 = edge_at(h, -h.a, true), hi1 = edge_at(h, g.N - h.a, true);
    if (h.a > 0)   // cells 0..a-1 lie left of the image: their mass at m_lo
        O = __fadd_ru(O, sound::cell_hi(lo0.a, lo0.t, w0.a, w0.t));
    if (h.a + h.W < g.N)   // cells right of the window: their mass at m_hi
        O = __fadd_ru(O, sound::cell_hi(c1.a, c1.t, hi1.a, hi1.t));
    // out-of-domain mass Q(m) = T(-alpha(lo_D)) + T(alpha(hi_D))
    const float q0 = __fadd_ru(lo0.t.m_hi, hi0.t.p_hi);
    const float q1 = __fadd_ru(lo1.t.m_hi, hi1.t.p_hi);
    o.qhi = fminf(fmaxf(q0, q1), 1.0f);
    float qlo;
    if (mid_below(lo0, hi0))
        qlo = __fadd_rd(lo0.t.m_lo, hi0.t.p_lo);
    else if (mid_above(lo1, hi1))
        qlo = __fadd_rd(lo1.t.m_lo, hi1.t.p_lo);
    else
        qlo = g.qmin_lo;
    o.qlo = fminf(qlo, 1.0f);
    o.tw = first >= 0 ? last - first + 1 : 0;
    o.f0 = first >= 0 ? first : 0;
    o.M = M;
    o.SW = mid;
    o.O = O;
    return o;
}

// setup_fp32: one warp per 32/n rows of one build, one lane per (row,
// dimension). Each lane builds its dimension's table; the lanes of a row then
// exchange their maxima and sums by shuffles and each finishes its entry of
// the record: the pruning threshold (a child t of a node with product P
// survives iff RU(RU(P U[t]) R') >= cutoff, R' the product of the later
// dimensions' largest factors grown by 2^-18 to cover the rounding of the
// rest of the chain; cp is the least such child product). The lane of
// dimension 0 also writes the row's sink bounds and the mass of the targets
// outside the window box (FP64, outward rounding), unless the row outputs
// are null (records rebuilt for an emit pass).
__global__ void __launch_bounds__(256, 3)
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
        if (act) {
            float2 *ul = reinterpret_cast<float2 *>(rr + 32 * n) + D.dim[d].rec_off;
            o = setup_dim(D, rl, d, ul, status);
        }
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
                acc = __dadd_ru(__dmul_ru(acc, __dadd_ru((double)SWk, (double)Ok)),
                                __dmul_ru(pre, (double)Ok));
                pre = __dmul_ru(pre, (double)SWk);
            }
        }
        if (!act) continue;
        const float cut = D.cutoff32;
        RecDim rd;
        rd.tw = o.tw;
        rd.tb = D.dim[d].rec_off + o.f0;
        rd.cb = (o.a + o.f0) * D.dim[d].stride;
        rd.magic = o.tw > 1 ? (uint32_t)((0x100000000ull + (unsigned)o.tw - 1) / (unsigned)o.tw) : 0u;
        rd.cp = 0.0f;
        if (cut > 0.0f) rd.cp = (d == n - 1) ? cut : threshold(cut, __fmul_ru(R, kGrow18));
        rd.SR = SR;
        rd.stride = D.dim[d].stride;
        rd.lay = (o.tw >= 1 && o.tw <= 32)
                     ? ((32 / o.tw) | (((IMPACT_WALK_CAP / o.tw) * o.tw) << 16)) : 0;
        reinterpret_cast<RecDim *>(rr)[d] = rd;
        if (d == 0 && trunc) {
            const int64_t row = B->row_begin[q] + rl;   // global row
            sink_lo[row] = fmax(__dsub_rd(1.0, pin_up), 0.0);
            sink_up[row] = fmin(__dsub_ru(1.0, pin_dn), 1.0);
            trunc[row] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// the walk
// ---------------------------------------------------------------------------

constexpr int kCap = IMPACT_WALK_CAP;      // nodes per level list (one chunk)
constexpr int kClaimBytes = 32;            // per warp: the claimed row range, rows per claim
constexpr int kTrimMin = 512;              // emit: candidates of a chunk worth trimming its table for

// Warp shared memory: two record buffers of the batch's largest record (the
// row being walked and the next one, copied in meanwhile), then the work
// space (offsets fixed per problem by leaf_cap):
//   h      RecDim[n]                 the row record's per-dimension entries
//   ul     (U, L) x tsum_cap         the record's window tables, right after
//   work   (n - 2) x (kCap + 1) x 12 B  node lists of levels 0..n-3
//   leaf   3 x (leaf_cap + 1) words  the staged leaf table (see Leaf), and
//          5 x (leaf_cap + 1) words  the count pass's sorted form and sums, or
//                                    the emit pass's table trimmed per chunk
struct WarpMem {
    RecDim *h;
    float2 *ul;
    unsigned char *work;
    float *leaf;
    int leaf_cap;
};

__host__ __device__ constexpr int align16(int x) { return (x + 15) & ~15; }

// Node lists of levels 0..n-3, padded to 16 bytes: the warp blocks are laid
// end to end and each starts with 16-byte record copies.
__host__ __device__ inline int list_bytes(int n) { return align16((n > 2 ? n - 2 : 0) * (kCap + 1) * 12); }

__device__ __forceinline__ WarpMem carve(unsigned char *work, unsigned char *rec, const ImpactDesc &D)
{
    WarpMem m;
    m.h = reinterpret_cast<RecDim *>(rec);
    m.ul = reinterpret_cast<float2 *>(rec + 32 * D.n);
    m.work = work;
    m.leaf = reinterpret_cast<float *>(m.work + list_bytes(D.n));
    m.leaf_cap = D.leaf_cap;
    return m;
}

// Level k node list: P (RU product of upper factors), Pl (RD product of lower
// factors), col (column of the prefix).
struct NodeList {
    float *P, *Pl;
    int *col;
};

__device__ __forceinline__ NodeList node_list(unsigned char *work, int k)
{
    NodeList L;
    // kCap nodes and one spare slot that takes the stores of the lanes
    // whose candidate was not kept (stores without a branch)
    unsigned char *b = work + (size_t)k * (kCap + 1) * 12;
    L.P = reinterpret_cast<float *>(b);
    L.Pl = reinterpret_cast<float *>(b + (kCap + 1) * 4);
    L.col = reinterpret_cast<int *>(b + (kCap + 1) * 8);
    return L;
}

// Per-lane partial sums of the count walk (rounded outward, FP32): pairs
// kept, upper-bound mass of the dropped in-window targets, and the sums of
// the kept pairs' upper and lower bounds (row checks). All terms are
// non-negative, so the sums are bounds with a relative excess of at most a
// few units of 2^-23.
struct CountAcc {
    int cnt = 0;
    float drop = 0.0f, sup = 0.0f, slo = 0.0f;
};

// Where the emit walk writes: the row's len pairs, the arrays offset to its
// first pair.
struct EmitOut {
    int32_t *col;
    float *lo, *up;
    int len;
};

// The leaf table of a row: the last two dimensions m = n - 2 and l = n - 1
// (dimension 0 alone when n = 1) as one list of entries j = a * tw_l + b in C
// order: bu[j] = RU(U_m[a] U_l[b]), bl[j] = RD(L_m[a] L_l[b]) and the column
// offset bc[j] = cb_m + a stride_m + cb_l + b. For the count pass also the
// entries sorted by bu descending (su, with their bl in sl) and the sums
// pu[k] = RU sum of su[0..k), pl[k] = RD sum of sl[0..k), sf[k] = RU sum of
// su[k..nb). Staged when nb <= leaf_cap, else evaluated where needed.
struct Leaf {
    float tot_u, tot_l;   // count pass: RU sum of bu and RD sum of bl over all entries
    int nb;        // entries
    int tw_l;      // width of the last dimension (b runs fastest)
    uint32_t magic_l;
    bool staged;
    bool sorted;          // count pass: su, sl, pu, pl, sf are built
    uint32_t magic_nb;    // ceil(2^32 / nb) when 1 < nb <= 4096, for the emit's flat layout
    float *bu, *bl, *su, *sl, *pu, *pl, *sf;
    int *bc;
};

__device__ __forceinline__ Leaf leaf_of(const WarpMem &S, int n)
{
    Leaf f;
    const RecDim &hl = S.h[n - 1];
    f.tw_l = hl.tw;
    f.magic_l = hl.magic;
    f.nb = n >= 2 ? S.h[n - 2].tw * hl.tw : hl.tw;
    f.staged = f.nb <= S.leaf_cap;
    f.sorted = false;
    f.magic_nb = (f.nb > 1 && f.nb <= 4096)
                     ? (uint32_t)((0x100000000ull + (unsigned)f.nb - 1) / (unsigned)f.nb) : 0u;
    const int c = S.leaf_cap + 1;
    f.bu = S.leaf;
    f.bl = f.bu + c;
    f.bc = reinterpret_cast<int *>(f.bl + c);
    f.su = reinterpret_cast<float *>(f.bc + c);
    f.sl = f.su + c;
    f.pu = f.sl + c;
    f.pl = f.pu + c;
    f.sf = f.pl + c;
    return f;
}

// Entry j of the leaf table, evaluated from the record's tables.
struct LeafEntry {
    float u, l;
    int c;
};

__device__ __forceinline__ LeafEntry leaf_eval(const WarpMem &S, int n, const Leaf &f, int j)
{
    const RecDim &hl = S.h[n - 1];
    LeafEntry e;
    if (n == 1) {
        const float2 v = S.ul[hl.tb + j];
        e.u = v.x;
        e.l = v.y;
        e.c = hl.cb + j;
        return e;
    }
    const RecDim &hm = S.h[n - 2];
    const int a = f.tw_l > 1 ? (int)__umulhi((uint32_t)j, f.magic_l) : j;
    const int b = j - a * f.tw_l;
    const float2 vm = S.ul[hm.tb + a], vl = S.ul[hl.tb + b];
    e.u = __fmul_ru(vm.x, vl.x);
    e.l = __fmul_rd(vm.y, vl.y);
    e.c = hm.cb + a * hm.stride + hl.cb + b;
    return e;
}

template <bool STAGED>
__device__ __forceinline__ LeafEntry leaf_at(const WarpMem &S, int n, const Leaf &f, int j)
{
    if (!STAGED) return leaf_eval(S, n, f, j);
    return LeafEntry{f.bu[j], f.bl[j], f.bc[j]};
}

// Inclusive warp scans of a lane's value with directed rounding (a fixed
// association: the same bits whatever ran before).
__device__ __forceinline__ float scan_ru(float x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x = __fadd_ru(x, y);
    }
    return x;
}
__device__ __forceinline__ float scan_rd(float x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x = __fadd_rd(x, y);
    }
    return x;
}

// Stages the leaf table of a row (and, for the count pass, its sorted form
// and sums) when it fits.
template <bool COUNT>
__device__ void leaf_build(const WarpMem &S, int n, Leaf &f, int lane, float cut)
{
    float su_l = 0.0f, sl_l = 0.0f;   // this lane's part of the totals
    for (int j = lane; j < f.nb; j += 32) {
        const LeafEntry e = leaf_eval(S, n, f, j);
        if (f.staged) {
            f.bu[j] = e.u;
            f.bl[j] = e.l;
            f.bc[j] = e.c;
        }
        su_l = __fadd_ru(su_l, e.u);
        sl_l = __fadd_rd(sl_l, e.l);
    }
    __syncwarp();
    if (!COUNT) return;
    if (!(cut > 0.0f)) {   // the totals serve the dense count only
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            su_l = __fadd_ru(su_l, __shfl_xor_sync(0xffffffffu, su_l, o));
            sl_l = __fadd_rd(sl_l, __shfl_xor_sync(0xffffffffu, sl_l, o));
        }
        f.tot_u = __shfl_sync(0xffffffffu, su_l, 0);
        f.tot_l = __shfl_sync(0xffffffffu, sl_l, 0);
    }
    // a row of at most two dimensions has one parent (the root): testing
    // its entries directly costs less than sorting them
    if (!f.staged || !(cut > 0.0f) || n <= 2) return;
    f.sorted = true;
    if (f.nb <= 32) {
        // one entry per lane: a bitonic sorting network over the warp puts
        // the entry of rank r (bu descending, ties by index) in lane r, then
        // scans in registers give the sums. The sort key is the bits of bu
        // inverted (bu >= 0, so its bits grow with it) above the index:
        // ascending keys are bu descending, ties by index; lanes past the
        // table hold the largest key and sort last.
        const bool in = lane < f.nb;
        unsigned long long key = ~0ull;
        if (in)
            key = ((unsigned long long)(~__float_as_uint(f.bu[lane])) << 32) | (unsigned)lane;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                const unsigned long long pk = __shfl_xor_sync(0xffffffffu, key, jj);
                const bool want_first = ((lane & jj) == 0) == ((lane & k) == 0);
                if (want_first != (key < pk)) key = pk;
            }
        }
        const float u = in ? __uint_as_float(~(unsigned)(key >> 32)) : 0.0f;
        const float lv = in ? f.bl[(int)(key & 0xffffffffu)] : 0.0f;
        const float ux = u;
        const float iu = scan_ru(ux, lane);
        const float il = scan_rd(lv, lane);
        float su_ = ux;   // suffix sums, rounded up
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_down_sync(0xffffffffu, su_, o);
            if (lane + o < 32) su_ = __fadd_ru(su_, y);
        }
        if (lane < f.nb) {
            f.su[lane] = u;
            f.pu[lane + 1] = iu;
            f.pl[lane + 1] = il;
            f.sf[lane] = su_;
        }
        if (lane == 0) {
            f.pu[0] = 0.0f;
            f.pl[0] = 0.0f;
            f.sf[f.nb] = 0.0f;
        }
        __syncwarp();
        return;
    }
    // rank of entry j by bu descending (ties by index): its sorted position
    for (int j = lane; j < f.nb; j += 32) {
        const float u = f.bu[j];
        int r = 0;
        for (int i = 0; i < f.nb; ++i) {
            const float v = f.bu[i];
            r += (v > u) || (v == u && i < j);
        }
        f.su[r] = u;
        f.sl[r] = f.bl[j];
    }
    __syncwarp();
    // prefix sums in sorted order (pu, pl: entries 0..k-1 -> index k) and
    // suffix sums (sf[k]: entries k..nb-1), rounded outward
    float cu = 0.0f, cl = 0.0f;
    for (int k0 = 0; k0 < f.nb; k0 += 32) {
        const int k = k0 + lane;
        const float u = k < f.nb ? f.su[k] : 0.0f;
        const float l = k < f.nb ? f.sl[k] : 0.0f;
        const float iu = __fadd_ru(scan_ru(u, lane), cu);
        const float il = __fadd_rd(scan_rd(l, lane), cl);
        if (k < f.nb) {
            f.pu[k + 1] = iu;
            f.pl[k + 1] = il;
        }
        cu = __shfl_sync(0xffffffffu, iu, 31);
        cl = __shfl_sync(0xffffffffu, il, 31);
    }
    if (lane == 0) {
        f.pu[0] = 0.0f;
        f.pl[0] = 0.0f;
    }
    float cs = 0.0f;   // suffix sums, from the end
    for (int k1 = f.nb; k1 > 0; k1 -= 32) {
        const int k = k1 - 1 - lane;
        const float u = k >= 0 ? f.su[k] : 0.0f;
        const float iu = __fadd_ru(scan_ru(u, lane), cs);
        if (k >= 0) f.sf[k] = iu;
        cs = __shfl_sync(0xffffffffu, iu, 31);
    }
    if (lane == 0) f.sf[f.nb] = 0.0f;
    __syncwarp();
}

// Node of a level list, or the root (P = Pl = 1, column 0).
struct Node {
    float P, Pl;
    int c;
};

__device__ __forceinline__ Node node_at(const NodeList &L, bool root, int i)
{
    Node x{1.0f, 1.0f, 0};
    if (!root) {
        x.P = L.P[i];
        x.Pl = L.Pl[i];
        x.c = L.col[i];
    }
    return x;
}

// A narrow window (tw <= 32) is walked with each lane fixed on one target t
// of it: the warp holds floor(32 / tw) parents at a time, lane = slot * tw + t
// (slot-major, so ballot order is C order), and the lane's factors and
// column offset stay in registers. Wider windows are walked flat: candidate e
// = parent * tw + t, one lane each.
struct Lanes {
    int slots;     // parents per warp step (narrow), 0: flat
    int slot, t;   // this lane's slot and target (narrow)
    bool on;       // this lane holds a candidate slot (narrow)
};

__device__ __forceinline__ Lanes lanes_of(const RecDim &h, int lane)
{
    Lanes z{0, 0, 0, false};
    if (h.lay != 0) {
        z.slots = h.lay & 0xffff;
        z.slot = h.tw > 1 ? (int)__umulhi((uint32_t)lane, h.magic) : lane;
        z.t = lane - z.slot * h.tw;
        z.on = z.slot < z.slots;
    }
    return z;
}

// Candidates per chunk of a level list: whole parents when the window is
// narrow (the narrow walk steps over parents), else kCap.
__device__ __forceinline__ int chunk_of(const RecDim &h)
{
    return h.lay != 0 ? (h.lay >> 16) : kCap;
}

// Children of candidates [c0, c1) of the level k - 1 list (the root when
// k = 0) in dimension k, kept ones compacted into the level k list in order.
// A candidate e is (parent e / tw, target t = e mod tw of the trimmed window).
__device__ __forceinline__ int expand(const WarpMem &S, int k, int c0, int c1, int lane,
                                      CountAcc &acc, bool count)
{
    const RecDim &h = S.h[k];
    const int tw = h.tw, tb = h.tb, cb = h.cb, st = h.stride;
    const uint32_t magic = h.magic;
    const float cp = h.cp, SR = h.SR;
    const NodeList Lc = node_list(S.work, k);
    const NodeList Lp = node_list(S.work, k > 0 ? k - 1 : 0);
    const bool root = k == 0;
    const Lanes z = lanes_of(h, lane);
    int nout = 0;
    auto offer = [&](bool act, const Node &par, float2 ul, int t) {
        const float Pc = __fmul_ru(par.P, ul.x);
        const bool keep = act && Pc >= cp;
        if (count) {
            const float d = __fadd_ru(acc.drop, __fmul_ru(Pc, SR));
            acc.drop = (act && !keep) ? d : acc.drop;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int o = keep ? nout + __popc(bal & lanemask_lt()) : kCap;
        Lc.P[o] = Pc;
        Lc.Pl[o] = __fmul_rd(par.Pl, ul.y);
        Lc.col[o] = par.c + cb + t * st;
        nout += __popc(bal);
    };
    if (z.slots > 0) {   // narrow: c0, c1 are multiples of tw
        const int p0 = tw > 1 ? (int)__umulhi((uint32_t)c0, magic) : c0;
        const int p1 = tw > 1 ? (int)__umulhi((uint32_t)c1, magic) : c1;
        const float2 ul = z.on ? S.ul[tb + z.t] : make_float2(0.0f, 0.0f);
        for (int pb = p0; pb < p1; pb += z.slots) {
            const int pi = pb + z.slot;
            const bool act = z.on && pi < p1;
            offer(act, act ? node_at(Lp, root, pi) : Node{0.0f, 0.0f, 0}, ul, z.t);
        }
    } else {
        for (int e0 = c0; e0 < c1; e0 += 32) {
            const int e = e0 + lane;
            const bool act = e < c1;
            const int pi = (int)__umulhi((uint32_t)e, magic);
            const int t = e - pi * tw;
            offer(act, act ? node_at(Lp, root, pi) : Node{0.0f, 0.0f, 0},
                  act ? S.ul[tb + t] : make_float2(0.0f, 0.0f), t);
        }
    }
    __syncwarp();
    return nout;
}


// Bounds of the sum of k emitted products RU(P x_i) (up) or RD(Pl y_i) (lo)
// from the RU / RD sum s of the x_i / y_i: each rounded product is within a
// relative 2^-23 (plus 2^-149 below the normal range) of the exact one.
__device__ __forceinline__ float up_sum(float P, float s, int k)
{
    return __fmaf_ru((float)k, 1.17549435e-38f, __fmul_ru(__fmul_ru(P, s), 1.00000095f));
}
__device__ __forceinline__ float lo_sum(float Pl, float s, int k)
{
    return fmaxf(__fmaf_rd(-(float)k, 1.17549435e-38f, __fmul_rd(__fmul_rd(Pl, s), 0.99999905f)),
                 0.0f);
}

// Count pass over the leaves of npar parents (a level n - 3 list, or the
// root): pairs, their up and lo sums and the upper bound of the dropped
// mass, per lane (one lane per parent).
__device__ void leaf_count(const WarpMem &S, int n, const Leaf &f, const NodeList &Lp, bool root,
                           int npar, int lane, CountAcc &acc, float cut)
{
    const int nb = f.nb;
    if (!(cut > 0.0f)) {   // dense: every entry is kept
        for (int pi = lane; pi < npar; pi += 32) {
            const Node par = node_at(Lp, root, pi);
            acc.cnt += nb;
            acc.sup = __fadd_ru(acc.sup, up_sum(par.P, f.tot_u, nb));
            acc.slo = __fadd_rd(acc.slo, lo_sum(par.Pl, f.tot_l, nb));
        }
        return;
    }
    if (f.sorted) {
        // the kept entries of a parent are a prefix of the sorted table:
        // RU(P su[k]) >= cut for k below the count, not above it
        for (int pi = lane; pi < npar; pi += 32) {
            const Node par = node_at(Lp, root, pi);
            int lo = 0, hi = nb;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (__fmul_ru(par.P, f.su[mid]) >= cut) lo = mid + 1;
                else hi = mid;
            }
            acc.cnt += lo;
            acc.sup = __fadd_ru(acc.sup, up_sum(par.P, f.pu[lo], lo));
            acc.slo = __fadd_rd(acc.slo, lo_sum(par.Pl, f.pl[lo], lo));
            acc.drop = __fadd_ru(acc.drop, __fmul_ru(par.P, f.sf[lo]));
        }
        return;
    }
    // the root's table, or a table too wide to stage: every entry under
    // every parent
    for (int pi = 0; pi < npar; ++pi) {
        const Node par = node_at(Lp, root, pi);
        for (int j0 = 0; j0 < nb; j0 += 32) {
            const int j = j0 + lane;
            if (j < nb) {
                const LeafEntry e = leaf_eval(S, n, f, j);
                const float Pc = __fmul_ru(par.P, e.u);
                if (Pc >= cut) {
                    acc.cnt += 1;
                    acc.sup = __fadd_ru(acc.sup, Pc);
                    acc.slo = __fadd_rd(acc.slo, __fmul_rd(par.Pl, e.l));
                } else {
                    acc.drop = __fadd_ru(acc.drop, Pc);
                }
            }
        }
    }
}

// Stores that the predicate guards, without a branch around them.
__device__ __forceinline__ void st_if(bool p, int32_t *a, int32_t v)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.global.b32 [%1], %2;\n\t}"
                 :: "r"((int)p), "l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void st_if(bool p, float *a, float v)
{
    st_if(p, reinterpret_cast<int32_t *>(a), __float_as_int(v));
}

// One candidate per lane: the kept ones are compacted in lane order after the
// pairs already written and stored (predicated, no divergence).
__device__ __forceinline__ void offer_pair(bool act, const Node &par, const LeafEntry &e, float cut,
                                           const EmitOut &out, int &written)
{
    const float Pc = __fmul_ru(par.P, e.u);
    const bool keep = act && Pc >= cut;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    const int pos = written + __popc(bal & lanemask_lt());
    const bool st = keep && pos < out.len;
    st_if(st, out.col + pos, par.c + e.c);
    st_if(st, out.lo + pos, __fmul_rd(par.Pl, e.l));
    st_if(st, out.up + pos, Pc);
    written += __popc(bal);
}

// Emit pass over the leaves of npar parents: each entry of the table under
// each parent one lane (flat: candidate e = parent * nb + entry, so no lane
// idles but in the last step); kept pairs are compacted in C order and stored
// warp-contiguously. A layout that keeps the table in registers and steps
// over parents measured slower: its lanes idle when 32 is not a multiple of
// nb, and its registers cost occupancy.
template <bool ROOT, bool STAGED>
__device__ void leaf_emit(const WarpMem &S, int n, const Leaf &f, const NodeList &Lp, int npar,
                          int lane, const EmitOut &out, int &written, float cut)
{
    int nb = f.nb;
    uint32_t magic = f.magic_nb;
    // the table walked: upper, lower and column columns leaf_cap + 1 words
    // apart (the staged table, or its trimmed copy in the count pass's space)
    const float *tu = f.bu;
    const int cs = S.leaf_cap + 1;
    if (STAGED && !ROOT && cut > 0.0f && npar * nb >= kTrimMin) {
        // entries that no parent of these can keep: RU(P x) is monotone in P,
        // so an entry below the cutoff under the largest P is below it under
        // every P. The rest, in C order, form the table walked below; the
        // pairs are the same. (A pass over the table and a division: worth it
        // only when the parents and the table are large.)
        float pm = 0.0f;
        for (int pi = lane; pi < npar; pi += 32) pm = fmaxf(pm, node_at(Lp, ROOT, pi).P);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pm = fmaxf(pm, __shfl_xor_sync(0xffffffffu, pm, o));
        float *const su = f.su;
        int nt = 0;
        for (int j0 = 0; j0 < f.nb; j0 += 32) {
            const int j = j0 + lane;
            const float u = j < f.nb ? f.bu[j] : 0.0f;
            const bool k = j < f.nb && __fmul_ru(pm, u) >= cut;
            const unsigned bal = __ballot_sync(0xffffffffu, k);
            if (k) {
                const int o = nt + __popc(bal & lanemask_lt());
                su[o] = u;
                su[o + cs] = f.bl[j];
                su[o + 2 * cs] = f.bu[j + 2 * cs];   // the column's bits
            }
            nt += __popc(bal);
        }
        __syncwarp();
        if (nt == 0) return;
        nb = nt;
        magic = nt > 1 ? 0xffffffffu / (unsigned)nt + 1u : 0u;   // ceil(2^32 / nt)
        tu = su;
    }
    auto entry = [&](int j) -> LeafEntry {
        if (!STAGED) return leaf_eval(S, n, f, j);
        return LeafEntry{tu[j], tu[j + cs], __float_as_int(tu[j + 2 * cs])};
    };
    // every lane computes, the kept ones store (predicated, no divergence)
    auto offer = [&](bool act, const Node &par, const LeafEntry &e) {
        offer_pair(act, par, e, cut, out, written);
    };
    if (ROOT || nb <= 4096) {
        // the division is exact for e < 64 nb, nb <= 4096; lanes past the end
        // read the last candidate and store nothing
        const int total = npar * nb;
        int e0 = 0;
        // two candidates per lane and step, both loaded before either ballot
        for (; e0 + 32 < total; e0 += 64) {
            const int ea = e0 + lane, eb = min(e0 + 32 + lane, total - 1);
            const int pa = (ROOT || nb == 1) ? (ROOT ? 0 : ea) : (int)__umulhi((uint32_t)ea, magic);
            const int pb = (ROOT || nb == 1) ? (ROOT ? 0 : eb) : (int)__umulhi((uint32_t)eb, magic);
            const Node node_a = node_at(Lp, ROOT, pa), node_b = node_at(Lp, ROOT, pb);
            const LeafEntry leaf_a = entry(ea - pa * nb);
            const LeafEntry leaf_b = entry(eb - pb * nb);
            offer(true, node_a, leaf_a);
            offer(e0 + 32 + lane < total, node_b, leaf_b);
        }
        for (; e0 < total; e0 += 32) {
            const int e = min(e0 + lane, total - 1);
            const int pi = (ROOT || nb == 1) ? (ROOT ? 0 : e) : (int)__umulhi((uint32_t)e, magic);
            const int j = e - pi * nb;
            offer(e0 + lane < total, node_at(Lp, ROOT, pi), entry(j));
        }
        return;
    }
    for (int pi = 0; pi < npar; ++pi) {
        const Node par = node_at(Lp, ROOT, pi);
        for (int j0 = 0; j0 < nb; j0 += 32) {
            const int j = min(j0 + lane, nb - 1);
            offer(j0 + lane < nb, par, entry(j));
        }
    }
}

// Walks one row whose record is in S: levels 0..n-3 as node lists, depth
// first over chunks, the leaf table under every chunk of the deepest list.
// Returns false if the step guard ran out (a broken invariant, reported as
// an error).
template <bool EMIT>
__device__ bool walk_row(const WarpMem &S, int n, const Leaf &f, int lane, CountAcc &acc,
                         const EmitOut &out, int &written, float cut)
{
    if (n <= 2) {
        if (EMIT) {
            if (f.staged) leaf_emit<true, true>(S, n, f, node_list(S.work, 0), 1, lane, out, written, cut);
            else leaf_emit<true, false>(S, n, f, node_list(S.work, 0), 1, lane, out, written, cut);
        }
        else leaf_count(S, n, f, node_list(S.work, 0), true, 1, lane, acc, cut);
        return true;
    }
    auto leaves = [&](const NodeList &Lp, int npar) {
        if (EMIT) {
            if (f.staged) leaf_emit<false, true>(S, n, f, Lp, npar, lane, out, written, cut);
            else leaf_emit<false, false>(S, n, f, Lp, npar, lane, out, written, cut);
        }
        else leaf_count(S, n, f, Lp, false, npar, lane, acc, cut);
    };
    const int last = n - 3;   // deepest list level
    // every step fills a list, leaves one or runs the leaves of one: bound
    // them by the candidates of every level (loose, overflow-safe)
    int64_t guard = 16, prod = 1;
    for (int k = 0; k <= last; ++k) {
        prod = min(prod * (int64_t)S.h[k].tw, (int64_t)1 << 40);
        guard += 8 * (int64_t)(k + 1) * (1 + prod / kCap);
    }
    int my_cur = 0, my_sz = 0;   // lane k: next candidate of level k, size of list k
    int k = 0;
    while (true) {
        if (--guard < 0) return false;
        if (k == last + 1) {
            leaves(node_list(S.work, last), __shfl_sync(0xffffffffu, my_sz, last));
            k = last;
            continue;
        }
        const int npar = k == 0 ? 1 : __shfl_sync(0xffffffffu, my_sz, k - 1);
        const int cur = __shfl_sync(0xffffffffu, my_cur, k);
        const int total = npar * S.h[k].tw;
        if (cur >= total) {
            if (k == 0) break;
            --k;
            continue;
        }
        const int end = min(cur + chunk_of(S.h[k]), total);
        const int nout = expand(S, k, cur, end, lane, acc, !EMIT);
        if (lane == k) {
            my_cur = end;
            my_sz = nout;
        }
        if (lane == k + 1) my_cur = 0;
        ++k;
    }
    return true;
}
// ---------------------------------------------------------------------------
// row offsets by decoupled look-back, and the FP64 row terms
// ---------------------------------------------------------------------------

// Per-row look-back word: flag (bits 62-63: 0 not yet counted, 1 count
// only, 2 inclusive prefix) and value (bits 0-61).
constexpr unsigned long long kLbAgg = 1ull << 62;
constexpr unsigned long long kLbIncl = 2ull << 62;
constexpr unsigned long long kLbVal = (1ull << 62) - 1;

// Publishes the row's pair count and returns the number of pairs in the
// rows before it. A row waits only for rows that warps took before it from
// the ascending row counter; those are running and publish their counts
// without waiting on anything, so every wait ends. The wait is still bounded
// (spin_limit sleeps): on expiry, or once another warp has given up (`abort`),
// it sets the timeout status and returns false, and the row publishes no
// prefix (the rows after it give up in turn).
__device__ bool lookback(unsigned long long *lb, int64_t row, int64_t cnt, int lane,
                         unsigned *abort_flag, uint32_t *status, int spin_limit, bool stall,
                         int64_t &prefix)
{
    volatile unsigned long long *v = lb;
    volatile unsigned *ab = abort_flag;
    prefix = 0;
    if (lane == 0 && !stall) v[row] = (row == 0 ? +kLbIncl : +kLbAgg) | (unsigned long long)cnt;
    if (row == 0) return true;
    int64_t j = row - 1;   // window of rows j - 31 .. j, lane i at j - i
    int spins = 0;
    while (true) {
        const int64_t r = j - lane;
        unsigned long long w = +kLbIncl;   // before row 0: prefix 0
        if (r >= 0) w = v[r];
        const unsigned flag = (unsigned)(w >> 62);
        const unsigned incl = __ballot_sync(0xffffffffu, flag == 2u);
        const unsigned none = __ballot_sync(0xffffffffu, flag == 0u);
        // lanes up to the nearest inclusive prefix (all 32 if there is none)
        const unsigned upto = incl ? ((incl & (0u - incl)) << 1) - 1u : 0xffffffffu;
        if (none & upto) {
            int give_up = 0;
            if (lane == 0) give_up = (++spins > spin_limit) || (*ab != 0u);
            give_up = __shfl_sync(0xffffffffu, give_up, 0);
            if (give_up) {
                if (lane == 0) {
                    atomicOr(status, IMPACT_STATUS_TIMEOUT);
                    atomicExch(abort_flag, 1u);
                }
                return false;
            }
            __nanosleep(100);
            continue;
        }
        long long s = ((upto >> lane) & 1u) ? (long long)(w & kLbVal) : 0ll;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        prefix += s;
        if (incl) break;
        j -= 32;
    }
    if (lane == 0 && !stall) v[row] = kLbIncl | (unsigned long long)(prefix + cnt);
    return true;
}


__device__ __forceinline__ float warp_sum_ru(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = __fadd_ru(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
__device__ __forceinline__ float warp_sum_rd(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = __fadd_rd(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// ---------------------------------------------------------------------------
// the walk kernel
// ---------------------------------------------------------------------------

// 16-byte asynchronous copy global -> shared (both 16-byte aligned), and its
// group fences.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The problem of global row x, searched from problem q (rows only grow along
// a warp's sequence).
__device__ __forceinline__ int next_problem(const int64_t *__restrict__ begin, int count, int q,
                                            int64_t x)
{
    if (q + 1 >= count || begin[q + 1] > x) return q;
    return find_problem(begin, count, x);
}

enum { MODE_COUNT = 0, MODE_EMIT = 1, MODE_FUSED = 2 };

struct WalkArgs {
    const BatchIndex *B;
    int warp_smem;           // shared-memory bytes of one warp
    int row_block;           // rows a warp claims per atomic
    int rec_max;             // bytes of one record buffer
    int64_t *row_ptr;        // COUNT: per-row counts; FUSED: row pointers; EMIT: read
    int32_t *col;
    float *lo, *up;
    double *trunc;           // COUNT / FUSED: outside-window mass in, full truncated mass out
    double *sink_lo, *sink_up;
    uint32_t *flags;
    uint32_t *status;        // [0] status bits, [1] look-back abort flag
    unsigned long long *lb;  // FUSED: look-back words, zeroed, one per row
    int64_t capacity;        // pairs the output arrays hold (< 0: unchecked)
    int64_t total_at;        // EMIT: index of the total in row_ptr
    int spin_limit;          // look-back sleeps before giving up
    int64_t row_begin;       // the launch covers global rows [row_begin, row_end)
    int64_t row_end;
    int64_t stall_row;       // fault injection: this row never publishes (-1: none)
    int64_t fault_row;       // fault injection: this row's checks see a bad sum (-1: none)
    int64_t guard_row;       // fault injection: this row's step guard starts spent (-1: none)
};

template <int MODE>
__global__ void __launch_bounds__(IMPACT_TREE_WARPS_MAX * 32) walk_fp32(const WalkArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool kCount = MODE != MODE_EMIT;
    constexpr bool kEmit = MODE != MODE_COUNT;
    const int lane = threadIdx.x & 31;
    unsigned char *const wbase = smem_raw + (size_t)(threadIdx.x >> 5) * A.warp_smem;
    const BatchIndex *B = A.B;
    if (MODE == MODE_EMIT && A.capacity >= 0 && A.row_ptr[A.total_at] > A.capacity) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(A.status, IMPACT_STATUS_CAPACITY);
        return;
    }
    unsigned long long *const next_row = B->next_row + (MODE == MODE_EMIT ? 1 : 0);
    bool lb_ok = true;

    // persistent: each warp takes rows from the batch's row counter,
    // A.row_block consecutive rows per atomic (one counter serves every warp
    // of the grid: claiming short rows one by one queues the atomics), in
    // ascending order. The passes that count take them two ahead: while a
    // warp walks a row, the index of the row after the next is known and the
    // next row's record is copied (cp.async) into the warp's other record
    // buffer. The emit pass (more registers live in its walk) copies each
    // record when it starts it.
    constexpr bool kAhead = MODE != MODE_EMIT;
    const unsigned long long nrows = (unsigned long long)(A.row_end - A.row_begin);
    unsigned char *const work = wbase + (kAhead ? 2 : 1) * A.rec_max;
    // the warp's claimed rows [claim[0], claim[1]) and the rows per claim
    // (claim[2]), in the last bytes of its block (not registers: the walk
    // needs all of them)
    unsigned long long *const claim =
        reinterpret_cast<unsigned long long *>(wbase + A.warp_smem - kClaimBytes);
    if (lane == 0) {
        claim[0] = claim[1] = 0;
        claim[2] = (unsigned long long)A.row_block;
    }
    __syncwarp();
    auto take = [&]() -> unsigned long long {
        unsigned long long t = claim[0];
        if (t == claim[1]) {   // warp-uniform: every lane reads the same words
            unsigned long long c = 0;
            if (lane == 0) c = atomicAdd(next_row, claim[2]);
            t = __shfl_sync(0xffffffffu, c, 0);
            if (lane == 0) claim[1] = t + claim[2];
        }
        __syncwarp();
        if (lane == 0) claim[0] = t + 1;
        __syncwarp();
        return t;
    };
    auto fetch = [&](unsigned long long t, int &q, unsigned char *dst) {
        if (t >= nrows) return;
        const int64_t row = A.row_begin + (int64_t)t;
        q = next_problem(B->row_begin, B->count, q, row);
        const int stride = B->desc[q]->rec_stride;
        const unsigned char *src = B->rec[q] + (row - B->row_begin[q]) * (int64_t)stride;
        for (int i = lane; i < (stride >> 4); i += 32) cp_async16(dst + 16 * i, src + 16 * i);
    };
    unsigned long long t_cur = take();
    unsigned long long t_nxt = 0;
    int q_cur = 0, b = 0;
    if (kAhead) {
        t_nxt = take();
        fetch(t_cur, q_cur, wbase);
        cp_async_commit();
    }
    while (t_cur < nrows) {
        unsigned long long t_after = 0;
        int q_nxt = q_cur;
        if (kAhead) {
            t_after = take();
            fetch(t_nxt, q_nxt, wbase + (b ^ 1) * A.rec_max);
            cp_async_commit();
            cp_async_wait_prior();   // this row's record has landed
        } else {
            fetch(t_cur, q_cur, wbase);
            cp_async_commit();
            cp_async_wait_all();
        }
        __syncwarp();
        const int64_t row = A.row_begin + (int64_t)t_cur;   // global row of the batch
        const int q = q_cur;
        const ImpactDesc &D = *B->desc[q];
        const int n = D.n;
        const float cut = D.cutoff32;
        const WarpMem S = carve(work, wbase + b * A.rec_max, D);
        __syncwarp();
        bool empty = false;
        for (int k = 0; k < n; ++k) empty |= (S.h[k].tw == 0);
        Leaf f = leaf_of(S, n);
        if (!empty) leaf_build<kCount>(S, n, f, lane, cut);
        bool walked = true;
        int64_t base = 0, len = 0;
        if (kCount) {
            CountAcc acc;
            const EmitOut none{nullptr, nullptr, nullptr, 0};
            int w0 = 0;
            if (row == A.guard_row) walked = false;
            else if (!empty) walked = walk_row<false>(S, n, f, lane, acc, none, w0, cut);
            int c = walked ? acc.cnt : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            const float drop = warp_sum_ru(walked ? acc.drop : 0.0f);
            const float sup = warp_sum_ru(walked ? acc.sup : 0.0f);
            const float slo = warp_sum_rd(walked ? acc.slo : 0.0f);
            int64_t prefix = 0;
            if (MODE == MODE_FUSED) {
                lb_ok = lookback(A.lb, row, c, lane, A.status + 1, A.status, A.spin_limit,
                                 row == A.stall_row, prefix);
                if (lane == 0 && lb_ok) {
                    A.row_ptr[row] = prefix;
                    if (row == B->rows - 1) A.row_ptr[B->rows] = prefix + c;
                }
            } else if (lane == 0) {
                A.row_ptr[row] = c;   // counts; the scan turns them into row pointers
            }
            base = prefix;
            len = c;
            if (lane == 0) {
                // FP64 row terms: the dropped in-window mass joins the mass
                // outside the window box; then the row checks of Def. 3.1
                const double tr = __dadd_ru(A.trunc[row], (double)drop);
                A.trunc[row] = tr;
                if (A.flags) {
                    const double slv = A.sink_lo[row], suv = A.sink_up[row];
                    const double lo_sum = row == A.fault_row ? 2.0 : (double)slo;
                    uint32_t fl = 0;
                    if (__dadd_rd(lo_sum, slv) > 1.0) fl |= IMPACT_ROW_LO_SUM_ABOVE_ONE;
                    if (__dadd_ru(__dadd_ru((double)sup, suv), tr) < 1.0)
                        fl |= IMPACT_ROW_UP_SUM_BELOW_ONE;
                    A.flags[row] = fl;
                    if (fl) atomicOr(A.status, IMPACT_STATUS_UNSOUND);
                }
            }
        } else {
            base = A.row_ptr[row];
            len = A.row_ptr[row + 1] - base;
        }
        if (kEmit && walked && lb_ok) {
            if (base < 0 || len < 0 || (A.capacity >= 0 && base + len > A.capacity)) {
                if (lane == 0)
                    atomicOr(A.status, MODE == MODE_FUSED ? IMPACT_STATUS_CAPACITY
                                                          : IMPACT_STATUS_EMIT_MISMATCH);
            } else {
                const EmitOut out{A.col + base, A.lo + base, A.up + base, (int)len};
                CountAcc none;
                int written = 0;
                bool wok = true;
                if (row == A.guard_row) wok = false;
                else if (!empty) wok = walk_row<true>(S, n, f, lane, none, out, written, cut);
                if (lane == 0 && (!wok || written != len))
                    atomicOr(A.status, wok ? IMPACT_STATUS_EMIT_MISMATCH : IMPACT_STATUS_INTERNAL);
            }
        }
        if (lane == 0 && !walked) atomicOr(A.status, IMPACT_STATUS_INTERNAL);
        if (!lb_ok) break;   // the rows after this one cannot find their offsets
        __syncwarp();        // every lane is done with the buffer before it is refilled
        if (kAhead) {
            t_cur = t_nxt;
            q_cur = q_nxt;
            t_nxt = t_after;
            b ^= 1;
        } else {
            t_cur = take();
        }
    }
    cp_async_wait_all();
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
    return ((int64_t)32 * n + (int64_t)8 * tsum_cap + 15) / 16 * 16;
}

int walk_work_bytes(int n, int leaf_cap, bool count)
{
    return list_bytes(n) + align16((count ? 32 : 24) * (leaf_cap + 1));
}

int walk_core_bytes(int n, int tsum_cap, int leaf_cap)
{
    const int64_t b = 2 * record_stride(n, tsum_cap) + walk_work_bytes(n, leaf_cap, true);
    return (int)std::min<int64_t>(b, INT32_MAX / 2);
}

cudaError_t launch_setup_fp32(const BatchIndex *d_index, int64_t units, uint32_t *status,
                              double *sink_lo, double *sink_up, double *trunc, cudaStream_t stream)
{
    if (units <= 0) return cudaSuccess;
    const int g = occupancy_grid((const void *)setup_fp32, 256, 0, units, 256 / 32);
    setup_fp32<<<g, 256, 0, stream>>>(d_index, status, sink_lo, sink_up, trunc);
    return cudaGetLastError();
}

cudaError_t launch_walk_fp32(const BatchIndex *d_index, int64_t row_begin, int64_t row_end,
                             int rec_max, const int work_max[2], int warps, int mode,
                             const RowOutputs &o,
                             unsigned long long *lb, const WalkFaults &f, cudaStream_t stream)
{
    const int64_t rows = row_end - row_begin;
    if (rows <= 0) return cudaSuccess;
    // record buffers and warp blocks start 16-byte aligned (record strides are
    // multiples of 16)
    rec_max = (rec_max + 15) & ~15;
    const int work = work_max[mode == MODE_EMIT ? 0 : 1];
    const int warp_smem = (mode == MODE_EMIT ? 1 : 2) * rec_max + ((work + 15) & ~15) + kClaimBytes;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    warps = std::max(1, std::min({warps, IMPACT_TREE_WARPS_MAX, optin / std::max(warp_smem, 1)}));
    const int threads = warps * 32;
    const size_t smem = (size_t)warp_smem * warps;
    const void *k = mode == MODE_COUNT  ? (const void *)walk_fp32<MODE_COUNT>
                    : mode == MODE_EMIT ? (const void *)walk_fp32<MODE_EMIT>
                                        : (const void *)walk_fp32<MODE_FUSED>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    WalkArgs A;
    A.B = d_index;
    A.warp_smem = warp_smem;
    A.rec_max = rec_max;
    A.row_ptr = o.row_ptr;
    A.col = o.col;
    A.lo = (float *)o.lo;
    A.up = (float *)o.up;
    A.trunc = o.trunc;
    A.sink_lo = o.sink_lo;
    A.sink_up = o.sink_up;
    A.flags = o.flags;
    A.status = o.status;
    A.lb = lb;
    A.capacity = o.capacity;
    A.total_at = o.total_at;
    A.spin_limit = f.spin_limit > 0 ? f.spin_limit : (1 << 24);
    A.row_begin = row_begin;
    A.row_end = row_end;
    A.stall_row = f.stall_row;
    A.fault_row = f.fault_row;
    A.guard_row = f.guard_row;
    // persistent grid: as many blocks as fit at once (rows are taken dynamically)
    const int g = occupancy_grid(k, threads, smem, rows, warps);
    // rows per claim: 4 in the count pass (its rows are short: the atomics
    // cost more than the last claims' imbalance), else up to 4 while that
    // imbalance (up to 3 rows per warp) stays under 1/256 of each warp's rows
    A.row_block = mode == MODE_COUNT
                      ? 4
                      : (int)std::max<int64_t>(1, std::min<int64_t>(4, rows / ((int64_t)g * warps * 256)));
    if (mode == MODE_COUNT)
        walk_fp32<MODE_COUNT><<<g, threads, smem, stream>>>(A);
    else if (mode == MODE_EMIT)
        walk_fp32<MODE_EMIT><<<g, threads, smem, stream>>>(A);
    else
        walk_fp32<MODE_FUSED><<<g, threads, smem, stream>>>(A);
    return cudaGetLastError();
}

}  // namespace impact
