// walk_fp32.cu -- FP32-sound construction (Def. 3.1 with outward rounding,
// Sec. 4.4 cutoff, Remark 4.1 sink): one warp per row (source cell x input,
// Alg. 2: rows are independent), persistent, rows taken from an atomic
// counter in ascending order. Per row:
//
//   setup   the interval image of the cell in every dimension, the window of
//           target cells that can pass the cutoff, one erf/erfc evaluation
//           per window edge at the image's lower and upper end (edges spread
//           over the lanes), and from them the factor table of every window
//           target: U[t] >= the largest Gaussian mass of target t over the
//           image (T_max of Def. 3.1 relaxed to the image box) and L[t] <= the
//           smallest (T_min). The lanes of dimensions 0..n-1 then trim each
//           window to the targets that pass on their own, sum the mass outside
//           the trimmed windows and the out-of-domain bounds (the sink).
//   walk    the prefix tree of target cells, level by level in C order: a
//           node at level k is a prefix (t_0..t_k) with the RU-rounded
//           product P of its upper factors. The children of a list of nodes
//           are enumerated flat (candidate e = parent * width + t, one lane
//           each); a child is kept iff RU(P U[t]) can still reach the cutoff
//           under the largest factors of the later dimensions, and the warp
//           compacts the kept ones (ballot + popc) into the next level's
//           list. Lists hold at most kCap nodes: a longer expansion is taken
//           in chunks of kCap candidates, depth first, so the leaves still
//           come out in C order. At the last dimension the kept candidates
//           are the row's pairs (up = RU(P U[t]) >= cutoff).
//
// Three kernel modes share the code: COUNT (pairs per row, truncated mass,
// row checks), EMIT (pairs at given row offsets) and FUSED (both in one pass:
// each row publishes its pair count, finds its offset by a decoupled
// look-back over the rows before it, and writes its pairs).
//
// Products run left to right over the dimensions with directed rounding (up:
// round up, lo: round down) whatever the enumeration order, so a pair's value
// depends only on its row. Every lane-to-candidate assignment is a function of
// the row alone (kCap is a compile-time constant), so the per-lane partial
// sums and their fixed reduction tree give the same bits under every launch
// shape and in every batch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "impact_desc.h"
#include "kernels.h"
#include "sound_fp32.cuh"

namespace {

constexpr int kCap = IMPACT_WALK_CAP;           // nodes per level list (one chunk)
constexpr int kHdrBytes = 96 * IMPACT_MAX_DIM;  // per-dimension row header
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

// Per (row, dimension) scalars, in the warp's shared memory.
struct DimHdr {
    int a;           // first window cell
    int W;           // window width (cells)
    int eoff;        // first edge item of the dimension (setup scratch)
    int toff;        // first table entry of the window
    int tw;          // trimmed width: targets first..last that pass on their own
    int tb;          // table entry of the first trimmed target (toff + first)
    int cb;          // column of the first trimmed target: (a + first) * stride
    uint32_t magic;  // ceil(2^32 / tw): e / tw = umulhi(e, magic) for e < 2^16
    float kh, kl, err;          // kappa (cell width in erf units) pair, edge error
    float rh0, rl0, rh1, rl1;   // rho = (E_a - m)/(sigma sqrt2) at m_lo and m_hi, pairs
    float M;         // largest U over the trimmed window
    float SW;        // sum of U over the trimmed window (rounded up)
    float O;         // mass outside the trimmed window (rounded up)
    float qlo, qhi;  // out-of-domain mass bounds
    float cp;        // least child product whose subtree can still reach the cutoff
    float SR;        // RU product of the later dimensions' SW
    int stride;      // column stride of the dimension (C order)
    int pad;
};
static_assert(sizeof(DimHdr) == 96, "DimHdr layout");

__device__ __forceinline__ EdgePt edge_at(const DimHdr &h, int k, bool hi_end)
{
    EdgePt e;
    sound::alpha_point(k, h.kh, h.kl, h.err, hi_end ? h.rh1 : h.rh0, hi_end ? h.rl1 : h.rl0, e.a,
                       e.da);
    e.t = sound::tails(e.a, e.da);
    return e;
}

// Setup scratch: one item per window edge (W + 1 per dimension) plus the two
// domain edges, each evaluated at both image ends; structure of arrays.
struct EdgeSoA {
    float *f;   // 12 arrays of `cap` floats
    int cap;
    __device__ __forceinline__ void put(int i, int end, const EdgePt &p) const
    {
        float *b = f + (end * 6) * cap + i;
        b[0] = p.a;
        b[cap] = p.da;
        b[2 * cap] = p.t.p_lo;
        b[3 * cap] = p.t.p_hi;
        b[4 * cap] = p.t.m_lo;
        b[5 * cap] = p.t.m_hi;
    }
    __device__ __forceinline__ EdgePt get(int i, int end) const
    {
        const float *b = f + (end * 6) * cap + i;
        EdgePt p;
        p.a = b[0];
        p.da = b[cap];
        p.t.p_lo = b[2 * cap];
        p.t.p_hi = b[3 * cap];
        p.t.m_lo = b[4 * cap];
        p.t.m_hi = b[5 * cap];
        return p;
    }
};

// Warp shared memory: header, factor table (U, L) pairs, and a work area that
// first holds the setup scratch and then the node lists of levels 0..n-2.
struct WarpMem {
    DimHdr *h;
    float2 *ul;
    unsigned char *work;
};

__device__ __forceinline__ WarpMem carve(unsigned char *base, const ImpactDesc &D)
{
    WarpMem m;
    m.h = reinterpret_cast<DimHdr *>(base);
    m.ul = reinterpret_cast<float2 *>(base + kHdrBytes);
    m.work = base + kHdrBytes + (((size_t)8 * D.tsum_cap + 15) & ~(size_t)15);
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
    unsigned char *b = work + (size_t)k * kCap * 12;
    L.P = reinterpret_cast<float *>(b);
    L.Pl = reinterpret_cast<float *>(b + kCap * 4);
    L.col = reinterpret_cast<int *>(b + kCap * 8);
    return L;
}

// What the setup tells the walk about a row (the same in every lane).
struct RowTerms {
    bool ok;      // every window fit the planner's bound
    bool empty;   // some dimension keeps no target: the row has no pairs
};

// Lane d < n: the interval image of the cell in dimension d (affine sign
// split or unicycle trig ranges from host tables, or the caller's images),
// the window [a, a + W) of targets that can pass the cutoff (every target
// outside lies more than delta beyond the image), and rho = (E_a - m) /
// (sigma sqrt2) at both image ends as FP32 pairs. False if the window
// exceeds the planner's bound wcap.
__device__ bool dim_window(const ImpactDesc &D, int64_t row, int d, DimHdr &h)
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

// Setup of one row by the whole warp (see the file comment). Fills the
// header and the (U, L) table of every dimension.
__device__ RowTerms row_setup(const ImpactDesc &D, const WarpMem &S, int64_t row, int lane)
{
    const int n = D.n;
    RowTerms rt;
    // 1. windows (lane d), then offsets of the edge items and table entries
    bool ok = true;
    int W = 0;
    if (lane < n) {
        DimHdr &h = S.h[lane];
        ok = dim_window(D, row, lane, h);
        W = ok ? h.W : 0;
    }
    rt.ok = __all_sync(0xffffffffu, ok);
    rt.empty = false;
    if (!rt.ok) return rt;
    int incl = W;   // inclusive prefix of W over lanes 0..n-1
#pragma unroll
    for (int o = 1; o < IMPACT_MAX_DIM; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane < n) {
        S.h[lane].toff = incl - W;
        S.h[lane].eoff = incl - W + 3 * lane;
    }
    const int T = __shfl_sync(0xffffffffu, incl, n - 1);   // window targets of all dims
    const int E = T + 3 * n;                                // edge items
    __syncwarp();
    const EdgeSoA es{reinterpret_cast<float *>(S.work), D.edge_cap};

    // 2. edge items: k = 0..W are the window's edges a..a+W, then the
    // domain's lower and upper edge (k = -a, N - a); both image ends
    for (int i = lane; i < E; i += 32) {
        int d = 0;
#pragma unroll
        for (int k = 1; k < IMPACT_MAX_DIM; ++k)
            if (k < n && i >= S.h[k].eoff) d = k;
        const DimHdr &h = S.h[d];
        const int li = i - h.eoff;
        const int k = li <= h.W ? li : (li == h.W + 1 ? -h.a : D.dim[d].N - h.a);
        es.put(i, 0, edge_at(h, k, false));
        es.put(i, 1, edge_at(h, k, true));
    }
    __syncwarp();

    // 3. factor table of every window target: U >= T_max factor, L <= T_min
    // factor, from the tails of its two edges at the two image ends
    for (int i = lane; i < T; i += 32) {
        int d = 0;
#pragma unroll
        for (int k = 1; k < IMPACT_MAX_DIM; ++k)
            if (k < n && i >= S.h[k].toff) d = k;
        const DimHdr &h = S.h[d];
        const int e = h.eoff + (i - h.toff);
        const EdgePt c0 = es.get(e, 0), e0 = es.get(e + 1, 0);
        const EdgePt c1 = es.get(e, 1), e1 = es.get(e + 1, 1);
        float U, L;
        if (mid_below(c0, e0)) {            // target midpoint <= m_lo
            U = sound::cell_hi(c0.a, c0.t, e0.a, e0.t);
            L = sound::cell_lo(c1.a, c1.t, e1.a, e1.t);
        } else if (mid_above(c1, e1)) {     // target midpoint >= m_hi
            U = sound::cell_hi(c1.a, c1.t, e1.a, e1.t);
            L = sound::cell_lo(c0.a, c0.t, e0.a, e0.t);
        } else {                            // midpoint may be inside
            U = D.dim[d].plateau_hi;
            L = fminf(sound::cell_lo(c0.a, c0.t, e0.a, e0.t),
                      sound::cell_lo(c1.a, c1.t, e1.a, e1.t));
        }
        S.ul[i] = make_float2(U, L);
    }
    __syncwarp();

    // 4. lane d: trim the window to the targets that pass on their own, sums
    // inside and outside it (rounded up, fixed order), out-of-domain bounds
    const float cut = D.cutoff32;
    float M = 0.0f, SW = 0.0f, O = 0.0f, qlo = 0.0f, qhi = 0.0f;
    int tw = 0;
    if (lane < n) {
        DimHdr &h = S.h[lane];
        const ImpactDim &g = D.dim[lane];
        int first = -1, last = -1;
        float pre = 0.0f, mid = 0.0f, post = 0.0f;
        for (int k = 0; k < h.W; ++k) {
            const float U = S.ul[h.toff + k].x;
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
        }
        O = __fadd_ru(pre, post);
        const EdgePt w0 = es.get(h.eoff, 0);                 // edge a at m_lo
        const EdgePt c1 = es.get(h.eoff + h.W, 1);           // edge a + W at m_hi
        const EdgePt lo0 = es.get(h.eoff + h.W + 1, 0), hi0 = es.get(h.eoff + h.W + 2, 0);
        const EdgePt lo1 = es.get(h.eoff + h.W + 1, 1), hi1 = es.get(h.eoff + h.W + 2, 1);
        if (h.a > 0)   // cells 0..a-1 lie left of the image: their mass at m_lo
            O = __fadd_ru(O, sound::cell_hi(lo0.a, lo0.t, w0.a, w0.t));
        if (h.a + h.W < g.N)   // cells right of the window: their mass at m_hi
            O = __fadd_ru(O, sound::cell_hi(c1.a, c1.t, hi1.a, hi1.t));
        // out-of-domain mass Q(m) = T(-alpha(lo_D)) + T(alpha(hi_D))
        const float q0 = __fadd_ru(lo0.t.m_hi, hi0.t.p_hi);
        const float q1 = __fadd_ru(lo1.t.m_hi, hi1.t.p_hi);
        qhi = fminf(fmaxf(q0, q1), 1.0f);
        if (mid_below(lo0, hi0))
            qlo = __fadd_rd(lo0.t.m_lo, hi0.t.p_lo);
        else if (mid_above(lo1, hi1))
            qlo = __fadd_rd(lo1.t.m_lo, hi1.t.p_lo);
        else
            qlo = g.qmin_lo;
        qlo = fminf(qlo, 1.0f);
        tw = first >= 0 ? last - first + 1 : 0;
        const int f0 = first >= 0 ? first : 0;
        SW = mid;
        h.tw = tw;
        h.tb = h.toff + f0;
        h.cb = (h.a + f0) * g.stride;
        h.stride = g.stride;
        h.magic = tw > 1 ? (uint32_t)((0x100000000ull + (unsigned)tw - 1) / (unsigned)tw) : 0u;
        h.M = M;
        h.SW = SW;
        h.O = O;
        h.qlo = qlo;
        h.qhi = qhi;
    }
    rt.empty = __any_sync(0xffffffffu, lane < n && tw == 0);

    // 5. each lane of dimension d: the RU products of the later dimensions'
    // largest factors and window sums, which give its pruning threshold
    // (the sink and the mass outside the window box are combined in FP64
    // later, per row, by the epilogue)
    float R = 1.0f, SR = 1.0f;
#pragma unroll
    for (int k = 0; k < IMPACT_MAX_DIM; ++k) {
        if (k < n) {
            const float Mk = __shfl_sync(0xffffffffu, M, k);
            const float SWk = __shfl_sync(0xffffffffu, SW, k);
            if (k > lane) {
                R = __fmul_ru(R, Mk);
                SR = __fmul_ru(SR, SWk);
            }
        }
    }
    if (lane < n) {
        float cp = 0.0f;
        if (cut > 0.0f) cp = (lane == n - 1) ? cut : threshold(cut, __fmul_ru(R, kGrow18));
        S.h[lane].cp = cp;
        S.h[lane].SR = SR;
    }
    __syncwarp();
    return rt;
}

// ---------------------------------------------------------------------------
// the walk
// ---------------------------------------------------------------------------

// Per-lane partial sums of the count walk (rounded outward, FP32): pairs
// kept, upper-bound mass of the dropped in-window targets, and the sums of
// the kept pairs' upper and lower bounds (row checks). All terms are
// non-negative, so the sums are bounds with a relative excess of at most a
// few units of 2^-23.
struct CountAcc {
    int cnt = 0;
    float drop = 0.0f, sup = 0.0f, slo = 0.0f;
};

// Where the emit walk writes: pairs [base, base + len) of the output arrays.
struct EmitOut {
    int32_t *col;
    float *lo, *up;
    int64_t base, len;
};

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

__device__ __forceinline__ Lanes lanes_of(int tw, uint32_t magic, int lane)
{
    Lanes z{0, 0, 0, false};
    if (tw <= 32) {
        z.slots = 32 / tw;
        z.slot = tw > 1 ? (int)__umulhi((uint32_t)lane, magic) : lane;
        z.t = lane - z.slot * tw;
        z.on = z.slot < z.slots;
    }
    return z;
}

// Candidates per chunk of a level list: whole parents when the window is
// narrow (the narrow walk steps over parents), else kCap.
__device__ __forceinline__ int chunk_of(int tw)
{
    return tw <= 32 ? (kCap / tw) * tw : kCap;
}

// Children of candidates [c0, c1) of the level k - 1 list (the root when
// k = 0) in dimension k, kept ones compacted into the level k list in order.
// A candidate e is (parent e / tw, target t = e mod tw of the trimmed window).
__device__ __forceinline__ int expand(const WarpMem &S, int k, int c0, int c1, int lane,
                                      CountAcc &acc, bool count)
{
    const DimHdr &h = S.h[k];
    const int tw = h.tw, tb = h.tb, cb = h.cb, st = h.stride;
    const uint32_t magic = h.magic;
    const float cp = h.cp, SR = h.SR;
    const NodeList Lc = node_list(S.work, k);
    const NodeList Lp = node_list(S.work, k > 0 ? k - 1 : 0);
    const bool root = k == 0;
    const Lanes z = lanes_of(tw, magic, lane);
    int nout = 0;
    auto offer = [&](bool act, const Node &par, float2 ul, int t) {
        const float Pc = __fmul_ru(par.P, ul.x);
        const bool keep = act && Pc >= cp;
        if (count && act && !keep) acc.drop = __fadd_ru(acc.drop, __fmul_ru(Pc, SR));
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int o = nout + __popc(bal & lanemask_lt());
            Lc.P[o] = Pc;
            Lc.Pl[o] = __fmul_rd(par.Pl, ul.y);
            Lc.col[o] = par.c + cb + t * st;
        }
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

// The pairs under the npar nodes of the level n - 2 list (the root when
// n = 1). Count: a narrow window is walked serially by one lane per parent
// (the factors are broadcast reads, nothing is compacted); emit: the kept
// candidates are compacted and stored warp-contiguously.
template <bool EMIT>
__device__ __forceinline__ void leaf(const WarpMem &S, int n, int npar, int lane, CountAcc &acc,
                                     const EmitOut &out, int64_t &written)
{
    const DimHdr &h = S.h[n - 1];
    const int tw = h.tw, tb = h.tb, cb = h.cb;
    const uint32_t magic = h.magic;
    const float cp = h.cp;
    const NodeList Lp = node_list(S.work, n >= 2 ? n - 2 : 0);
    const bool root = n == 1;
    if (!EMIT && tw <= 32) {
        for (int p0 = 0; p0 < npar; p0 += 32) {
            const int pi = p0 + lane;
            if (pi < npar) {
                const Node par = node_at(Lp, root, pi);
                for (int t = 0; t < tw; ++t) {
                    const float2 ul = S.ul[tb + t];
                    const float Pc = __fmul_ru(par.P, ul.x);
                    if (Pc >= cp) {
                        acc.cnt += 1;
                        acc.sup = __fadd_ru(acc.sup, Pc);
                        acc.slo = __fadd_rd(acc.slo, __fmul_rd(par.Pl, ul.y));
                    } else {
                        acc.drop = __fadd_ru(acc.drop, Pc);
                    }
                }
            }
        }
        return;
    }
    auto offer = [&](bool act, const Node &par, float2 ul, int t) {
        const float Pc = __fmul_ru(par.P, ul.x);
        const bool keep = act && Pc >= cp;
        if (!EMIT) {
            if (keep) {
                acc.cnt += 1;
                acc.sup = __fadd_ru(acc.sup, Pc);
                acc.slo = __fadd_rd(acc.slo, __fmul_rd(par.Pl, ul.y));
            } else if (act) {
                acc.drop = __fadd_ru(acc.drop, Pc);
            }
        } else {
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int64_t pos = written + __popc(bal & lanemask_lt());
                if (pos < out.len) {
                    const int64_t p = out.base + pos;
                    out.col[p] = par.c + cb + t;
                    out.lo[p] = __fmul_rd(par.Pl, ul.y);
                    out.up[p] = Pc;
                }
            }
            written += __popc(bal);
        }
    };
    const Lanes z = lanes_of(tw, magic, lane);
    if (z.slots > 0) {
        const float2 ul = z.on ? S.ul[tb + z.t] : make_float2(0.0f, 0.0f);
        for (int pb = 0; pb < npar; pb += z.slots) {
            const int pi = pb + z.slot;
            const bool act = z.on && pi < npar;
            offer(act, act ? node_at(Lp, root, pi) : Node{0.0f, 0.0f, 0}, ul, z.t);
        }
    } else {
        const int total = npar * tw;
        for (int e0 = 0; e0 < total; e0 += 32) {
            const int e = e0 + lane;
            const bool act = e < total;
            const int pi = (int)__umulhi((uint32_t)e, magic);
            const int t = e - pi * tw;
            offer(act, act ? node_at(Lp, root, pi) : Node{0.0f, 0.0f, 0},
                  act ? S.ul[tb + t] : make_float2(0.0f, 0.0f), t);
        }
    }
}

// Walks one row whose setup is in S (levels 0..n-2 as node lists, depth
// first over chunks of kCap candidates, then the leaves). Returns false if
// the step guard ran out (a broken invariant, reported as an error).
template <bool EMIT>
__device__ bool walk_row(const WarpMem &S, int n, int lane, CountAcc &acc, const EmitOut &out,
                         int64_t &written)
{
    // every step advances a cursor, fills a list or leaves one: bound them by
    // the candidates of every level (a loose, overflow-safe count)
    int64_t guard = 16, prod = 1;
    for (int k = 0; k < n; ++k) {
        prod = min(prod * (int64_t)S.h[k].tw, (int64_t)1 << 40);
        guard += 8 * (int64_t)(k + 1) * (1 + prod / kCap);
    }
    int my_cur = 0, my_sz = 0;   // lane k: next candidate of level k, size of list k
    int k = 0;
    while (true) {
        if (--guard < 0) return false;
        if (k == n - 1) {
            const int npar = n == 1 ? 1 : __shfl_sync(0xffffffffu, my_sz, n - 2);
            leaf<EMIT>(S, n, npar, lane, acc, out, written);
            if (n == 1) break;
            k = n - 2;
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
        const int end = min(cur + chunk_of(S.h[k].tw), total);
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

// Rows whose FP64 terms wait in the warp's epilogue buffer: per slot the
// FP32 inputs (per dimension qlo, qhi, SW, O; the row's drop, sup, slo
// sums). Every kEpi rows one lane per row combines them in FP64, which keeps
// the scarce FP64 issue of this part at about kEpi times fewer instructions
// than combining each row in the whole warp.
constexpr int kEpi = IMPACT_WALK_EPI;
struct EpiBuf {
    float *f;       // [4 * nm + 3][kEpi]
    int64_t *row;   // [kEpi] global row
    int *nd;        // [kEpi] dimensions (0: the row failed its setup)
    int nm;         // largest n of the batch
};

__device__ __forceinline__ void epi_flush(const EpiBuf &E, int used, int lane, double *sink_lo,
                                          double *sink_up, double *trunc, uint32_t *flags,
                                          uint32_t *status, int64_t fault_row)
{
    __syncwarp();
    if (lane < used) {
        const int s = lane, nm = E.nm;
        const int64_t row = E.row[s];
        const int n = E.nd[s];
        double pin_up = 1.0, pin_dn = 1.0, acc = 0.0, pre = 1.0;
        for (int k = 0; k < n; ++k) {
            const double ql = E.f[k * kEpi + s], qh = E.f[(nm + k) * kEpi + s];
            const double sw = E.f[(2 * nm + k) * kEpi + s], o = E.f[(3 * nm + k) * kEpi + s];
            // sink: 1 - prod_k (1 - Q_k)
            pin_up = __dmul_ru(pin_up, __dsub_ru(1.0, ql));
            pin_dn = __dmul_rd(pin_dn, __dsub_rd(1.0, qh));
            // mass outside the window box, partitioned by the first dimension
            // that leaves its window: sum_k prod_{i<k} SW_i O_k prod_{i>k} (SW_i + O_i)
            acc = __dadd_ru(__dmul_ru(acc, __dadd_ru(sw, o)), __dmul_ru(pre, o));
            pre = __dmul_ru(pre, sw);
        }
        const double drop = E.f[(4 * nm) * kEpi + s];
        const double sup = E.f[(4 * nm + 1) * kEpi + s];
        double slo = E.f[(4 * nm + 2) * kEpi + s];
        const double slo_v = n > 0 ? fmax(__dsub_rd(1.0, pin_up), 0.0) : 0.0;
        const double sup_v = n > 0 ? fmin(__dsub_ru(1.0, pin_dn), 1.0) : 0.0;
        const double tr = __dadd_ru(acc, drop);
        sink_lo[row] = slo_v;
        sink_up[row] = sup_v;
        trunc[row] = tr;
        if (flags) {
            if (row == fault_row) slo = 2.0;   // fault injection: a row that claims too much
            uint32_t f = 0;
            if (n > 0) {
                if (__dadd_rd(slo, slo_v) > 1.0) f |= 0x1u;
                if (__dadd_ru(__dadd_ru(sup, sup_v), tr) < 1.0) f |= 0x2u;
            }
            flags[row] = f;
            if (f) atomicOr(status, IMPACT_STATUS_UNSOUND);
        }
    }
    __syncwarp();
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
// the kernel
// ---------------------------------------------------------------------------

enum { MODE_COUNT = 0, MODE_EMIT = 1, MODE_FUSED = 2 };

struct WalkArgs {
    const BatchIndex *B;
    int warp_smem;           // shared-memory bytes of one warp
    int nm;                  // largest n of the batch
    int64_t *row_ptr;        // COUNT / FUSED: written; EMIT: read
    int32_t *col;
    float *lo, *up;
    double *sink_lo, *sink_up, *trunc;
    uint32_t *flags;
    uint32_t *status;        // [0] status bits, [1] look-back abort flag
    unsigned long long *lb;  // COUNT / FUSED: look-back words, zeroed, one per row
    int64_t capacity;        // pairs the output arrays hold (< 0: unchecked)
    int64_t total_at;        // EMIT: index of the total in row_ptr
    int spin_limit;          // look-back sleeps before giving up
    int64_t row_begin;       // the launch covers global rows [row_begin, row_end)
    int64_t row_end;
    int64_t stall_row;       // fault injection: this row never publishes (-1: none)
    int64_t fault_row;       // fault injection: this row's checks see a bad sum (-1: none)
};

__host__ __device__ constexpr int epi_bytes(int nm)
{
    return kEpi * (8 + 4 + 4 * (4 * nm + 3));
}

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
    EpiBuf E;
    {
        unsigned char *eb = wbase + A.warp_smem - epi_bytes(A.nm);
        E.row = reinterpret_cast<int64_t *>(eb);
        E.nd = reinterpret_cast<int *>(eb + 8 * kEpi);
        E.f = reinterpret_cast<float *>(eb + 12 * kEpi);
        E.nm = A.nm;
    }
    int used = 0;
    bool lb_ok = true;

    // persistent: each warp takes the next row of the batch until none is left
    while (true) {
        unsigned long long taken = 0;
        if (lane == 0) taken = atomicAdd(next_row, 1ull);
        taken = __shfl_sync(0xffffffffu, taken, 0);
        if (taken >= (unsigned long long)(A.row_end - A.row_begin)) break;
        const int64_t row = A.row_begin + (int64_t)taken;   // global row of the batch
        const int q = find_problem(B->row_begin, B->count, row);
        const ImpactDesc &D = *B->desc[q];
        const int n = D.n;
        const WarpMem S = carve(wbase, D);
        const RowTerms rt = row_setup(D, S, row - B->row_begin[q], lane);
        bool ok = rt.ok, walked = true;
        int64_t base = 0, len = 0;
        if (kCount) {
            CountAcc acc;
            const EmitOut none{nullptr, nullptr, nullptr, 0, 0};
            int64_t w0 = 0;
            if (ok && !rt.empty) walked = walk_row<false>(S, n, lane, acc, none, w0);
            const bool good = ok && walked;
            int c = good ? acc.cnt : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            const float drop = warp_sum_ru(good ? acc.drop : 0.0f);
            const float sup = warp_sum_ru(good ? acc.sup : 0.0f);
            const float slo = warp_sum_rd(good ? acc.slo : 0.0f);
            int64_t prefix = 0;
            lb_ok = lookback(A.lb, row, c, lane, A.status + 1, A.status, A.spin_limit,
                             row == A.stall_row, prefix);
            if (lane == 0 && lb_ok) {
                A.row_ptr[row] = prefix;
                if (row == B->rows - 1) A.row_ptr[B->rows] = prefix + c;
            }
            base = prefix;
            len = c;
            // the row's FP64 terms wait in the epilogue buffer
            if (lane < n) {
                const DimHdr &h = S.h[lane];
                E.f[lane * kEpi + used] = good ? h.qlo : 0.0f;
                E.f[(E.nm + lane) * kEpi + used] = good ? h.qhi : 0.0f;
                E.f[(2 * E.nm + lane) * kEpi + used] = good ? h.SW : 0.0f;
                E.f[(3 * E.nm + lane) * kEpi + used] = good ? h.O : 0.0f;
            }
            if (lane == 0) {
                E.row[used] = row;
                E.nd[used] = good ? n : 0;
                E.f[(4 * E.nm) * kEpi + used] = drop;
                E.f[(4 * E.nm + 1) * kEpi + used] = sup;
                E.f[(4 * E.nm + 2) * kEpi + used] = slo;
            }
            if (++used == kEpi) {
                epi_flush(E, used, lane, A.sink_lo, A.sink_up, A.trunc, A.flags, A.status,
                          A.fault_row);
                used = 0;
            }
        } else {
            base = A.row_ptr[row];
            len = A.row_ptr[row + 1] - base;
        }
        if (kEmit && ok && walked && lb_ok) {
            if (base < 0 || len < 0 || (A.capacity >= 0 && base + len > A.capacity)) {
                if (lane == 0)
                    atomicOr(A.status, MODE == MODE_FUSED ? IMPACT_STATUS_CAPACITY
                                                          : IMPACT_STATUS_EMIT_MISMATCH);
            } else {
                const EmitOut out{A.col, A.lo, A.up, base, len};
                CountAcc none;
                int64_t written = 0;
                bool wok = true;
                if (!rt.empty) wok = walk_row<true>(S, n, lane, none, out, written);
                if (lane == 0 && (!wok || written != len))
                    atomicOr(A.status, wok ? IMPACT_STATUS_EMIT_MISMATCH : IMPACT_STATUS_INTERNAL);
            }
        }
        if (lane == 0) {
            if (!ok) atomicOr(A.status, IMPACT_STATUS_TABLE_OVERFLOW);
            if (!walked) atomicOr(A.status, IMPACT_STATUS_INTERNAL);
            if (MODE == MODE_EMIT && !ok) atomicOr(A.status, IMPACT_STATUS_EMIT_MISMATCH);
        }
        if (!lb_ok) break;   // the rows after this one cannot find their offsets
    }
    if (kCount && used > 0)
        epi_flush(E, used, lane, A.sink_lo, A.sink_up, A.trunc, A.flags, A.status, A.fault_row);
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

int walk_core_bytes(int n, int tsum_cap, int edge_cap)
{
    const int64_t lists = (int64_t)std::max(n - 1, 1) * kCap * 12;
    const int64_t edges = (int64_t)48 * edge_cap;
    int64_t b = kHdrBytes + (((int64_t)8 * tsum_cap + 15) & ~(int64_t)15) +
                ((std::max(lists, edges) + 15) & ~(int64_t)15);
    return (int)std::min<int64_t>(b, INT32_MAX / 2);
}

int walk_smem_bytes(int core_max, int nm, bool count)
{
    return core_max + (count ? epi_bytes(nm) : 0);
}

cudaError_t launch_walk_fp32(const BatchIndex *d_index, int64_t row_begin, int64_t row_end,
                             int nm, int core_max, int warps, int mode, const RowOutputs &o,
                             unsigned long long *lb, const WalkFaults &f, cudaStream_t stream)
{
    const int64_t rows = row_end - row_begin;
    if (rows <= 0) return cudaSuccess;
    const int warp_smem = walk_smem_bytes(core_max, nm, mode != MODE_EMIT);
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
    A.nm = nm;
    A.row_ptr = o.row_ptr;
    A.col = o.col;
    A.lo = (float *)o.lo;
    A.up = (float *)o.up;
    A.sink_lo = o.sink_lo;
    A.sink_up = o.sink_up;
    A.trunc = o.trunc;
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
    // persistent grid: as many blocks as fit at once (rows are taken dynamically)
    const int g = occupancy_grid(k, threads, smem, rows, warps);
    if (mode == MODE_COUNT)
        walk_fp32<MODE_COUNT><<<g, threads, smem, stream>>>(A);
    else if (mode == MODE_EMIT)
        walk_fp32<MODE_EMIT><<<g, threads, smem, stream>>>(A);
    else
        walk_fp32<MODE_FUSED><<<g, threads, smem, stream>>>(A);
    return cudaGetLastError();
}

}  // namespace impact
