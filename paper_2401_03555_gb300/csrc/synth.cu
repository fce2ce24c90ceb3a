// synth.cu -- interval-iteration controller synthesis on a device-resident
// IMDP (impact_synthesize / impact_synthesize_ex, include/impact.h): the
// paper's Alg. 3 (safety) and Alg. 4 (reach-avoid), pessimistic or optimistic
// policy (Sec. 5), infinite or finite horizon (Remark 5.1), the disturbance
// points as an adversary, with the linear program of Sec. 5 solved per row by
// the sorting method of Sec. 6.2.
//
// Per row the successors are the kept target cells t with [lo_t, up_t], the
// out-of-domain sink with [sink_lo, sink_up] and the truncated mass as one
// more successor with [0, trunc]; with region vectors (Sec. 3.1) the
// labelled cells and the sink give way to the target region [R_min, R_max]
// and the avoid region [A_min, A_max]. The sorting method starts every successor
// at its lower bound and raises them in ascending (min LP) or descending (max
// LP) order of their value until the total is 1. Instead of sorting, one warp
// finds the value threshold tau of that greedy fill by bisection: with
// w = up - lo and G(x) = sum of w over the successors whose value is <= x,
// tau is the least x with G(x) >= 1 - sum lo. After the bisection the
// remaining mass sits between the bracket's ends; it is valued at the lower
// end when the result must not be too high (the V0 update of a min LP) and at
// the upper end otherwise, so V0 stays below and V1 above their exact values.
// The max LP is the min LP of the values 1 - v.
//
// One warp per row computes the row's LP for both vectors; one thread per cell
// then keeps the best input (or the policy's) and writes the cell's next V0
// and V1; the largest |V1 - V0| is gathered with an atomic max on the bits of
// a non-negative double.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/impact.h"
#include "alloc.h"
#include "plan.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCache = 16;    // successors per lane kept in registers (rows <= 512)

#define CK(expr)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return impact::fail(e_ == cudaErrorMemoryAllocation ? IMPACT_ERR_OOM              \
                                                                : IMPACT_ERR_CUDA,            \
                                std::string(#expr) + ": " + cudaGetErrorString(e_));          \
    } while (0)

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Order-preserving integer key of a finite double (-0 and +0 share key 0):
// x <= y exactly when okey(x) <= okey(y).
__device__ __forceinline__ long long okey(double x)
{
    const long long b = __double_as_longlong(x);
    if ((b & 0x7fffffffffffffffll) == 0) return 0;   // +0 and -0, without an FP64 compare
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}

// The double whose key is k (the inverse of okey; key -1 gives -0).
__device__ __forceinline__ double from_okey(long long k)
{
    return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffll));
}

struct RowRef {
    int64_t a, b;           // successor range in col/lo/up
    // three further successors: the sink and an empty one, or the two
    // regions; then the truncated mass. Lower bounds, widths and values
    // (before the max LP's mapping v -> 1 - v)
    double xlo[3], xw[3], xv[3];
};

// Greedy (sorting-method) optimum of one row for the value vector V.
// `maximize`: the max LP; `high`: value the remaining mass of the bracket at
// its upper end (else its lower end); `excl`: when not null, successors t
// with excl[t] != 0 are left out (their mass is in the region successors).
template <typename VT>
__device__ double row_lp(const RowRef &R, const int32_t *__restrict__ col,
                         const VT *__restrict__ lo, const VT *__restrict__ up,
                         const long long *__restrict__ wfix, const uint8_t *__restrict__ excl,
                         const double *__restrict__ V, const long long *__restrict__ K,
                         bool maximize, bool high)
{
    const int lane = threadIdx.x & 31;
    // the value as seen by the min LP (max LP: 1 - v); K holds the keys of
    // these values per cell
    auto val = [&](double v) { return maximize ? 1.0 - v : v; };
    auto out = [&](int32_t t) { return excl != nullptr && excl[t] != 0; };
    // sums over the successors: lo, lo * v
    double slo = 0.0, slov = 0.0;
    for (int64_t i = R.a + lane; i < R.b; i += 32) {
        const int32_t t = col[i];
        if (out(t)) continue;
        const double l = (double)lo[i];
        slo += l;
        slov += l * val(V[t]);
    }
    slo = warp_sum(slo);
    slov = warp_sum(slov);
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        slo += R.xlo[x];
        slov += R.xlo[x] * val(R.xv[x]);
    }
    const double rest = 1.0 - slo;
    if (rest <= 0.0) return maximize ? 1.0 - slov : slov;
    // the further successors: keys and fixed-point widths
    long long xk[3], xwf[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        xk[k] = okey(val(R.xv[k]));
        xwf[k] = __double2ll_rn(R.xw[k] * 0x1p52);
    }
    const long long rest_f = __double2ll_rn(rest * 0x1p52);
    auto finish = [&](long long g, long long kx) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (xk[k] <= kx) g += xwf[k];
        return g;
    };
    // G(x): mass (2^-52 units) of the successors whose value is <= x, x given
    // by its key. The bisection below runs in key order down to adjacent
    // doubles: integer work only, the same trip count on every lane (FP64
    // issue is scarce on this part).
    long long kl = okey(-1.0), kh = okey(1.0);   // G(-1) = 0 < rest; G(1) >= rest
    if (R.b - R.a <= 32 * kCache) {
        // short rows: each lane keeps its successors' keys and widths in
        // registers for the whole bisection
        long long ck[kCache], cwf[kCache];
#pragma unroll
        for (int k = 0; k < kCache; ++k) {
            const int64_t i = R.a + lane + 32 * k;
            const bool in = i < R.b && !out(col[i]);
            ck[k] = in ? K[col[i]] : LLONG_MAX;
            cwf[k] = in ? wfix[i] : 0ll;
        }
        while (kh - kl > 1) {
            const long long km = kl + ((kh - kl) >> 1);
            long long g = 0;
#pragma unroll
            for (int k = 0; k < kCache; ++k)
                if (ck[k] <= km) g += cwf[k];
            if (finish(g, km) >= rest_f) kh = km; else kl = km;
        }
    } else {
        // long rows: every pass reads the keys and widths again (from L2)
        while (kh - kl > 1) {
            const long long km = kl + ((kh - kl) >> 1);
            long long g = 0;
            for (int64_t i = R.a + lane; i < R.b; i += 32) {
                const int32_t t = col[i];
                if (!out(t) && K[t] <= km) g += wfix[i];
            }
            if (finish(g, km) >= rest_f) kh = km; else kl = km;
        }
    }
    const double xl = from_okey(kl), xh = from_okey(kh);
    // the final value in FP64 at the bracket: the mass below it, its
    // weighted value, and the rest valued at the bracket's end that keeps
    // V0 below and V1 above the exact update
    double g = 0.0, gv = 0.0;
    for (int64_t i = R.a + lane; i < R.b; i += 32) {
        const int32_t t = col[i];
        if (out(t)) continue;
        const double v = val(V[t]);
        if (v <= xl) {
            const double w = (double)up[i] - (double)lo[i];
            g += w;
            gv += w * v;
        }
    }
    g = warp_sum(g);
    gv = warp_sum(gv);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double v = val(R.xv[k]);
        if (v <= xl) {
            g += R.xw[k];
            gv += R.xw[k] * v;
        }
    }
    const double x = maximize ? (high ? xl : xh) : (high ? xh : xl);
    const double res = slov + gv + (rest - g) * fmax(x, 0.0);
    return maximize ? 1.0 - res : res;
}

struct Phase {
    int spec;         // IMPACT_REACH_AVOID or IMPACT_SAFETY
    bool choose;      // optimise over the inputs (phase 1) or follow the policy
    bool maximize;    // the LP direction
    bool pol_v1;      // phase 1: the policy follows the V1 choice (else V0)
    int n_disturb;    // disturbance points per input
};

// Region vectors of the rows (all four, or all null).
struct Regions {
    const double *r_lo, *r_up, *a_lo, *a_up;
};

// The LP of every row the phase needs (all inputs in phase 1, the policy's in
// phase 2), one warp per row, for both vectors.
template <typename VT>
__global__ void __launch_bounds__(kThreads)
row_values(Phase ph, int64_t rows, int n_inputs, const uint8_t *__restrict__ labels,
           const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
           const VT *__restrict__ lo, const VT *__restrict__ up,
           const double *__restrict__ sink_lo, const double *__restrict__ sink_up,
           const double *__restrict__ trunc, const long long *__restrict__ wfix, Regions rg,
           const double *__restrict__ V0, const double *__restrict__ V1,
           const long long *__restrict__ K0, const long long *__restrict__ K1,
           const int32_t *__restrict__ policy, double *__restrict__ R0, double *__restrict__ R1)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool reach = ph.spec == IMPACT_REACH_AVOID;
    const int64_t per_cell = (int64_t)n_inputs * ph.n_disturb;
    const uint8_t *excl = rg.r_lo ? labels : nullptr;
    for (int64_t r = warp0; r < rows; r += nwarps) {
        const int64_t c = r / per_cell;
        const int j = (int)((r - c * per_cell) / ph.n_disturb);
        if (labels[c] != 0 || (!ph.choose && j != policy[c])) continue;
        RowRef R;
        R.a = row_ptr[r];
        R.b = row_ptr[r + 1];
        if (rg.r_lo) {
            // the target region (reach: value 1) and the avoid region with
            // the sink (safety: value 1)
            R.xlo[0] = rg.r_lo[r];
            R.xw[0] = rg.r_up[r] - rg.r_lo[r];
            R.xv[0] = reach ? 1.0 : 0.0;
            R.xlo[1] = rg.a_lo[r];
            R.xw[1] = rg.a_up[r] - rg.a_lo[r];
            R.xv[1] = reach ? 0.0 : 1.0;
        } else {
            R.xlo[0] = sink_lo[r];
            R.xw[0] = sink_up[r] - sink_lo[r];
            R.xv[0] = reach ? 0.0 : 1.0;
            R.xlo[1] = 0.0;
            R.xw[1] = 0.0;
            R.xv[1] = 0.0;
        }
        // the truncated mass, at its worst end: 0 in a min LP, 1 in a max LP
        R.xlo[2] = 0.0;
        R.xw[2] = trunc[r];
        R.xv[2] = ph.maximize ? 1.0 : 0.0;
        // V0 never rises above, V1 never falls below the exact update
        const double a = row_lp(R, col, lo, up, wfix, excl, V0, K0, ph.maximize, false);
        const double b = row_lp(R, col, lo, up, wfix, excl, V1, K1, ph.maximize, true);
        if (lane == 0) {
            R0[r] = a;
            R1[r] = b;
        }
    }
}

// The disturbance's choice among the W rows of one input: the least
// satisfaction (reach-avoid) or the most unsafe value (safety).
__device__ __forceinline__ double worst(const double *__restrict__ p, int W, bool reach)
{
    double w = p[0];
    for (int k = 1; k < W; ++k) w = reach ? fmin(w, p[k]) : fmax(w, p[k]);
    return w;
}

// Per cell: for each input the disturbance's worst row, then the best input
// (phase 1) or the policy's input (phase 2), the next V0 and V1, and the
// largest |V1 - V0|. The values are satisfaction probabilities (reach-avoid:
// inputs maximise, disturbances minimise) or unsafe ones (safety: inputs
// minimise, disturbances maximise).
__global__ void __launch_bounds__(kThreads)
cell_update(Phase ph, int64_t cells, int n_inputs, const uint8_t *__restrict__ labels,
            const double *__restrict__ R0, const double *__restrict__ R1,
            double *__restrict__ N0, double *__restrict__ N1, long long *__restrict__ KN0,
            long long *__restrict__ KN1, int32_t *__restrict__ policy,
            unsigned long long *__restrict__ diff)
{
    const bool reach = ph.spec == IMPACT_REACH_AVOID;
    const int W = ph.n_disturb;
    double dmax = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t lab = labels[c];
        double n0, n1;
        if (lab != 0) {   // absorbing: target (reach) or avoid (safety) has value 1
            n0 = n1 = (reach ? lab == 1 : lab == 2) ? 1.0 : 0.0;
            if (ph.choose) policy[c] = 0;
        } else if (ph.choose) {
            double b0 = 0.0, b1 = 0.0;
            int arg0 = 0, arg1 = 0;
            for (int j = 0; j < n_inputs; ++j) {
                const double a = worst(R0 + (c * n_inputs + j) * W, W, reach);
                const double b = worst(R1 + (c * n_inputs + j) * W, W, reach);
                if (j == 0 || (reach ? a > b0 : a < b0)) {
                    b0 = a;
                    arg0 = j;
                }
                if (j == 0 || (reach ? b > b1 : b < b1)) {
                    b1 = b;
                    arg1 = j;
                }
            }
            policy[c] = ph.pol_v1 ? arg1 : arg0;
            n0 = b0;
            n1 = b1;
        } else {
            n0 = worst(R0 + (c * n_inputs + policy[c]) * W, W, reach);
            n1 = worst(R1 + (c * n_inputs + policy[c]) * W, W, reach);
        }
        n0 = fmin(fmax(n0, 0.0), 1.0);
        n1 = fmin(fmax(n1, 0.0), 1.0);
        N0[c] = n0;
        N1[c] = n1;
        // the keys of the values the next iteration's LPs compare
        KN0[c] = okey(ph.maximize ? 1.0 - n0 : n0);
        KN1[c] = okey(ph.maximize ? 1.0 - n1 : n1);
        dmax = fmax(dmax, fabs(n1 - n0));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0 && dmax > 0.0)
        atomicMax(diff, (unsigned long long)__double_as_longlong(dmax));
}

// V0 from 0 and V1 from 1 on the free cells (from 0 both, for a finite
// horizon); the labelled cells hold their absorbing value.
__global__ void __launch_bounds__(kThreads)
init_values(int spec, bool horizon, bool maximize, int64_t cells,
            const uint8_t *__restrict__ labels, double *__restrict__ V0, double *__restrict__ V1,
            long long *__restrict__ K0, long long *__restrict__ K1)
{
    const bool reach = spec == IMPACT_REACH_AVOID;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t lab = labels[c];
        double a, b;
        if (lab == 0) {
            a = 0.0;
            b = horizon ? 0.0 : 1.0;
        } else {
            a = b = (reach ? lab == 1 : lab == 2) ? 1.0 : 0.0;
        }
        V0[c] = a;
        V1[c] = b;
        K0[c] = okey(maximize ? 1.0 - a : a);
        K1[c] = okey(maximize ? 1.0 - b : b);
    }
}

// Widths up - lo of every pair in 2^-52 units (the LP passes sum integers).
template <typename VT>
__global__ void __launch_bounds__(kThreads)
pair_widths(int64_t nnz, const VT *__restrict__ lo, const VT *__restrict__ up,
            long long *__restrict__ wfix)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz;
         i += (int64_t)gridDim.x * blockDim.x)
        wfix[i] = __double2ll_rn(((double)up[i] - (double)lo[i]) * 0x1p52);
}

__global__ void __launch_bounds__(kThreads)
finish(int spec, int64_t cells, const double *__restrict__ V, bool complement,
       double *__restrict__ out)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
         c += (int64_t)gridDim.x * blockDim.x)
        out[c] = complement ? 1.0 - V[c] : V[c];
}

int grid_of(int64_t items, int per_block)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (items + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
}

bool device_array(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" impact_status impact_synthesize_ex(const impact_csr *imdp, impact_precision precision,
                                              int64_t cells, int n_inputs, const uint8_t *labels,
                                              const impact_synth_options *opt, double *p_min,
                                              double *p_max, int32_t *policy, int *iterations,
                                              void *stream)
{
    using impact::fail;
    if (!imdp || !opt) return fail(IMPACT_ERR_ARG, "null IMDP or options");
    if (precision != IMPACT_FP32_SOUND && precision != IMPACT_FP64_PLAIN)
        return fail(IMPACT_ERR_ARG, "unknown precision");
    const int spec = opt->spec;
    if (spec != IMPACT_REACH_AVOID && spec != IMPACT_SAFETY)
        return fail(IMPACT_ERR_ARG, "unknown specification");
    if (opt->optimistic != 0 && opt->optimistic != 1)
        return fail(IMPACT_ERR_ARG, "optimistic must be 0 or 1");
    if (opt->horizon < 0) return fail(IMPACT_ERR_ARG, "horizon must be >= 0");
    const int W = opt->n_disturb;
    if (W < 1) return fail(IMPACT_ERR_ARG, "n_disturb must be >= 1");
    if (cells < 1 || n_inputs < 1 || imdp->rows != cells * n_inputs * W)
        return fail(IMPACT_ERR_ARG, "the IMDP must have cells * n_inputs * n_disturb rows");
    const bool horizon = opt->horizon > 0;
    if (!horizon && (!(opt->eps > 0.0) || opt->max_iters < 1))
        return fail(IMPACT_ERR_ARG, "eps > 0 and max_iters >= 1");
    if (!device_array(imdp->row_ptr) || !device_array(imdp->sink_lo) ||
        !device_array(imdp->sink_up) || !device_array(imdp->trunc) || !device_array(labels) ||
        !device_array(p_min) || !device_array(p_max) || !device_array(policy) ||
        (imdp->nnz > 0 && (!device_array(imdp->col) || !device_array(imdp->lo) ||
                           !device_array(imdp->up))))
        return fail(IMPACT_ERR_ARG, "the IMDP, labels and outputs must be device arrays");
    Regions rg{opt->r_lo, opt->r_up, opt->a_lo, opt->a_up};
    const int given = !!rg.r_lo + !!rg.r_up + !!rg.a_lo + !!rg.a_up;
    if (given != 0 && given != 4) return fail(IMPACT_ERR_ARG, "give all four region vectors or none");
    if (given == 4 && (!device_array(rg.r_lo) || !device_array(rg.r_up) ||
                       !device_array(rg.a_lo) || !device_array(rg.a_up)))
        return fail(IMPACT_ERR_ARG, "the region vectors must be device arrays");
    cudaStream_t st = (cudaStream_t)stream;
    double *buf = nullptr, *rbuf = nullptr;
    long long *kbuf = nullptr, *wfix = nullptr;
    unsigned long long *d_diff = nullptr, *h_diff = nullptr;
    const int64_t rows = imdp->rows;
    const int64_t nnz = imdp->nnz;
    auto free_all = [&]() {
        impact::dev_free_async(buf, st);
        impact::dev_free_async(kbuf, st);
        impact::dev_free_async(wfix, st);
        impact::dev_free_async(rbuf, st);
        impact::dev_free_async(d_diff, st);
        cudaStreamSynchronize(st);
        impact::host_free(h_diff);
    };
    {
        cudaError_t e = impact::dev_malloc_async(&buf, (size_t)cells * 4 * sizeof(double), st);
        if (e == cudaSuccess)
            e = impact::dev_malloc_async(&kbuf, (size_t)cells * 4 * sizeof(long long), st);
        if (e == cudaSuccess)
            e = impact::dev_malloc_async(
                &wfix, (size_t)std::max<int64_t>(nnz, 1) * sizeof(long long), st);
        if (e == cudaSuccess)
            e = impact::dev_malloc_async(&rbuf, (size_t)rows * 2 * sizeof(double), st);
        if (e == cudaSuccess) e = impact::dev_malloc_async(&d_diff, sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = impact::host_malloc(&h_diff, sizeof(unsigned long long));
        if (e != cudaSuccess) {
            free_all();
            return fail(e == cudaErrorMemoryAllocation ? IMPACT_ERR_OOM : IMPACT_ERR_CUDA,
                        std::string("synthesis scratch: ") + cudaGetErrorString(e));
        }
    }
    const bool reach = spec == IMPACT_REACH_AVOID;
    // the LP that bounds satisfaction from below: reach-avoid the min LP,
    // safety the max LP of the unsafe value; phase 1 optimises the inputs on
    // it (pessimistic) or on the other one (optimistic)
    const bool lower_max = !reach;
    const bool lp1_max = opt->optimistic ? !lower_max : lower_max;
    const int limit = horizon ? opt->horizon : opt->max_iters;
    const int g_cells = grid_of(cells, kThreads);
    const int g_rows = grid_of(rows, kThreads / 32);
    impact_status status = IMPACT_OK;
    int its[2] = {0, 0};
    if (nnz > 0) {
        const int g_nnz = grid_of(nnz, kThreads);
        if (precision == IMPACT_FP32_SOUND)
            pair_widths<float><<<g_nnz, kThreads, 0, st>>>(nnz, (const float *)imdp->lo,
                                                           (const float *)imdp->up, wfix);
        else
            pair_widths<double><<<g_nnz, kThreads, 0, st>>>(nnz, (const double *)imdp->lo,
                                                            (const double *)imdp->up, wfix);
    }
    for (int phase = 0; phase < 2 && status == IMPACT_OK; ++phase) {
        double *V0 = buf, *V1 = buf + cells, *N0 = buf + 2 * cells, *N1 = buf + 3 * cells;
        long long *K0 = kbuf, *K1 = kbuf + cells, *KN0 = kbuf + 2 * cells, *KN1 = kbuf + 3 * cells;
        Phase ph;
        ph.spec = spec;
        ph.choose = phase == 0;
        ph.maximize = phase == 0 ? lp1_max : !lp1_max;
        // the vector whose end phase 1 reports: reach min LP -> V0, reach max
        // LP -> V1, safety max LP -> V1 (P_min = 1 - V1), min LP -> V0
        ph.pol_v1 = lp1_max;
        ph.n_disturb = W;
        init_values<<<g_cells, kThreads, 0, st>>>(spec, horizon, ph.maximize, cells, labels, V0,
                                                  V1, K0, K1);
        int it = 0;
        while (it < limit) {
            cudaMemsetAsync(d_diff, 0, sizeof(unsigned long long), st);
            double *R0 = rbuf, *R1 = rbuf + rows;
            if (precision == IMPACT_FP32_SOUND)
                row_values<float><<<g_rows, kThreads, 0, st>>>(
                    ph, rows, n_inputs, labels, imdp->row_ptr, imdp->col,
                    (const float *)imdp->lo, (const float *)imdp->up, imdp->sink_lo,
                    imdp->sink_up, imdp->trunc, wfix, rg, V0, V1, K0, K1, policy, R0, R1);
            else
                row_values<double><<<g_rows, kThreads, 0, st>>>(
                    ph, rows, n_inputs, labels, imdp->row_ptr, imdp->col,
                    (const double *)imdp->lo, (const double *)imdp->up, imdp->sink_lo,
                    imdp->sink_up, imdp->trunc, wfix, rg, V0, V1, K0, K1, policy, R0, R1);
            cell_update<<<g_cells, kThreads, 0, st>>>(ph, cells, n_inputs, labels, R0, R1, N0, N1,
                                                      KN0, KN1, policy, d_diff);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) {
                status = fail(IMPACT_ERR_CUDA, cudaGetErrorString(e));
                break;
            }
            std::swap(V0, N0);
            std::swap(V1, N1);
            std::swap(K0, KN0);
            std::swap(K1, KN1);
            ++it;
            if (horizon) continue;   // a fixed number of steps: no stopping test
            // the stopping test of Alg. 3/4 on the vectors just computed
            cudaMemcpyAsync(h_diff, d_diff, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                status = fail(IMPACT_ERR_CUDA, "synthesis iteration failed");
                break;
            }
            double dmax;
            memcpy(&dmax, h_diff, sizeof(dmax));
            if (dmax <= opt->eps) break;
        }
        its[phase] = it;
        if (status != IMPACT_OK) break;
        // reach-avoid: the min LP gives P_min = V0, the max LP P_max = V1;
        // safety: the max LP gives P_min = 1 - V1, the min LP P_max = 1 - V0
        double *dst;
        const double *src;
        if (reach) {
            dst = ph.maximize ? p_max : p_min;
            src = ph.maximize ? V1 : V0;
        } else {
            dst = ph.maximize ? p_min : p_max;
            src = ph.maximize ? V1 : V0;
        }
        finish<<<g_cells, kThreads, 0, st>>>(spec, cells, src, !reach, dst);
        if (horizon && cudaStreamSynchronize(st) != cudaSuccess)
            status = fail(IMPACT_ERR_CUDA, "synthesis phase failed");
    }
    free_all();
    if (iterations) {
        iterations[0] = its[0];
        iterations[1] = its[1];
    }
    return status;
}

extern "C" impact_status impact_synthesize(const impact_csr *imdp, impact_precision precision,
                                           int64_t cells, int n_inputs, const uint8_t *labels,
                                           int spec, double eps, int max_iters, double *p_min,
                                           double *p_max, int32_t *policy, int *iterations,
                                           void *stream)
{
    impact_synth_options o;
    memset(&o, 0, sizeof(o));
    o.spec = spec;
    o.n_disturb = 1;
    o.eps = eps;
    o.max_iters = max_iters;
    return impact_synthesize_ex(imdp, precision, cells, n_inputs, labels, &o, p_min, p_max,
                                policy, iterations, stream);
}
