// synth.cu -- interval-iteration controller synthesis on a device-resident
// IMDP (impact_synthesize, include/impact.h): the paper's Alg. 3 (safety) and
// Alg. 4 (reach-avoid), pessimistic policy, with the linear program of Sec. 5
// solved per row by the sorting method of Sec. 6.2.
//
// Per row the successors are the kept target cells t with [lo_t, up_t], the
// out-of-domain sink with [sink_lo, sink_up] and the truncated mass as one
// more successor with [0, trunc]. The sorting method starts every successor
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
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/impact.h"
#include "plan.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBisect = 52;   // bracket width 2^-52 of [0, 1]
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

struct RowRef {
    int64_t a, b;           // successor range in col/lo/up
    double sink_lo, sink_up, trunc;
};

// Greedy (sorting-method) optimum of one row for the value vector V.
// `maximize`: the max LP; `sink_v`: value of the sink; `high`: value the
// remaining mass of the bracket at its upper end (else its lower end).
template <typename VT>
__device__ double row_lp(const RowRef &R, const int32_t *__restrict__ col,
                         const VT *__restrict__ lo, const VT *__restrict__ up,
                         const double *__restrict__ V, bool maximize, double sink_v, bool high)
{
    const int lane = threadIdx.x & 31;
    // the value as seen by the min LP (max LP: 1 - v)
    auto val = [&](double v) { return maximize ? 1.0 - v : v; };
    const double tv = val(maximize ? 1.0 : 0.0);   // the truncated mass: the worst end
    const double sv = val(sink_v);
    // sums over the successors: lo, lo * v
    double slo = 0.0, slov = 0.0;
    for (int64_t i = R.a + lane; i < R.b; i += 32) {
        const double l = (double)lo[i];
        slo += l;
        slov += l * val(V[col[i]]);
    }
    slo = warp_sum(slo);
    slov = warp_sum(slov);
    slo += R.sink_lo;
    slov += R.sink_lo * sv;
    const double rest = 1.0 - slo;
    // mass of the successors with value <= x, and their weighted value
    auto G = [&](double x, double &gv) {
        double g = 0.0, v2 = 0.0;
        for (int64_t i = R.a + lane; i < R.b; i += 32) {
            const double v = val(V[col[i]]);
            if (v <= x) {
                const double w = (double)up[i] - (double)lo[i];
                g += w;
                v2 += w * v;
            }
        }
        g = warp_sum(g);
        v2 = warp_sum(v2);
        if (sv <= x) {
            g += R.sink_up - R.sink_lo;
            v2 += (R.sink_up - R.sink_lo) * sv;
        }
        if (tv <= x) {
            g += R.trunc;
            v2 += R.trunc * tv;
        }
        gv = v2;
        return g;
    };
    double res;
    if (rest <= 0.0) {
        res = slov;
    } else if (R.b - R.a <= 32 * kCache) {
        // short rows: each lane keeps its successors' values and widths in
        // registers for the whole bisection
        double cv[kCache], cw[kCache];
#pragma unroll
        for (int k = 0; k < kCache; ++k) {
            const int64_t i = R.a + lane + 32 * k;
            const bool in = i < R.b;
            cv[k] = in ? val(V[col[i]]) : 2.0;   // 2: never <= x
            cw[k] = in ? (double)up[i] - (double)lo[i] : 0.0;
        }
        auto Gc = [&](double x, double &gv) {
            double g = 0.0, v2 = 0.0;
#pragma unroll
            for (int k = 0; k < kCache; ++k)
                if (cv[k] <= x) {
                    g += cw[k];
                    v2 += cw[k] * cv[k];
                }
            g = warp_sum(g);
            v2 = warp_sum(v2);
            if (sv <= x) {
                g += R.sink_up - R.sink_lo;
                v2 += (R.sink_up - R.sink_lo) * sv;
            }
            if (tv <= x) {
                g += R.trunc;
                v2 += R.trunc * tv;
            }
            gv = v2;
            return g;
        };
        double xl = -1.0, xh = 1.0;
        for (int it = 0; it < kBisect; ++it) {
            const double xm = 0.5 * (xl + xh);
            double gv;
            if (Gc(xm, gv) >= rest) xh = xm; else xl = xm;
        }
        double gv;
        const double g = Gc(xl, gv);
        const double x = maximize ? (high ? xl : xh) : (high ? xh : xl);
        res = slov + gv + (rest - g) * fmax(x, 0.0);
    } else {
        double xl = -1.0, xh = 1.0;   // G(xl) = 0 < rest; G(1) >= rest by the row invariants
        for (int it = 0; it < kBisect; ++it) {
            const double xm = 0.5 * (xl + xh);
            double gv;
            if (G(xm, gv) >= rest) xh = xm; else xl = xm;
        }
        double gv;
        const double g = G(xl, gv);
        const double x = maximize ? (high ? xl : xh) : (high ? xh : xl);
        res = slov + gv + (rest - g) * fmax(x, 0.0);
    }
    return maximize ? 1.0 - res : res;
}

struct Phase {
    int spec;         // IMPACT_REACH_AVOID or IMPACT_SAFETY
    bool choose;      // optimise over the inputs (phase 1) or follow the policy
    bool maximize;    // the LP direction
};

// The LP of every row the phase needs (all inputs in phase 1, the policy's in
// phase 2), one warp per row, for both vectors.
template <typename VT>
__global__ void __launch_bounds__(kThreads)
row_values(Phase ph, int64_t rows, int n_inputs, const uint8_t *__restrict__ labels,
           const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
           const VT *__restrict__ lo, const VT *__restrict__ up,
           const double *__restrict__ sink_lo, const double *__restrict__ sink_up,
           const double *__restrict__ trunc, const double *__restrict__ V0,
           const double *__restrict__ V1, const int32_t *__restrict__ policy,
           double *__restrict__ R0, double *__restrict__ R1)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double sink_v = ph.spec == IMPACT_REACH_AVOID ? 0.0 : 1.0;
    for (int64_t r = warp0; r < rows; r += nwarps) {
        const int64_t c = r / n_inputs;
        const int j = (int)(r - c * n_inputs);
        if (labels[c] != 0 || (!ph.choose && j != policy[c])) continue;
        RowRef R{row_ptr[r], row_ptr[r + 1], sink_lo[r], sink_up[r], trunc[r]};
        // V0 never rises above, V1 never falls below the exact update
        const double a = row_lp(R, col, lo, up, V0, ph.maximize, sink_v, false);
        const double b = row_lp(R, col, lo, up, V1, ph.maximize, sink_v, true);
        if (lane == 0) {
            R0[r] = a;
            R1[r] = b;
        }
    }
}

// Per cell: the best input (phase 1) or the policy's row (phase 2), the next
// V0 and V1, and the largest |V1 - V0|.
__global__ void __launch_bounds__(kThreads)
cell_update(Phase ph, int64_t cells, int n_inputs, const uint8_t *__restrict__ labels,
            const double *__restrict__ R0, const double *__restrict__ R1,
            double *__restrict__ N0, double *__restrict__ N1, int32_t *__restrict__ policy,
            unsigned long long *__restrict__ diff)
{
    const bool reach = ph.spec == IMPACT_REACH_AVOID;
    // reach-avoid phase 1: max over inputs of the min LP; safety: min of max
    const bool pick_max = reach;
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
            int arg = 0;
            for (int j = 0; j < n_inputs; ++j) {
                const double a = R0[c * n_inputs + j], b = R1[c * n_inputs + j];
                if (j == 0 || (pick_max ? a > b0 : a < b0)) {
                    b0 = a;
                    arg = j;
                }
                if (j == 0 || (pick_max ? b > b1 : b < b1)) b1 = b;
            }
            policy[c] = arg;
            n0 = b0;
            n1 = b1;
        } else {
            const int64_t r = c * n_inputs + policy[c];
            n0 = R0[r];
            n1 = R1[r];
        }
        n0 = fmin(fmax(n0, 0.0), 1.0);
        n1 = fmin(fmax(n1, 0.0), 1.0);
        N0[c] = n0;
        N1[c] = n1;
        dmax = fmax(dmax, fabs(n1 - n0));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0 && dmax > 0.0)
        atomicMax(diff, (unsigned long long)__double_as_longlong(dmax));
}

__global__ void __launch_bounds__(kThreads)
init_values(int spec, int64_t cells, const uint8_t *__restrict__ labels, double *__restrict__ V0,
            double *__restrict__ V1)
{
    const bool reach = spec == IMPACT_REACH_AVOID;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t lab = labels[c];
        if (lab == 0) {
            V0[c] = 0.0;
            V1[c] = 1.0;
        } else {
            V0[c] = V1[c] = (reach ? lab == 1 : lab == 2) ? 1.0 : 0.0;
        }
    }
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

extern "C" impact_status impact_synthesize(const impact_csr *imdp, impact_precision precision,
                                           int64_t cells, int n_inputs, const uint8_t *labels,
                                           int spec, double eps, int max_iters, double *p_min,
                                           double *p_max, int32_t *policy, int *iterations,
                                           void *stream)
{
    using impact::fail;
    if (!imdp) return fail(IMPACT_ERR_ARG, "null IMDP");
    if (precision != IMPACT_FP32_SOUND && precision != IMPACT_FP64_PLAIN)
        return fail(IMPACT_ERR_ARG, "unknown precision");
    if (spec != IMPACT_REACH_AVOID && spec != IMPACT_SAFETY)
        return fail(IMPACT_ERR_ARG, "unknown specification");
    if (cells < 1 || n_inputs < 1 || imdp->rows != cells * n_inputs)
        return fail(IMPACT_ERR_ARG, "the IMDP must have cells * n_inputs rows");
    if (!(eps > 0.0) || max_iters < 1) return fail(IMPACT_ERR_ARG, "eps > 0 and max_iters >= 1");
    if (!device_array(imdp->row_ptr) || !device_array(imdp->sink_lo) ||
        !device_array(imdp->sink_up) || !device_array(imdp->trunc) || !device_array(labels) ||
        !device_array(p_min) || !device_array(p_max) || !device_array(policy) ||
        (imdp->nnz > 0 && (!device_array(imdp->col) || !device_array(imdp->lo) ||
                           !device_array(imdp->up))))
        return fail(IMPACT_ERR_ARG, "the IMDP, labels and outputs must be device arrays");
    cudaStream_t st = (cudaStream_t)stream;
    double *buf = nullptr, *rbuf = nullptr;
    unsigned long long *d_diff = nullptr, *h_diff = nullptr;
    const int64_t rows = cells * n_inputs;
    CK(cudaMallocAsync((void **)&buf, (size_t)cells * 4 * sizeof(double), st));
    CK(cudaMallocAsync((void **)&rbuf, (size_t)rows * 2 * sizeof(double), st));
    CK(cudaMallocAsync((void **)&d_diff, sizeof(unsigned long long), st));
    CK(cudaMallocHost((void **)&h_diff, sizeof(unsigned long long)));
    const bool reach = spec == IMPACT_REACH_AVOID;
    const int g_cells = grid_of(cells, kThreads);
    const int g_rows = grid_of(rows, kThreads / 32);
    impact_status status = IMPACT_OK;
    int its[2] = {0, 0};
    for (int phase = 0; phase < 2 && status == IMPACT_OK; ++phase) {
        double *V0 = buf, *V1 = buf + cells, *N0 = buf + 2 * cells, *N1 = buf + 3 * cells;
        Phase ph;
        ph.spec = spec;
        ph.choose = phase == 0;
        // reach-avoid: phase 1 min LP, phase 2 max LP; safety the other way
        ph.maximize = reach ? phase == 1 : phase == 0;
        init_values<<<g_cells, kThreads, 0, st>>>(spec, cells, labels, V0, V1);
        int it = 0;
        while (it < max_iters) {
            cudaMemsetAsync(d_diff, 0, sizeof(unsigned long long), st);
            double *R0 = rbuf, *R1 = rbuf + rows;
            if (precision == IMPACT_FP32_SOUND)
                row_values<float><<<g_rows, kThreads, 0, st>>>(
                    ph, rows, n_inputs, labels, imdp->row_ptr, imdp->col,
                    (const float *)imdp->lo, (const float *)imdp->up, imdp->sink_lo,
                    imdp->sink_up, imdp->trunc, V0, V1, policy, R0, R1);
            else
                row_values<double><<<g_rows, kThreads, 0, st>>>(
                    ph, rows, n_inputs, labels, imdp->row_ptr, imdp->col,
                    (const double *)imdp->lo, (const double *)imdp->up, imdp->sink_lo,
                    imdp->sink_up, imdp->trunc, V0, V1, policy, R0, R1);
            cell_update<<<g_cells, kThreads, 0, st>>>(ph, cells, n_inputs, labels, R0, R1, N0, N1,
                                                      policy, d_diff);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) {
                status = fail(IMPACT_ERR_CUDA, cudaGetErrorString(e));
                break;
            }
            std::swap(V0, N0);
            std::swap(V1, N1);
            ++it;
            // the stopping test of Alg. 3/4 on the vectors just computed
            cudaMemcpyAsync(h_diff, d_diff, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                status = fail(IMPACT_ERR_CUDA, "synthesis iteration failed");
                break;
            }
            double dmax;
            memcpy(&dmax, h_diff, sizeof(dmax));
            if (dmax <= eps) break;
        }
        its[phase] = it;
        if (status != IMPACT_OK) break;
        // reach-avoid: P_min = V0 of phase 1, P_max = V1 of phase 2;
        // safety: P_min = 1 - V1 of phase 1, P_max = 1 - V0 of phase 2
        double *dst = phase == 0 ? p_min : p_max;
        const double *src = reach ? (phase == 0 ? V0 : V1) : (phase == 0 ? V1 : V0);
        finish<<<g_cells, kThreads, 0, st>>>(spec, cells, src, !reach, dst);
    }
    cudaFreeAsync(buf, st);
    cudaFreeAsync(rbuf, st);
    cudaFreeAsync(d_diff, st);
    cudaStreamSynchronize(st);
    cudaFreeHost(h_diff);
    if (iterations) {
        iterations[0] = its[0];
        iterations[1] = its[1];
    }
    return status;
}
