// mc.cu -- impact_build_mc (include/impact.h): the IMDP of x+ = f(x,u) + w for
// a noise given by draws (Sec. 4.1: a full covariance Gaussian or a custom
// distribution, integrated by Monte-Carlo sampling instead of the closed-form
// Gaussian factors). Same image, grid, rows and output layout as impact_build;
// the per-row histogram kernels are in kernels.cu (mc_rows).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/impact.h"
#include "alloc.h"
#include "kernels.h"
#include "pipeline.h"
#include "plan.h"

namespace impact {
impact_status fail(impact_status s, const std::string &msg);
impact_request single(const impact_system *sys, const impact_grid *grid,
                      const impact_inputs *inputs, const double *sigma, double cutoff);
impact_status get_work(const Batch &B, const impact_csr *out, cudaStream_t st, Work &W);
impact_status release(Work &W, cudaStream_t st);
bool is_device_ptr(const void *p);
impact_status check_row_arrays(const impact_csr *out);
impact_status pair_view(const impact_csr *out, impact_csr &v);
void free_owned(impact_csr *out, cudaStream_t st);
}  // namespace impact

using namespace impact;

#define CK(expr)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? IMPACT_ERR_OOM : IMPACT_ERR_CUDA,   \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

extern "C" impact_status impact_build_mc(const impact_system *sys, const impact_grid *grid,
                                         const impact_inputs *inputs, const double *samples,
                                         int64_t n_samples, double cutoff,
                                         impact_precision precision, impact_csr *out,
                                         void *stream)
{
    if (!sys || !grid || !inputs || !out) return fail(IMPACT_ERR_ARG, "null argument");
    if (precision != IMPACT_FP32_SOUND && precision != IMPACT_FP64_PLAIN)
        return fail(IMPACT_ERR_ARG, "unknown precision");
    if (n_samples < 1 || n_samples > ((int64_t)1 << 24))
        return fail(IMPACT_ERR_ARG, "n_samples must be in [1, 2^24]");
    if (!(cutoff >= 0.0 && cutoff < 1.0)) return fail(IMPACT_ERR_ARG, "cutoff must be in [0, 1)");
    if (!is_device_ptr(samples)) return fail(IMPACT_ERR_ARG, "samples must be a device array");
    const int n = grid->n;
    if (n < 1 || n > IMPACT_MAX_DIM) return fail(IMPACT_ERR_ARG, "grid.n must be in [1, 8]");
    cudaStream_t st = (cudaStream_t)stream;
    // the FP64 tables of the build (edges and image terms). The planner's
    // Gaussian windows do not enter here: it is given a negligible noise
    // scale and a cutoff near 1 so that they stay small, and the descriptor
    // then carries the caller's cutoff and output precision.
    if (!grid->lo || !grid->hi || !grid->cells) return fail(IMPACT_ERR_ARG, "null grid");
    std::vector<double> tiny((size_t)n, 1.0);
    for (int d = 0; d < n; ++d)
        if (grid->cells[d] >= 1 && isfinite(grid->hi[d] - grid->lo[d]) && grid->hi[d] > grid->lo[d])
            tiny[d] = 1e-6 * (grid->hi[d] - grid->lo[d]) / grid->cells[d];
    impact_request req = single(sys, grid, inputs, tiny.data(), 0.999);
    Batch B;
    impact_status s = make_batch(&req, 1, IMPACT_FP64_PLAIN, nullptr, B);
    if (s != IMPACT_OK) return s;
    B.plans[0].desc.cutoff = cutoff;
    B.plans[0].desc.prec = precision;
    configure_pool_once();
    const bool lib_owned = (out->col == nullptr);
    const size_t vbytes = precision == IMPACT_FP32_SOUND ? 4 : 8;
    // a library-owned result that fails is released whole
    auto give_back = [&](impact_status r) {
        if (lib_owned && r != IMPACT_OK) {
            free_owned(out, st);
            cudaStreamSynchronize(st);
        }
        return r;
    };
    if (lib_owned) {
        memset(out, 0, sizeof(*out));
        out->owned = 1;
        cudaError_t e = dev_malloc_async(&out->row_ptr, (B.rows + 1) * 8, st);
        if (e == cudaSuccess) e = dev_malloc_async(&out->sink_lo, B.rows * 8, st);
        if (e == cudaSuccess) e = dev_malloc_async(&out->sink_up, B.rows * 8, st);
        if (e == cudaSuccess) e = dev_malloc_async(&out->trunc, B.rows * 8, st);
        if (e == cudaSuccess) e = dev_malloc_async(&out->row_flags, B.rows * 4, st);
        if (e != cudaSuccess) return give_back(fail(IMPACT_ERR_OOM, "row arrays"));
    } else if ((s = check_row_arrays(out)) != IMPACT_OK) {
        return s;
    }
    Work W;
    impact_csr no_ws = *out;
    no_ws.workspace = nullptr;
    if ((s = get_work(B, &no_ws, st, W)) != IMPACT_OK) return give_back(s);
    // per-call tables: draw keys [n][S], range [n][2], values u / S for
    // u = 0..S (FP64, FP32 down, FP32 up), the non-finite flag
    const int64_t S = n_samples;
    const size_t t_keys = (size_t)n * S * 8, t_range = (size_t)n * 16, t_val = (size_t)(S + 1) * 8;
    const size_t t_f = (size_t)(S + 1) * 4;
    const size_t total = t_keys + t_range + t_val + 2 * t_f + 16;
    unsigned char *tab = nullptr;
    s = upload(B, W, st);
    if (s == IMPACT_OK && dev_malloc_async(&tab, total, st) != cudaSuccess)
        s = fail(IMPACT_ERR_OOM, "sampled-noise tables");
    auto done = [&](impact_status r) {
        dev_free_async(tab, st);
        impact_status q = release(W, st);
        return give_back(r != IMPACT_OK ? r : q);
    };
    if (s != IMPACT_OK) return done(s);
    long long *keys = (long long *)tab;
    double *range = (double *)(tab + t_keys);
    double *val = (double *)(tab + t_keys + t_range);
    float *val_dn = (float *)(tab + t_keys + t_range + t_val);
    float *val_up = (float *)(tab + t_keys + t_range + t_val + t_f);
    unsigned *bad = (unsigned *)(tab + t_keys + t_range + t_val + 2 * t_f);
    // the least count u with u / S >= cutoff (the definition's FP64 test)
    const double dS = (double)S;
    int64_t kmin = cutoff > 0.0 ? (int64_t)ceil(cutoff * dS) : 0;
    while (kmin > 0 && (double)(kmin - 1) / dS >= cutoff) --kmin;
    while (cutoff > 0.0 && (double)kmin / dS < cutoff) ++kmin;
    RowOutputs o;
    memset(&o, 0, sizeof(o));
    o.row_ptr = out->row_ptr;
    o.sink_lo = out->sink_lo;
    o.sink_up = out->sink_up;
    o.trunc = out->trunc;
    o.flags = out->row_flags;
    o.status = W.status();
    o.capacity = -1;
    o.total_at = B.rows;
    const ImpactDesc *desc = W.desc(0);
    cudaError_t e = cudaMemsetAsync(bad, 0, 4, st);
    if (e == cudaSuccess)
        e = launch_mc_prep(samples, n, S, keys, val, val_dn, val_up, bad, range, st);
    if (e == cudaSuccess)
        e = launch_mc_rows(desc, false, B.rows, keys, S, range, val, val_dn, val_up,
                           (unsigned)kmin, o, st);
    if (e == cudaSuccess) e = launch_scan(out->row_ptr, B.rows, W.scan(), st);
    if (e != cudaSuccess) return done(fail(IMPACT_ERR_CUDA, cudaGetErrorString(e)));
    int64_t nnz = 0;
    uint32_t status = 0, nonfinite = 0;
    if (cudaMemcpyAsync(&nnz, out->row_ptr + B.rows, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&status, W.status(), 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&nonfinite, bad, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return done(fail(IMPACT_ERR_CUDA, "count pass failed"));
    if (nonfinite) return done(fail(IMPACT_ERR_ARG, "the draws must be finite"));
    if (status & IMPACT_STATUS_MC_WINDOW)
        return done(fail(IMPACT_ERR_ARG, "a row's cells within reach of the draws exceed " +
                                             std::to_string(IMPACT_MC_HIST_MAX) + " (or " +
                                             std::to_string(IMPACT_MC_EDGES_MAX) +
                                             " in one dimension): use a coarser grid"));
    int64_t capacity = out->nnz;
    if (lib_owned) {
        const size_t k = (size_t)std::max<int64_t>(nnz, 1);
        if (dev_malloc_async(&out->col, k * 4, st) != cudaSuccess ||
            dev_malloc_async(&out->lo, k * vbytes, st) != cudaSuccess ||
            dev_malloc_async(&out->up, k * vbytes, st) != cudaSuccess)
            return done(fail(IMPACT_ERR_OOM, "pair arrays"));
        capacity = nnz;
    }
    out->rows = B.rows;
    out->nnz = nnz;
    if (capacity < nnz)
        return done(fail(IMPACT_ERR_CAPACITY, "output capacity " + std::to_string(capacity) +
                                                  " < needed pairs " + std::to_string(nnz)));
    impact_csr view;
    if ((s = pair_view(out, view)) != IMPACT_OK) return done(s);
    o.col = view.col;
    o.lo = view.lo;
    o.up = view.up;
    o.capacity = capacity;
    e = launch_mc_rows(desc, true, B.rows, keys, S, range, val, val_dn, val_up, (unsigned)kmin,
                       o, st);
    if (e != cudaSuccess) return done(fail(IMPACT_ERR_CUDA, cudaGetErrorString(e)));
    if (cudaMemcpyAsync(&status, W.status(), 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return done(fail(IMPACT_ERR_CUDA, "emit pass failed"));
    if (status & IMPACT_STATUS_CAPACITY)
        return done(fail(IMPACT_ERR_CAPACITY, "output capacity too small"));
    return done(IMPACT_OK);
}
