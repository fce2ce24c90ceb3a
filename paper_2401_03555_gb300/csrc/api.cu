// api.cu -- the C ABI entry points (include/impact.h). A call works on a
// batch of builds (a single build is a batch of one): the planner (plan.cu)
// makes each build's descriptor and tables, this file lays them out with the
// batch index, the scan scratch and the per-row records in one device
// workspace, and runs the count -> scan -> emit pipeline on the caller's
// stream, directly or as a captured CUDA graph. It also holds the launch-shape
// autotuner of the FP32 walk.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/impact.h"
#include "alloc.h"
#include "impact_desc.h"
#include "kernels.h"
#include "pipeline.h"
#include "plan.h"

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace impact {
impact_status fail(impact_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace impact


#define CK(expr)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? IMPACT_ERR_OOM : IMPACT_ERR_CUDA,   \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));                 \
        }                                                                                     \
    } while (0)

namespace impact {

constexpr int kBatchMax = 1 << 16;   // builds per batch

uint64_t mix(uint64_t h, uint64_t v)
{
    for (int i = 0; i < 8; ++i) h = (h ^ ((v >> (8 * i)) & 0xff)) * 1099511628211ull;
    return h;
}

impact_status tuning_of(const impact_tuning *t, Tuning &T)
{
    T = Tuning();
    if (!t) return IMPACT_OK;
    if (t->count_warps) T.count_warps = t->count_warps;
    if (t->emit_warps) T.emit_warps = t->emit_warps;
    if (T.count_warps < 1 || T.count_warps > IMPACT_TREE_WARPS_MAX || T.emit_warps < 1 ||
        T.emit_warps > IMPACT_TREE_WARPS_MAX)
        return fail(IMPACT_ERR_ARG, "tuning: warps per block must be in [1, 8]");
    if (t->spin_limit < 0 || t->stall_row < 0 || t->fault_row < 0 || t->guard_row < 0 ||
        (t->one_pass != 0 && t->one_pass != 1))
        return fail(IMPACT_ERR_ARG,
                    "tuning: spin_limit, stall_row, fault_row and guard_row must be >= 0, "
                    "one_pass 0 or 1");
    T.one_pass = t->one_pass == 1;
    T.faults.spin_limit = t->spin_limit;
    T.faults.stall_row = t->stall_row - 1;
    T.faults.fault_row = t->fault_row - 1;
    T.faults.guard_row = t->guard_row - 1;
    return IMPACT_OK;
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------


impact_status make_batch(const impact_request *reqs, int count, impact_precision precision,
                         const impact_tuning *tuning, Batch &B)
{
    if (!reqs) return fail(IMPACT_ERR_ARG, "null request array");
    if (count < 1 || count > kBatchMax)
        return fail(IMPACT_ERR_ARG, "request count must be in [1, 65536]");
    impact_status s = tuning_of(tuning, B.tune);
    if (s != IMPACT_OK) return s;
    B.plans.assign(count, Plan());
    B.images.assign(count, nullptr);
    B.row_begin.assign(count + 1, 0);
    B.unit_begin.assign(count + 1, 0);
    B.prec = precision;
    uint64_t h = 1469598103934665603ull;
    for (int q = 0; q < count; ++q) {
        const impact_request &r = reqs[q];
        s = impact::make_plan(r.sys, r.grid, r.inputs, r.sigma, r.cutoff, precision, B.plans[q]);
        if (s != IMPACT_OK) {
            if (count > 1) g_last_error = "request " + std::to_string(q) + ": " + g_last_error;
            return s;
        }
        const Plan &P = B.plans[q];
        B.images[q] = r.sys->dev_images;
        B.row_begin[q + 1] = B.row_begin[q] + P.rows;
        const int64_t rpw = 32 / P.desc.n;
        B.unit_begin[q + 1] = B.unit_begin[q] + (P.rows + rpw - 1) / rpw;
        B.nnz_bound = (B.nnz_bound > INT64_MAX - P.nnz_bound) ? INT64_MAX
                                                              : B.nnz_bound + P.nnz_bound;
        if (precision == IMPACT_FP32_SOUND) {
            B.rec_max = std::max(B.rec_max, P.desc.rec_stride);
            for (int c = 0; c < 2; ++c)
                B.work_max[c] = std::max(B.work_max[c],
                                         impact::walk_work_bytes(P.desc.n, P.desc.leaf_cap, c == 1));
        }
        h = mix(h, P.hash);
    }
    B.rows = B.row_begin[count];
    B.units = B.unit_begin[count];
    B.hash = h;   // launch shapes change no result: they are not part of the identity
    if (precision == IMPACT_FP32_SOUND &&
        2 * (int64_t)B.rec_max + B.work_max[1] > IMPACT_WALK_SMEM_MAX)
        return fail(IMPACT_ERR_ARG,
                    "the builds of this batch together need " +
                        std::to_string(2 * (int64_t)B.rec_max + B.work_max[1]) +
                        " bytes of shared memory per warp, more than one warp has: "
                        "batch the widest windows separately");
    return IMPACT_OK;
}


BatchLayout batch_layout(const Batch &B)
{
    BatchLayout L;
    size_t o = 0;
    auto put = [&](size_t bytes) {
        size_t at = o;
        o = impact::align256(o + bytes);
        return at;
    };
    const int count = B.count();
    L.index = put(sizeof(BatchIndex));
    L.row_begin = put((size_t)(count + 1) * 8);
    L.unit_begin = put((size_t)(count + 1) * 8);
    L.descs = put((size_t)count * 8);
    L.recs = put((size_t)count * 8);
    L.tables.resize(count);
    L.tl.resize(count);
    for (int q = 0; q < count; ++q) {
        L.tl[q] = impact::table_layout(B.plans[q]);
        L.tables[q] = put(L.tl[q].total);
    }
    L.upload_end = o;
    L.status = put(64);
    L.counter = put(64);
    L.scan = put((size_t)impact::scan_scratch_elems(B.rows) * 8);
    L.lb = put(B.prec == PREC_FP32_SOUND ? (size_t)B.rows * 8 : 0);
    L.rec.resize(count);
    for (int q = 0; q < count; ++q) {
        const Plan &P = B.plans[q];
        L.rec[q] = put(B.prec == PREC_FP32_SOUND ? (size_t)P.rows * P.desc.rec_stride : 0);
    }
    L.total = o;
    return L;
}


std::mutex g_ws_mu;
std::unordered_map<const void *, uint64_t> g_ws_tag;   // caller workspace -> batch it holds

void ws_tag(const void *ws, uint64_t h)
{
    std::lock_guard<std::mutex> lock(g_ws_mu);
    if (h) g_ws_tag[ws] = h; else g_ws_tag.erase(ws);
}

bool ws_has(const void *ws, uint64_t h)
{
    std::lock_guard<std::mutex> lock(g_ws_mu);
    auto it = g_ws_tag.find(ws);
    return it != g_ws_tag.end() && it->second == h;
}

impact_status get_work(const Batch &B, const impact_csr *out, cudaStream_t st, Work &W)
{
    W.L = batch_layout(B);
    if (out && out->workspace) {
        if (out->workspace_bytes < (int64_t)W.L.total)
            return fail(IMPACT_ERR_ARG, "workspace too small: " +
                                            std::to_string(out->workspace_bytes) + " < " +
                                            std::to_string(W.L.total) + " bytes");
        if (((uintptr_t)out->workspace & 255) != 0)
            return fail(IMPACT_ERR_ARG, "workspace must be 256-byte aligned");
        W.base = (unsigned char *)out->workspace;
        W.owned = false;
        return IMPACT_OK;
    }
    CK(dev_malloc_async(&W.base, W.L.total, st));
    W.owned = true;
    return IMPACT_OK;
}

impact_status release(Work &W, cudaStream_t st)
{
    unsigned char *b = W.base;
    W.base = nullptr;
    if (W.owned && b) CK(dev_free_async(b, st));
    return IMPACT_OK;
}

// Releases a library-owned workspace on every return path that did not
// release it already.
struct WorkHold {
    Work &W;
    cudaStream_t st;
    ~WorkHold() { release(W, st); }
};

// Frees the arrays of a library-owned result (stream-ordered) and clears
// them, keeping the caller's workspace fields.
void free_owned(impact_csr *out, cudaStream_t st)
{
    void *ptrs[] = {out->row_ptr, out->col, out->lo, out->up, out->sink_lo,
                    out->sink_up, out->trunc, out->row_flags};
    for (void *p : ptrs) dev_free_async(p, st);
    void *ws = out->workspace;
    int64_t wsb = out->workspace_bytes;
    memset(out, 0, sizeof(*out));
    out->workspace = ws;
    out->workspace_bytes = wsb;
}

// Copies the batch index, the descriptors and the tables into the workspace.
impact_status upload(const Batch &B, Work &W, cudaStream_t st)
{
    const BatchLayout &L = W.L;
    const int count = B.count();
    std::vector<unsigned char> host(L.upload_end, 0);
    BatchIndex bi;
    memset(&bi, 0, sizeof(bi));
    bi.count = count;
    bi.rows = B.rows;
    bi.units = B.units;
    bi.row_begin = (const int64_t *)(W.base + L.row_begin);
    bi.unit_begin = (const int64_t *)(W.base + L.unit_begin);
    bi.desc = (const ImpactDesc *const *)(W.base + L.descs);
    bi.rec = (unsigned char *const *)(W.base + L.recs);
    bi.next_row = W.counter();
    memcpy(host.data() + L.index, &bi, sizeof(bi));
    memcpy(host.data() + L.row_begin, B.row_begin.data(), (size_t)(count + 1) * 8);
    memcpy(host.data() + L.unit_begin, B.unit_begin.data(), (size_t)(count + 1) * 8);
    for (int q = 0; q < count; ++q) {
        const ImpactDesc *d = W.desc(q);
        unsigned char *r = B.prec == PREC_FP32_SOUND ? W.base + L.rec[q] : nullptr;
        memcpy(host.data() + L.descs + 8 * (size_t)q, &d, 8);
        memcpy(host.data() + L.recs + 8 * (size_t)q, &r, 8);
        impact::pack_tables(B.plans[q], host.data() + L.tables[q], W.base + L.tables[q],
                            B.images[q]);
    }
    // pageable source: returns once the bytes are staged, so `host` may go
    CK(cudaMemcpyAsync(W.base, host.data(), host.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(W.status(), 0, 64, st));
    return IMPACT_OK;
}

void configure_pool_once()
{
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
        uint64_t keep = UINT64_MAX;   // keep freed blocks in the pool between builds
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    });
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

impact_status check_row_arrays(const impact_csr *out)
{
    if (!is_device_ptr(out->row_ptr) || !is_device_ptr(out->sink_lo) ||
        !is_device_ptr(out->sink_up) || !is_device_ptr(out->trunc))
        return fail(IMPACT_ERR_ARG, "row_ptr, sink_lo, sink_up and trunc must be device arrays");
    if (out->row_flags && !is_device_ptr(out->row_flags))
        return fail(IMPACT_ERR_ARG, "row_flags must be a device array or NULL");
    return IMPACT_OK;
}

impact_status status_result(uint32_t status)
{
    if (status & IMPACT_STATUS_TIMEOUT)
        return fail(IMPACT_ERR_TIMEOUT, "a row's look-back wait for the rows before it gave up");
    if (status & IMPACT_STATUS_INTERNAL)
        return fail(IMPACT_ERR_CUDA, "internal: the walk's step guard ran out");
    if (status & IMPACT_STATUS_TABLE_OVERFLOW)
        return fail(IMPACT_ERR_ARG,
                    "a row's window exceeded the planner's bound (caller images wider than "
                    "128 cells in a dimension): raise the cutoff or use fewer cells");
    if (status & IMPACT_STATUS_EMIT_MISMATCH)
        return fail(IMPACT_ERR_CUDA, "internal: the emit pass disagreed with the count pass");
    if (status & IMPACT_STATUS_UNSOUND)
        return fail(IMPACT_ERR_UNSOUND, "a row check proved a row-sum invariant violated");
    return IMPACT_OK;
}

// Row outputs of build q with row-indexed arrays shifted to its first row
// (the FP64 kernels index rows from 0 within a build).
impact::RowOutputs shifted(const impact::RowOutputs &o, int64_t rb, int64_t rows_total)
{
    impact::RowOutputs s = o;
    s.row_ptr = o.row_ptr + rb;
    if (o.sink_lo) s.sink_lo = o.sink_lo + rb;
    if (o.sink_up) s.sink_up = o.sink_up + rb;
    if (o.trunc) s.trunc = o.trunc + rb;
    if (o.flags) s.flags = o.flags + rb;
    s.total_at = rows_total - rb;
    return s;
}

// FP32 walk launches of one pass over the batch's rows, in chunks of
// `chunk_rows` rows (0: one launch) in row order on `st`; `counter` is the
// pass's row counter, reset before each launch.
cudaError_t walk_pass(const Batch &B, const Work &W, int mode, int warps,
                      const impact::RowOutputs &o, unsigned long long *counter,
                      int64_t chunk_rows, cudaStream_t st)
{
    const int64_t step = chunk_rows > 0 ? chunk_rows : std::max<int64_t>(B.rows, 1);
    for (int64_t r0 = 0; r0 < B.rows; r0 += step) {
        cudaError_t e = cudaMemsetAsync(counter, 0, 8, st);
        if (e == cudaSuccess)
            e = impact::launch_walk_fp32(W.index(), r0, std::min(B.rows, r0 + step),
                                         B.rec_max, B.work_max, warps, mode, o,
                                         mode == WALK_FUSED ? W.lb() : nullptr, B.tune.faults, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// count pass: row_ptr (row pointers and the total), sink_lo, sink_up, trunc,
// row_flags. FP32: one walk whose look-back writes the row pointers; FP64:
// per-row counts, then the scan.
impact_status run_count(const Batch &B, const Work &W, const impact_csr *out, cudaStream_t st,
                        int64_t chunk_rows)
{
    CK(cudaMemsetAsync(W.status(), 0, 64, st));
    impact::RowOutputs o{out->row_ptr, nullptr, nullptr, nullptr, out->sink_lo, out->sink_up,
                         out->trunc, out->row_flags, W.status(), -1, B.rows};
    if (B.prec == PREC_FP32_SOUND) {
        CK(impact::launch_setup_fp32(W.index(), B.units, W.status(), out->sink_lo, out->sink_up,
                                     out->trunc, st));
        CK(walk_pass(B, W, WALK_COUNT, B.tune.count_warps, o, W.counter(), chunk_rows, st));
        CK(impact::launch_scan(out->row_ptr, B.rows, W.scan(), st));
        return IMPACT_OK;
    }
    for (int q = 0; q < B.count(); ++q)
        CK(impact::launch_rows(W.desc(q), B.prec, false, 0, B.plans[q].rows,
                               shifted(o, B.row_begin[q], B.rows), st));
    CK(impact::launch_scan(out->row_ptr, B.rows, W.scan(), st));
    return IMPACT_OK;
}

// emit pass at the row pointers in out->row_ptr
impact_status run_emit(const Batch &B, const Work &W, const impact_csr *out, int64_t capacity,
                       bool records_ready, cudaStream_t st, int64_t chunk_rows)
{
    impact::RowOutputs o{out->row_ptr, out->col, out->lo, out->up, nullptr, nullptr, nullptr,
                         nullptr, W.status(), capacity, B.rows};
    if (B.prec == PREC_FP32_SOUND) {
        if (!records_ready)   // rebuild the records; the row outputs stay as counted
            CK(impact::launch_setup_fp32(W.index(), B.units, W.status(), nullptr, nullptr,
                                         nullptr, st));
        CK(walk_pass(B, W, WALK_EMIT, B.tune.emit_warps, o, W.counter() + 1, chunk_rows, st));
    } else {
        for (int q = 0; q < B.count(); ++q)
            CK(impact::launch_rows(W.desc(q), B.prec, true, 0, B.plans[q].rows,
                                   shifted(o, B.row_begin[q], B.rows), st));
    }
    return IMPACT_OK;
}

// the whole build into arrays of known capacity with no host round trip:
// count, scan and emit (the emit pass checks the total against the capacity
// on the device and writes nothing when it does not fit), or for FP32 with
// tuning one_pass a single walk in which each row finds its offset by the
// look-back and writes its pairs
impact_status run_fused(const Batch &B, const Work &W, const impact_csr *out, int64_t capacity,
                        cudaStream_t st, int64_t chunk_rows)
{
    if (B.prec != PREC_FP32_SOUND || !B.tune.one_pass) {
        impact_status s = run_count(B, W, out, st, chunk_rows);
        if (s != IMPACT_OK) return s;
        return run_emit(B, W, out, capacity, true, st, chunk_rows);
    }
    CK(cudaMemsetAsync(W.status(), 0, 64, st));
    CK(impact::launch_setup_fp32(W.index(), B.units, W.status(), out->sink_lo, out->sink_up,
                                 out->trunc, st));
    if (B.rows > 0) CK(cudaMemsetAsync(W.lb(), 0, (size_t)B.rows * 8, st));
    else CK(cudaMemsetAsync(out->row_ptr, 0, 8, st));
    impact::RowOutputs o{out->row_ptr, out->col, out->lo, out->up, out->sink_lo, out->sink_up,
                         out->trunc, out->row_flags, W.status(), capacity, B.rows};
    CK(walk_pass(B, W, WALK_FUSED, B.tune.count_warps, o, W.counter(), chunk_rows, st));
    return IMPACT_OK;
}

// col/lo/up may be device memory or pinned host memory the device can
// address (the emit pass then writes the pairs straight to host memory over
// the host link); `v` is `out` with device-visible addresses.
impact_status pair_view(const impact_csr *out, impact_csr &v)
{
    v = *out;
    if (out->nnz <= 0) return IMPACT_OK;
    void **ps[3] = {(void **)&v.col, &v.lo, &v.up};
    for (void **pp : ps) {
        cudaPointerAttributes a;
        if (!*pp || cudaPointerGetAttributes(&a, *pp) != cudaSuccess) {
            cudaGetLastError();
            return fail(IMPACT_ERR_ARG, "col, lo and up must be device or pinned host arrays");
        }
        if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) continue;
        if (a.type == cudaMemoryTypeHost && a.devicePointer) {
            *pp = a.devicePointer;
            continue;
        }
        return fail(IMPACT_ERR_ARG, "col, lo and up must be device or pinned host arrays");
    }
    return IMPACT_OK;
}

// ---------------------------------------------------------------------------
// the three phases behind the entry points
// ---------------------------------------------------------------------------

impact_status do_count(const Batch &B, impact_csr *out, cudaStream_t st)
{
    impact_status s;
    if ((s = check_row_arrays(out)) != IMPACT_OK) return s;
    configure_pool_once();
    Work W;
    if ((s = get_work(B, out, st, W)) != IMPACT_OK) return s;
    WorkHold hold{W, st};
    if (!W.owned) ws_tag(W.base, 0);
    if ((s = upload(B, W, st)) != IMPACT_OK) return s;
    if ((s = run_count(B, W, out, st)) != IMPACT_OK) return s;
    int64_t nnz = 0;
    uint32_t status = 0;
    CK(cudaMemcpyAsync(&nnz, out->row_ptr + B.rows, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&status, W.status(), 4, cudaMemcpyDeviceToHost, st));
    if ((s = release(W, st)) != IMPACT_OK) return s;
    CK(cudaStreamSynchronize(st));
    out->rows = B.rows;
    out->nnz = nnz;
    s = status_result(status);
    if (!W.owned && (s == IMPACT_OK || s == IMPACT_ERR_UNSOUND)) ws_tag(out->workspace, B.hash);
    return s;
}

impact_status do_emit(const Batch &B, impact_csr *out, cudaStream_t st)
{
    impact_status s;
    if (!is_device_ptr(out->row_ptr)) return fail(IMPACT_ERR_ARG, "row_ptr must be a device array");
    if (out->nnz < 0) return fail(IMPACT_ERR_ARG, "out->nnz (the capacity) must be >= 0");
    impact_csr view;
    if ((s = pair_view(out, view)) != IMPACT_OK) return s;
    configure_pool_once();
    bool ready = false;
    if (out->workspace) {
        if (!ws_has(out->workspace, B.hash))
            return fail(IMPACT_ERR_ARG,
                        "workspace was not filled by impact_count for these arguments");
        ready = true;
    }
    Work W;
    if ((s = get_work(B, out, st, W)) != IMPACT_OK) return s;
    WorkHold hold{W, st};
    if (!ready) {
        if ((s = upload(B, W, st)) != IMPACT_OK) return s;
    } else {
        CK(cudaMemsetAsync(W.status(), 0, 64, st));
    }
    if ((s = run_emit(B, W, &view, out->nnz, ready, st)) != IMPACT_OK) return s;
    uint32_t status = 0;
    CK(cudaMemcpyAsync(&status, W.status(), 4, cudaMemcpyDeviceToHost, st));
    if ((s = release(W, st)) != IMPACT_OK) return s;
    CK(cudaStreamSynchronize(st));
    out->rows = B.rows;
    if (status & IMPACT_STATUS_CAPACITY)
        return fail(IMPACT_ERR_CAPACITY, "row_ptr[rows] exceeds the capacity out->nnz");
    return status_result(status);
}

impact_status build_into(const Batch &B, impact_csr *out, bool lib_owned, cudaStream_t st)
{
    impact_status s;
    const size_t vbytes = B.prec == PREC_FP32_SOUND ? 4 : 8;
    if (lib_owned) {
        CK(dev_malloc_async(&out->row_ptr, (B.rows + 1) * 8, st));
        CK(dev_malloc_async(&out->sink_lo, B.rows * 8, st));
        CK(dev_malloc_async(&out->sink_up, B.rows * 8, st));
        CK(dev_malloc_async(&out->trunc, B.rows * 8, st));
        CK(dev_malloc_async(&out->row_flags, B.rows * 4, st));
    }
    Work W;
    if ((s = get_work(B, out, st, W)) != IMPACT_OK) return s;
    WorkHold hold{W, st};
    if (!W.owned) ws_tag(W.base, 0);
    if ((s = upload(B, W, st)) != IMPACT_OK) return s;
    int64_t capacity = out->nnz;
    if (lib_owned) {   // the output size is known after the count pass
        if ((s = run_count(B, W, out, st)) != IMPACT_OK) return s;
        int64_t nnz = 0;
        CK(cudaMemcpyAsync(&nnz, out->row_ptr + B.rows, 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        size_t k = (size_t)std::max<int64_t>(nnz, 1);
        CK(dev_malloc_async(&out->col, k * 4, st));
        CK(dev_malloc_async(&out->lo, k * vbytes, st));
        CK(dev_malloc_async(&out->up, k * vbytes, st));
        capacity = nnz;
        impact_csr view;
        if ((s = pair_view(out, view)) != IMPACT_OK) return s;
        if ((s = run_emit(B, W, &view, capacity, true, st)) != IMPACT_OK) return s;
    } else {   // caller capacity: no host round trip
        impact_csr view;
        if ((s = pair_view(out, view)) != IMPACT_OK) return s;
        if ((s = run_fused(B, W, &view, capacity, st)) != IMPACT_OK) return s;
    }
    int64_t nnz = 0;
    uint32_t status = 0;
    CK(cudaMemcpyAsync(&nnz, out->row_ptr + B.rows, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&status, W.status(), 4, cudaMemcpyDeviceToHost, st));
    if ((s = release(W, st)) != IMPACT_OK) return s;
    CK(cudaStreamSynchronize(st));
    out->rows = B.rows;
    out->nnz = nnz;
    if (status & IMPACT_STATUS_CAPACITY)
        return fail(IMPACT_ERR_CAPACITY, "output capacity " + std::to_string(capacity) +
                                             " < needed pairs " + std::to_string(nnz));
    return status_result(status);
}

impact_status do_build(const Batch &B, impact_csr *out, cudaStream_t st)
{
    configure_pool_once();
    const bool lib_owned = (out->col == nullptr);
    if (lib_owned) {
        void *ws = out->workspace;
        int64_t wsb = out->workspace_bytes;
        memset(out, 0, sizeof(*out));
        out->workspace = ws;
        out->workspace_bytes = wsb;
        out->owned = 1;
    } else {
        impact_status s;
        if ((s = check_row_arrays(out)) != IMPACT_OK) return s;
        if (out->nnz < 0) return fail(IMPACT_ERR_ARG, "out->nnz (the capacity) must be >= 0");
    }
    impact_status s = build_into(B, out, lib_owned, st);
    // a library-owned result that failed is released whole (an UNSOUND one is
    // complete and is kept: row_flags tells which rows)
    if (lib_owned && s != IMPACT_OK && s != IMPACT_ERR_UNSOUND) {
        std::string msg = g_last_error;
        free_owned(out, st);
        cudaStreamSynchronize(st);
        fail(s, msg);
    }
    return s;
}

impact_request single(const impact_system *sys, const impact_grid *grid,
                      const impact_inputs *inputs, const double *sigma, double cutoff)
{
    impact_request r;
    r.sys = sys;
    r.grid = grid;
    r.inputs = inputs;
    r.sigma = sigma;
    r.cutoff = cutoff;
    return r;
}

impact_status check_request_ptrs(const impact_request *reqs, int count)
{
    if (!reqs) return fail(IMPACT_ERR_ARG, "null request array");
    for (int q = 0; q < count; ++q)
        if (!reqs[q].sys || !reqs[q].grid || !reqs[q].inputs || !reqs[q].sigma)
            return fail(IMPACT_ERR_ARG, "request " + std::to_string(q) + ": null argument");
    return IMPACT_OK;
}

static_assert(IMPACT_REGION_BOXES == IMPACT_REGION_MAX_BOXES, "region box limits differ");

// Region boxes -> blocks of whole cells: in every dimension the cells whose
// centre (midpoint of the cell's edges, edges as the planner makes them)
// lies in the closed box. Boxes with no such cell are dropped; targets stay
// first. `disjoint`: refuse boxes that share a cell.
impact_status snap_regions(const impact_grid *grid, const impact_regions *reg, bool disjoint,
                           RegionBoxes &B)
{
    if (!grid || !grid->lo || !grid->hi || !grid->cells) return fail(IMPACT_ERR_ARG, "null grid");
    const int n = grid->n;
    if (n < 1 || n > IMPACT_MAX_DIM) return fail(IMPACT_ERR_ARG, "grid.n must be in [1, 8]");
    int64_t total = 1;
    for (int d = 0; d < n; ++d) {
        if (grid->cells[d] < 1) return fail(IMPACT_ERR_ARG, "cells must be >= 1");
        if (!(grid->lo[d] < grid->hi[d]) || !isfinite(grid->lo[d]) || !isfinite(grid->hi[d]))
            return fail(IMPACT_ERR_ARG, "grid needs finite lo < hi");
        total *= grid->cells[d];
        if (total >= ((int64_t)1 << 31)) return fail(IMPACT_ERR_ARG, "more than 2^31-1 cells");
    }
    if (!reg) return fail(IMPACT_ERR_ARG, "null regions");
    const int nt = reg->n_target, na = reg->n_avoid;
    if (nt < 0 || na < 0 || nt + na > IMPACT_REGION_MAX_BOXES)
        return fail(IMPACT_ERR_ARG, "region boxes: 0 <= n_target + n_avoid <= 16");
    if ((nt > 0 && (!reg->target_lo || !reg->target_hi)) ||
        (na > 0 && (!reg->avoid_lo || !reg->avoid_hi)))
        return fail(IMPACT_ERR_ARG, "null region box corners");
    memset(&B, 0, sizeof(B));
    B.n = n;
    for (int d = 0; d < n; ++d) B.cells[d] = grid->cells[d];
    for (int k = 0; k < nt + na; ++k) {
        const bool avoid = k >= nt;
        const double *lo = avoid ? reg->avoid_lo + (size_t)(k - nt) * n : reg->target_lo + (size_t)k * n;
        const double *hi = avoid ? reg->avoid_hi + (size_t)(k - nt) * n : reg->target_hi + (size_t)k * n;
        bool empty = false;
        for (int d = 0; d < n; ++d) {
            if (!isfinite(lo[d]) || !isfinite(hi[d]) || lo[d] > hi[d])
                return fail(IMPACT_ERR_ARG, "region boxes need finite lo <= hi");
            const int N = grid->cells[d];
            const double h = (grid->hi[d] - grid->lo[d]) / (double)N;
            auto edge = [&](int i) { return i >= N ? grid->hi[d] : grid->lo[d] + (double)i * h; };
            int f = -1, l = -2;
            for (int i = 0; i < N; ++i) {
                const double c = 0.5 * (edge(i) + edge(i + 1));
                if (c >= lo[d] && c <= hi[d]) {
                    if (f < 0) f = i;
                    l = i;
                }
            }
            if (f < 0) empty = true;
            B.first[B.count][d] = f;
            B.last[B.count][d] = l;
        }
        if (empty) continue;
        if (!avoid) ++B.n_target;
        ++B.count;
    }
    if (disjoint)
        for (int a = 0; a < B.count; ++a)
            for (int b = 0; b < a; ++b) {
                bool meet = true;
                for (int d = 0; d < n; ++d)
                    meet = meet && std::max(B.first[a][d], B.first[b][d]) <=
                                       std::min(B.last[a][d], B.last[b][d]);
                if (meet) return fail(IMPACT_ERR_ARG, "region boxes share cells");
            }
    return IMPACT_OK;
}

}  // namespace impact

using namespace impact;

// A captured pipeline: count, scan and emit of one batch into fixed caller
// buffers, replayed by impact_graph_launch.
struct impact_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t *h_result = nullptr;   // pinned: [0] nnz, [1] status
    unsigned char *own_ws = nullptr;
    int64_t rows = 0, capacity = 0;
};

extern "C" {

impact_status impact_plan(const impact_system *sys, const impact_grid *grid,
                          const impact_inputs *inputs, const double *sigma, double cutoff,
                          impact_precision precision, int64_t *rows, int64_t *nnz_upper_bound,
                          int64_t *bytes_upper_bound)
{
    impact_request r = single(sys, grid, inputs, sigma, cutoff);
    Batch B;
    impact_status s = make_batch(&r, 1, precision, nullptr, B);
    if (s != IMPACT_OK) return s;
    if (rows) *rows = B.rows;
    if (nnz_upper_bound) *nnz_upper_bound = B.nnz_bound;
    if (bytes_upper_bound) {
        int64_t per_pair = precision == IMPACT_FP32_SOUND ? 12 : 20;
        *bytes_upper_bound = B.nnz_bound * per_pair + (B.rows + 1) * 8 + B.rows * (3 * 8 + 4) +
                             (int64_t)batch_layout(B).total;
    }
    return IMPACT_OK;
}

impact_status impact_workspace_bytes(const impact_system *sys, const impact_grid *grid,
                                     const impact_inputs *inputs, const double *sigma,
                                     double cutoff, impact_precision precision, int64_t *bytes)
{
    impact_request r = single(sys, grid, inputs, sigma, cutoff);
    Batch B;
    impact_status s = make_batch(&r, 1, precision, nullptr, B);
    if (s != IMPACT_OK) return s;
    if (bytes) *bytes = (int64_t)batch_layout(B).total;
    return IMPACT_OK;
}

impact_status impact_count(const impact_system *sys, const impact_grid *grid,
                           const impact_inputs *inputs, const double *sigma, double cutoff,
                           impact_precision precision, impact_csr *out, void *stream)
{
    if (!out) return fail(IMPACT_ERR_ARG, "null output");
    impact_request r = single(sys, grid, inputs, sigma, cutoff);
    Batch B;
    impact_status s = make_batch(&r, 1, precision, nullptr, B);
    if (s != IMPACT_OK) return s;
    return do_count(B, out, (cudaStream_t)stream);
}

impact_status impact_emit(const impact_system *sys, const impact_grid *grid,
                          const impact_inputs *inputs, const double *sigma, double cutoff,
                          impact_precision precision, impact_csr *out, void *stream)
{
    if (!out) return fail(IMPACT_ERR_ARG, "null output");
    impact_request r = single(sys, grid, inputs, sigma, cutoff);
    Batch B;
    impact_status s = make_batch(&r, 1, precision, nullptr, B);
    if (s != IMPACT_OK) return s;
    return do_emit(B, out, (cudaStream_t)stream);
}

impact_status impact_build(const impact_system *sys, const impact_grid *grid,
                           const impact_inputs *inputs, const double *sigma, double cutoff,
                           impact_precision precision, impact_csr *out, void *stream)
{
    if (!out) return fail(IMPACT_ERR_ARG, "null output");
    impact_request r = single(sys, grid, inputs, sigma, cutoff);
    Batch B;
    impact_status s = make_batch(&r, 1, precision, nullptr, B);
    if (s != IMPACT_OK) return s;
    return do_build(B, out, (cudaStream_t)stream);
}

impact_status impact_batch_plan(const impact_request *reqs, int count, impact_precision precision,
                                const impact_tuning *tuning, int64_t *row_offsets,
                                int64_t *nnz_upper_bound, int64_t *workspace_bytes,
                                int64_t *upload_bytes)
{
    impact_status s = check_request_ptrs(reqs, count);
    if (s != IMPACT_OK) return s;
    Batch B;
    if ((s = make_batch(reqs, count, precision, tuning, B)) != IMPACT_OK) return s;
    if (row_offsets) memcpy(row_offsets, B.row_begin.data(), (size_t)(count + 1) * 8);
    if (nnz_upper_bound) *nnz_upper_bound = B.nnz_bound;
    if (workspace_bytes || upload_bytes) {
        const BatchLayout L = batch_layout(B);
        if (workspace_bytes) *workspace_bytes = (int64_t)L.total;
        if (upload_bytes) *upload_bytes = (int64_t)L.upload_end;
    }
    return IMPACT_OK;
}

impact_status impact_batch_count(const impact_request *reqs, int count,
                                 impact_precision precision, const impact_tuning *tuning,
                                 impact_csr *out, void *stream)
{
    if (!out) return fail(IMPACT_ERR_ARG, "null output");
    impact_status s = check_request_ptrs(reqs, count);
    if (s != IMPACT_OK) return s;
    Batch B;
    if ((s = make_batch(reqs, count, precision, tuning, B)) != IMPACT_OK) return s;
    return do_count(B, out, (cudaStream_t)stream);
}

impact_status impact_batch_emit(const impact_request *reqs, int count,
                                impact_precision precision, const impact_tuning *tuning,
                                impact_csr *out, void *stream)
{
    if (!out) return fail(IMPACT_ERR_ARG, "null output");
    impact_status s = check_request_ptrs(reqs, count);
    if (s != IMPACT_OK) return s;
    Batch B;
    if ((s = make_batch(reqs, count, precision, tuning, B)) != IMPACT_OK) return s;
    return do_emit(B, out, (cudaStream_t)stream);
}

impact_status impact_batch_build(const impact_request *reqs, int count,
                                 impact_precision precision, const impact_tuning *tuning,
                                 impact_csr *out, void *stream)
{
    if (!out) return fail(IMPACT_ERR_ARG, "null output");
    impact_status s = check_request_ptrs(reqs, count);
    if (s != IMPACT_OK) return s;
    Batch B;
    if ((s = make_batch(reqs, count, precision, tuning, B)) != IMPACT_OK) return s;
    return do_build(B, out, (cudaStream_t)stream);
}

impact_status impact_graph_create(const impact_request *reqs, int count,
                                  impact_precision precision, const impact_tuning *tuning,
                                  const impact_csr *out, void *stream, impact_graph **graph)
{
    if (!out || !graph) return fail(IMPACT_ERR_ARG, "null output or graph handle");
    *graph = nullptr;
    impact_status s = check_request_ptrs(reqs, count);
    if (s != IMPACT_OK) return s;
    Batch B;
    if ((s = make_batch(reqs, count, precision, tuning, B)) != IMPACT_OK) return s;
    if ((s = check_row_arrays(out)) != IMPACT_OK) return s;
    if (!out->col) return fail(IMPACT_ERR_ARG, "a graph writes into caller-owned col/lo/up");
    if (out->nnz < 0) return fail(IMPACT_ERR_ARG, "out->nnz (the capacity) must be >= 0");
    impact_csr view;
    if ((s = pair_view(out, view)) != IMPACT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    impact_graph *g = new impact_graph();
    g->rows = B.rows;
    g->capacity = out->nnz;
    Work W;
    W.L = batch_layout(B);
    auto cleanup = [&](impact_status r) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        host_free(g->h_result);
        dev_free(g->own_ws);
        delete g;
        return r;
    };
    if (out->workspace) {
        if (out->workspace_bytes < (int64_t)W.L.total || ((uintptr_t)out->workspace & 255))
            return cleanup(fail(IMPACT_ERR_ARG, "workspace too small or not 256-byte aligned"));
        W.base = (unsigned char *)out->workspace;
        ws_tag(W.base, 0);
    } else {
        cudaError_t e = dev_malloc(&g->own_ws, W.L.total);
        if (e != cudaSuccess) return cleanup(fail(IMPACT_ERR_OOM, cudaGetErrorString(e)));
        W.base = g->own_ws;
    }
    if (host_malloc(&g->h_result, 16) != cudaSuccess)
        return cleanup(fail(IMPACT_ERR_OOM, "pinned result word"));
    if ((s = upload(B, W, st)) != IMPACT_OK) return cleanup(s);
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return cleanup(fail(IMPACT_ERR_CUDA, "upload before capture failed"));
    // capture on a private stream: the caller's may be the legacy default one
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup(fail(IMPACT_ERR_CUDA, "capture stream"));
    impact_csr o = view;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        s = run_fused(B, W, &o, g->capacity, cs);
        if (s == IMPACT_OK) {
            cudaMemcpyAsync(g->h_result, o.row_ptr + B.rows, 8, cudaMemcpyDeviceToHost, cs);
            cudaMemcpyAsync(g->h_result + 1, W.status(), 4, cudaMemcpyDeviceToHost, cs);
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &g->graph);
        if (s == IMPACT_OK && e2 != cudaSuccess) s = fail(IMPACT_ERR_CUDA, cudaGetErrorString(e2));
    } else {
        s = fail(IMPACT_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaStreamDestroy(cs);
    if (s != IMPACT_OK) return cleanup(s);
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) return cleanup(fail(IMPACT_ERR_CUDA, cudaGetErrorString(e)));
    *graph = g;
    return IMPACT_OK;
}

impact_status impact_graph_launch(impact_graph *graph, void *stream)
{
    if (!graph || !graph->exec) return fail(IMPACT_ERR_ARG, "null graph");
    graph->h_result[0] = -1;
    graph->h_result[1] = 0;
    CK(cudaGraphLaunch(graph->exec, (cudaStream_t)stream));
    return IMPACT_OK;
}

impact_status impact_graph_result(impact_graph *graph, int64_t *nnz)
{
    if (!graph) return fail(IMPACT_ERR_ARG, "null graph");
    const int64_t got = graph->h_result[0];
    const uint32_t status = (uint32_t)graph->h_result[1];
    if (nnz) *nnz = got;
    if (got < 0) return fail(IMPACT_ERR_ARG, "no finished launch: synchronize the stream first");
    if (status & IMPACT_STATUS_CAPACITY)
        return fail(IMPACT_ERR_CAPACITY, "output capacity " + std::to_string(graph->capacity) +
                                             " < needed pairs " + std::to_string(got));
    return status_result(status);
}

impact_status impact_graph_destroy(impact_graph *graph)
{
    if (!graph) return IMPACT_OK;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    host_free(graph->h_result);
    dev_free(graph->own_ws);
    delete graph;
    return IMPACT_OK;
}

impact_status impact_batch_tune(const impact_request *reqs, int count,
                                impact_precision precision, impact_csr *out, int reps,
                                void *stream, impact_tuning *best, double *best_ms)
{
    if (!out || !best) return fail(IMPACT_ERR_ARG, "null output or result");
    if (precision != IMPACT_FP32_SOUND)
        return fail(IMPACT_ERR_ARG, "the autotuner tunes the FP32-sound walk");
    impact_status s = check_request_ptrs(reqs, count);
    if (s != IMPACT_OK) return s;
    if ((s = check_row_arrays(out)) != IMPACT_OK) return s;
    impact_csr view;
    if ((s = pair_view(out, view)) != IMPACT_OK) return s;
    out = &view;
    reps = std::max(1, std::min(reps, 50));
    cudaStream_t st = (cudaStream_t)stream;
    configure_pool_once();
    Batch B0;
    if ((s = make_batch(reqs, count, precision, nullptr, B0)) != IMPACT_OK) return s;
    Work W;
    impact_csr wout = *out;
    wout.workspace = nullptr;   // the tuner keeps its own scratch
    if ((s = get_work(B0, &wout, st, W)) != IMPACT_OK) return s;
    WorkHold hold{W, st};
    if ((s = upload(B0, W, st)) != IMPACT_OK) return s;
    if ((s = run_count(B0, W, out, st)) != IMPACT_OK) return s;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // pass 0: count, 1: emit
    auto timed = [&](int warps, int pass, double &ms) -> impact_status {
        Batch B = B0;
        B.tune.count_warps = B.tune.emit_warps = warps;
        ms = 1e30;
        for (int i = 0; i < reps; ++i) {
            CK(cudaEventRecord(e0, st));
            impact_status r = pass == 0 ? run_count(B, W, out, st)
                                        : run_emit(B, W, out, out->nnz, true, st);
            if (r != IMPACT_OK) return r;
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float f = 0.0f;
            CK(cudaEventElapsedTime(&f, e0, e1));
            ms = std::min(ms, (double)f);
        }
        uint32_t status = 0;
        CK(cudaMemcpy(&status, W.status(), 4, cudaMemcpyDeviceToHost));
        if (status & ~IMPACT_STATUS_UNSOUND) ms = 1e30;   // a shape that cannot run this batch
        return IMPACT_OK;
    };
    const bool can_emit = out->col != nullptr;
    const int warps[4] = {2, 4, 6, 8};
    impact_tuning tb;
    memset(&tb, 0, sizeof(tb));
    double best_a = 1e30, best_b = 1e30;
    // the count shape, then (with output arrays) the emit shape
    for (int w : warps) {
        double ms;
        if ((s = timed(w, 0, ms)) != IMPACT_OK) break;
        if (ms < best_a) {
            best_a = ms;
            tb.count_warps = w;
        }
    }
    if (s == IMPACT_OK && can_emit)
        for (int w : warps) {
            double ms;
            if ((s = timed(w, 1, ms)) != IMPACT_OK) break;
            if (ms < best_b) {
                best_b = ms;
                tb.emit_warps = w;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    impact_status r2 = release(W, st);
    if (s != IMPACT_OK) return s;
    if (r2 != IMPACT_OK) return r2;
    if (best_a >= 1e30) return fail(IMPACT_ERR_ARG, "no launch shape ran this batch");
    if (tb.emit_warps == 0) tb.emit_warps = IMPACT_TREE_WARPS;
    *best = tb;
    if (best_ms) *best_ms = best_a + (can_emit && best_b < 1e30 ? best_b : 0.0);
    return IMPACT_OK;
}

impact_status impact_free(impact_csr *out)
{
    if (!out) return fail(IMPACT_ERR_ARG, "null output");
    if (!out->owned) return IMPACT_OK;
    void *ptrs[] = {out->row_ptr, out->col, out->lo, out->up, out->sink_lo,
                    out->sink_up, out->trunc, out->row_flags};
    for (void *p : ptrs)
        if (p) CK(dev_free(p));
    void *ws = out->workspace;
    int64_t wsb = out->workspace_bytes;
    memset(out, 0, sizeof(*out));
    out->workspace = ws;
    out->workspace_bytes = wsb;
    return IMPACT_OK;
}

const char *impact_last_error(void) { return g_last_error.c_str(); }

impact_status impact_label_cells(const impact_grid *grid, const impact_regions *regions,
                                 uint8_t *labels, void *stream)
{
    RegionBoxes B;
    impact_status s = snap_regions(grid, regions, false, B);
    if (s != IMPACT_OK) return s;
    if (!is_device_ptr(labels)) return fail(IMPACT_ERR_ARG, "labels must be a device array");
    int64_t total = 1;
    for (int d = 0; d < grid->n; ++d) total *= grid->cells[d];
    cudaError_t e = launch_labels(B, total, labels, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(IMPACT_ERR_CUDA, cudaGetErrorString(e));
    return IMPACT_OK;
}

impact_status impact_region_vectors(const impact_system *sys, const impact_grid *grid,
                                    const impact_inputs *inputs, const double *sigma,
                                    const impact_regions *regions, impact_region_mode mode,
                                    impact_precision precision, double *r_lo, double *r_up,
                                    double *a_lo, double *a_up, void *stream)
{
    if (mode != IMPACT_REGION_BOX && mode != IMPACT_REGION_CELL_SUM)
        return fail(IMPACT_ERR_ARG, "unknown region mode");
    if (precision != IMPACT_FP32_SOUND && precision != IMPACT_FP64_PLAIN)
        return fail(IMPACT_ERR_ARG, "unknown precision");
    if (!sys || !grid || !inputs || !sigma) return fail(IMPACT_ERR_ARG, "null argument");
    RegionBoxes B;
    impact_status s = snap_regions(grid, regions, true, B);
    if (s != IMPACT_OK) return s;
    if (!is_device_ptr(r_lo) || !is_device_ptr(r_up) || !is_device_ptr(a_lo) ||
        !is_device_ptr(a_up))
        return fail(IMPACT_ERR_ARG, "the region vectors must be device arrays");
    configure_pool_once();
    cudaStream_t st = (cudaStream_t)stream;
    // the FP64 tables of the build (images in both roundings); the cutoff
    // does not enter the vectors, and one near 1 keeps the planner's windows
    // small
    impact_request req = single(sys, grid, inputs, sigma, 0.999);
    Batch batch;
    s = make_batch(&req, 1, IMPACT_FP64_PLAIN, nullptr, batch);
    if (s != IMPACT_OK) return s;
    Work W;
    s = get_work(batch, nullptr, st, W);
    if (s != IMPACT_OK) return s;
    WorkHold hold{W, st};
    s = upload(batch, W, st);
    if (s == IMPACT_OK) {
        cudaError_t e = launch_regions(W.desc(0), batch.rows, B, mode == IMPACT_REGION_CELL_SUM,
                                       precision == IMPACT_FP32_SOUND, r_lo, r_up, a_lo, a_up, st);
        if (e != cudaSuccess) s = fail(IMPACT_ERR_CUDA, cudaGetErrorString(e));
    }
    impact_status r = release(W, st);
    return s != IMPACT_OK ? s : r;
}

int impact_version(void) { return 301; }

}  // extern "C"
