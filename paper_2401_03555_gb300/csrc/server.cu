// server.cu -- the serving runtime (impact_server_*, include/impact.h).
//
// Requests (single builds) arrive from any host thread. One scheduler thread
// owns every CUDA call: it admits waiting requests in arrival order as long as
// their workspace and row arrays fit the device-memory budget, and launches
// them together as one batch count (one persistent launch per kernel for the
// whole group). When a group's count has finished, its exact output size is
// known; the group is emitted as soon as that output fits the budget, and
// its scratch is freed when the emit finishes. Groups run on a small pool of
// streams, so a group counting overlaps another group emitting, and requests
// that arrive while groups are on the device join the next group (continuous
// batching). Results stay on the device until the client releases them.
//
// Every row is computed by the same kernels with the same launch shapes
// whatever group it lands in, so a result is bitwise the same alone and in
// any mix.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/impact.h"
#include "alloc.h"
#include "pipeline.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// A request with deep copies of every host array it points to.
struct Request {
    int64_t ticket = 0;
    std::vector<double> A, B, c, lo, hi, pts, sigma;
    std::vector<int32_t> cells;
    impact_system sys{};
    impact_grid grid{};
    impact_inputs inputs{};
    double cutoff = 0.0;
    int64_t rows = 0;
    int64_t admit_bytes = 0;   // workspace + row arrays of this request alone
    Clock::time_point t_submit, t_done;
    Clock::time_point t_admit, t_counted, t_emit;   // group launched, counted, emit launched
    enum State { WAITING, RUNNING, DONE, FAILED } state = WAITING;
    impact_status status = IMPACT_OK;
    std::string error;
    struct Group *group = nullptr;
    int index = 0;             // position in its group
    int64_t nnz = 0;
    bool released = false;

    impact_request req() const
    {
        impact_request r;
        r.sys = &sys;
        r.grid = &grid;
        r.inputs = &inputs;
        r.sigma = sigma.data();
        r.cutoff = cutoff;
        return r;
    }
};

// One batch on the device.
struct Group {
    std::vector<Request *> reqs;
    impact::Batch B;
    impact::Work W;
    cudaStream_t stream = nullptr;
    int64_t rows = 0;
    int64_t *row_ptr = nullptr;
    double *sink_lo = nullptr, *sink_up = nullptr, *trunc = nullptr;
    uint32_t *flags = nullptr;
    int32_t *col = nullptr;
    void *lo = nullptr, *up = nullptr;
    int64_t *h_ptr = nullptr;        // pinned: row_ptr at every request's first row, and total
    uint32_t *h_status = nullptr;    // pinned
    cudaEvent_t ev_count = nullptr, ev_emit = nullptr;
    int64_t ws_bytes = 0, row_bytes = 0, pair_bytes = 0;
    int64_t held = 0;                // bytes of this group counted in the server's `used`
    int64_t nnz = 0;
    enum State { COUNTING, COUNTED, EMITTING, DONE } state = COUNTING;
    int64_t chunk_rows = 0;          // rows per walk launch (0: one launch)
    int live = 0;                    // requests not yet released
};

}  // namespace

struct impact_server {
    impact_server_config cfg{};
    int device = 0;
    int64_t budget = 0;
    std::vector<cudaStream_t> streams;
    cudaStream_t fast_stream = nullptr;   // high priority: small groups
    int next_stream = 0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> waiting;
    std::vector<Group *> groups;
    std::unordered_map<int64_t, Request *> reqs;
    int64_t next_ticket = 1;
    int64_t used = 0;                // device bytes held by groups
    bool emit_blocked = false;       // a counted group waits for output memory
    bool stop = false;
    std::thread worker;

    // counters
    int64_t completed = 0, pairs_done = 0, launched_groups = 0;
    std::string fatal;

    void run();
    bool step();                     // one scheduling pass; true if anything changed
    void admit();
    void fail_request(Request *r, impact_status s, const std::string &msg);
    void free_group(Group *g);
};

namespace {

int64_t row_bytes_of(int64_t rows) { return (rows + 1) * 8 + rows * (3 * 8 + 4); }

// Groups of at most kSmallRows rows run on the high-priority stream in one
// launch per pass; larger ones run their passes in chunks of kChunkRows rows.
constexpr int64_t kSmallRows = (int64_t)1 << 18;
constexpr int64_t kChunkRows = (int64_t)1 << 18;

int64_t align_up(int64_t x) { return (x + 255) & ~(int64_t)255; }

}  // namespace

void impact_server::fail_request(Request *r, impact_status s, const std::string &msg)
{
    r->state = Request::FAILED;
    r->status = s;
    r->error = msg;
    r->t_done = Clock::now();
    cv_done.notify_all();
}

void impact_server::free_group(Group *g)
{
    cudaStream_t st = g->stream;
    void *ptrs[] = {g->row_ptr, g->sink_lo, g->sink_up, g->trunc, g->flags,
                    g->col, g->lo, g->up};
    for (void *p : ptrs) impact::dev_free_async(p, st);
    impact::dev_free_async(g->W.base, st);
    if (g->h_ptr || g->h_status) cudaStreamSynchronize(st);   // pinned words the stream writes
    impact::host_free(g->h_ptr);
    impact::host_free(g->h_status);
    if (g->ev_count) cudaEventDestroy(g->ev_count);
    if (g->ev_emit) cudaEventDestroy(g->ev_emit);
    used -= g->held;
    delete g;
}

// Forms one group from the head of the waiting queue and launches its count.
void impact_server::admit()
{
    const int max_batch = cfg.max_batch > 0 ? cfg.max_batch : 64;
    const int64_t max_rows = cfg.max_group_rows > 0 ? cfg.max_group_rows : ((int64_t)1 << 22);
    const int max_groups = ((int)streams.size() + 1) * 2;
    int inflight = 0;
    for (Group *g : groups)
        if (g->state != Group::DONE) ++inflight;
    if (waiting.empty() || inflight >= max_groups || emit_blocked) return;
    std::vector<Request *> take;
    int64_t need = 0, rows = 0;
    while (!waiting.empty() && (int)take.size() < max_batch) {
        Request *r = waiting.front();
        if (r->admit_bytes > budget) {   // can never fit
            waiting.pop_front();
            fail_request(r, IMPACT_ERR_OOM, "request needs more device memory than the budget");
            continue;
        }
        if (used + need + r->admit_bytes > budget) break;
        if (!take.empty() && rows + r->rows > max_rows) break;
        need += r->admit_bytes;
        rows += r->rows;
        take.push_back(r);
        waiting.pop_front();
    }
    if (take.empty()) return;
    Group *g = new Group();
    g->reqs = take;
    g->live = (int)take.size();
    std::vector<impact_request> rq;
    for (Request *r : take) rq.push_back(r->req());
    impact_status s = impact::make_batch(rq.data(), (int)rq.size(), cfg.precision, nullptr, g->B);
    auto bail = [&](impact_status st, const std::string &m) {
        for (Request *r : take) fail_request(r, st, m);
        g->live = 0;
        g->state = Group::DONE;
        groups.push_back(g);
    };
    if (s != IMPACT_OK) return bail(s, impact_last_error());
    // small groups go to the high-priority stream, large ones take turns on
    // the others and run in chunks of rows, so that the SMs a large group
    // frees between its chunks go to the small groups first
    if (rq.size() > 0 && g->B.rows <= kSmallRows) {
        g->stream = fast_stream;
        g->chunk_rows = 0;
    } else {
        g->stream = streams[next_stream];
        next_stream = (next_stream + 1) % (int)streams.size();
        g->chunk_rows = kChunkRows;
    }
    cudaStream_t st = g->stream;
    g->rows = g->B.rows;
    g->W.L = impact::batch_layout(g->B);
    g->ws_bytes = align_up((int64_t)g->W.L.total);
    g->row_bytes = align_up(row_bytes_of(g->rows));
    cudaError_t e = impact::dev_malloc_async(&g->W.base, g->W.L.total, st);
    if (e == cudaSuccess) e = impact::dev_malloc_async(&g->row_ptr, (g->rows + 1) * 8, st);
    if (e == cudaSuccess) e = impact::dev_malloc_async(&g->sink_lo, g->rows * 8, st);
    if (e == cudaSuccess) e = impact::dev_malloc_async(&g->sink_up, g->rows * 8, st);
    if (e == cudaSuccess) e = impact::dev_malloc_async(&g->trunc, g->rows * 8, st);
    if (e == cudaSuccess) e = impact::dev_malloc_async(&g->flags, g->rows * 4, st);
    if (e == cudaSuccess) e = impact::host_malloc(&g->h_ptr, (take.size() + 1) * 8);
    if (e == cudaSuccess) e = impact::host_malloc(&g->h_status, 64);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_count, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_emit, cudaEventDisableTiming);
    g->held = g->ws_bytes + g->row_bytes;
    used += g->held;
    groups.push_back(g);
    if (e != cudaSuccess) {
        for (Request *r : take)
            fail_request(r, IMPACT_ERR_OOM, std::string("allocation: ") + cudaGetErrorString(e));
        g->live = 0;
        g->state = Group::DONE;
        return;
    }
    const Clock::time_point t_admit = Clock::now();
    for (size_t q = 0; q < take.size(); ++q) {
        take[q]->group = g;
        take[q]->index = (int)q;
        take[q]->state = Request::RUNNING;
        take[q]->t_admit = take[q]->t_counted = take[q]->t_emit = t_admit;
    }
    impact_csr out{};
    out.row_ptr = g->row_ptr;
    out.sink_lo = g->sink_lo;
    out.sink_up = g->sink_up;
    out.trunc = g->trunc;
    out.row_flags = g->flags;
    s = impact::upload(g->B, g->W, st);
    if (s == IMPACT_OK) s = impact::run_count(g->B, g->W, &out, st, g->chunk_rows);
    if (s == IMPACT_OK) {
        for (size_t q = 0; q <= take.size(); ++q)
            cudaMemcpyAsync(g->h_ptr + q, g->row_ptr + g->B.row_begin[q], 8,
                            cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(g->h_status, g->W.status(), 4, cudaMemcpyDeviceToHost, st);
        if (cudaEventRecord(g->ev_count, st) != cudaSuccess) s = IMPACT_ERR_CUDA;
    }
    if (s != IMPACT_OK) {
        for (Request *r : take) fail_request(r, s, impact_last_error());
        g->state = Group::DONE;
        return;
    }
    g->state = Group::COUNTING;
    ++launched_groups;
}

bool impact_server::step()
{
    bool changed = false;
    const int64_t per_pair = cfg.precision == IMPACT_FP32_SOUND ? 12 : 20;
    // groups start their emit strictly in arrival order, and a group's output
    // must fit beside what it and the earlier groups hold (later groups only
    // hold count-phase scratch, and no new group is admitted while one waits)
    emit_blocked = false;
    bool earlier_pending = false;    // an earlier group has not started its emit
    int64_t held_so_far = 0;
    for (size_t i = 0; i < groups.size(); ++i) {
        Group *g = groups[i];
        held_so_far += g->held;
        if (g->state == Group::COUNTING && cudaEventQuery(g->ev_count) == cudaSuccess) {
            g->state = Group::COUNTED;
            g->nnz = g->h_ptr[g->reqs.size()];
            const Clock::time_point now = Clock::now();
            for (size_t q = 0; q < g->reqs.size(); ++q) {
                g->reqs[q]->nnz = g->h_ptr[q + 1] - g->h_ptr[q];
                g->reqs[q]->t_counted = g->reqs[q]->t_emit = now;
            }
            changed = true;
        }
        if (g->state == Group::COUNTED && !earlier_pending) {
            const int64_t pb = align_up(std::max<int64_t>(g->nnz, 1) * per_pair);
            if (held_so_far + pb > budget && held_so_far > g->held) {   // wait for memory
                emit_blocked = true;
                earlier_pending = true;
                continue;
            }
            held_so_far += pb;
            cudaStream_t st = g->stream;
            const size_t vb = per_pair == 12 ? 4 : 8;
            const size_t k = (size_t)std::max<int64_t>(g->nnz, 1);
            cudaError_t e = impact::dev_malloc_async(&g->col, k * 4, st);
            if (e == cudaSuccess) e = impact::dev_malloc_async(&g->lo, k * vb, st);
            if (e == cudaSuccess) e = impact::dev_malloc_async(&g->up, k * vb, st);
            g->pair_bytes = pb;
            g->held += pb;
            used += pb;
            impact_status s = e == cudaSuccess ? IMPACT_OK : IMPACT_ERR_OOM;
            impact_csr out{};
            out.row_ptr = g->row_ptr;
            out.col = g->col;
            out.lo = g->lo;
            out.up = g->up;
            out.nnz = g->nnz;
            if (s == IMPACT_OK) s = impact::run_emit(g->B, g->W, &out, g->nnz, true, st, g->chunk_rows);
            if (s == IMPACT_OK) {
                cudaMemcpyAsync(g->h_status, g->W.status(), 4, cudaMemcpyDeviceToHost, st);
                if (cudaEventRecord(g->ev_emit, st) != cudaSuccess) s = IMPACT_ERR_CUDA;
            }
            if (s != IMPACT_OK) {
                for (Request *r : g->reqs) fail_request(r, s, "emit launch failed");
                g->state = Group::DONE;
            } else {
                g->state = Group::EMITTING;
                const Clock::time_point now = Clock::now();
                for (Request *r : g->reqs) r->t_emit = now;
            }
            changed = true;
        }
        if (g->state == Group::COUNTING || g->state == Group::COUNTED) earlier_pending = true;
        if (g->state == Group::EMITTING && cudaEventQuery(g->ev_emit) == cudaSuccess) {
            const Clock::time_point now = Clock::now();
            const impact_status s = impact::status_result(*g->h_status);
            for (Request *r : g->reqs) {
                if (r->state == Request::FAILED) continue;
                r->t_done = now;
                if (s == IMPACT_OK || s == IMPACT_ERR_UNSOUND) {
                    r->state = Request::DONE;
                    r->status = s;
                    ++completed;
                    pairs_done += r->nnz;
                } else {
                    fail_request(r, s, impact_last_error());
                }
            }
            impact::dev_free_async(g->W.base, g->stream);   // the tables are not needed any more
            g->W.base = nullptr;
            g->held -= g->ws_bytes;
            used -= g->ws_bytes;
            g->state = Group::DONE;
            changed = true;
            cv_done.notify_all();
        }
    }
    // groups whose every request was released
    for (size_t i = 0; i < groups.size();) {
        Group *g = groups[i];
        if (g->state == Group::DONE && g->live == 0) {
            free_group(g);
            groups.erase(groups.begin() + i);
            changed = true;
        } else {
            ++i;
        }
    }
    const size_t before = waiting.size();
    admit();
    if (waiting.size() != before) changed = true;
    return changed;
}

void impact_server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    while (true) {
        bool busy = false;
        for (Group *g : groups)
            if (g->state != Group::DONE) busy = true;
        if (stop && !busy && waiting.empty()) break;
        const bool changed = step();
        if (!changed) {
            if (busy || !waiting.empty())
                cv_work.wait_for(lock, std::chrono::microseconds(50));
            else
                cv_work.wait_for(lock, std::chrono::milliseconds(5));
        }
    }
}

extern "C" {

impact_status impact_server_create(const impact_server_config *config, impact_server **server)
{
    if (!config || !server) return impact::fail(IMPACT_ERR_ARG, "null config or handle");
    *server = nullptr;
    if (config->precision != IMPACT_FP32_SOUND && config->precision != IMPACT_FP64_PLAIN)
        return impact::fail(IMPACT_ERR_ARG, "unknown precision");
    if (config->streams < 0 || config->streams > 8 || config->max_batch < 0 ||
        config->memory_budget < 0 || config->max_group_rows < 0)
        return impact::fail(IMPACT_ERR_ARG, "streams must be in [0, 8], sizes >= 0");
    impact_server *S = new impact_server();
    S->cfg = *config;
    cudaGetDevice(&S->device);
    impact::configure_pool_once();
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete S;
        return impact::fail(IMPACT_ERR_CUDA, "cudaMemGetInfo failed");
    }
    S->budget = config->memory_budget > 0 ? config->memory_budget : (int64_t)(free_b * 0.8);
    const int ns = config->streams > 0 ? config->streams : 2;
    int lowest = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&lowest, &greatest);
    for (int i = 0; i <= ns; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, i == ns ? greatest : lowest) !=
            cudaSuccess) {
            for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
            if (S->fast_stream) cudaStreamDestroy(S->fast_stream);
            delete S;
            return impact::fail(IMPACT_ERR_CUDA, "stream creation failed");
        }
        if (i == ns) S->fast_stream = st;
        else S->streams.push_back(st);
    }
    S->worker = std::thread([S] { S->run(); });
    *server = S;
    return IMPACT_OK;
}

impact_status impact_server_submit(impact_server *S, const impact_request *request,
                                   int64_t *ticket)
{
    if (!S || !request || !ticket) return impact::fail(IMPACT_ERR_ARG, "null argument");
    const impact_request &q = *request;
    if (!q.sys || !q.grid || !q.inputs || !q.sigma)
        return impact::fail(IMPACT_ERR_ARG, "null request field");
    // check the arguments now (host only) and size the request
    impact::Batch B;
    impact_status s = impact::make_batch(request, 1, S->cfg.precision, nullptr, B);
    if (s != IMPACT_OK) return s;
    Request *r = new Request();
    const int n = q.grid->n, m = q.inputs->m, cnt = q.inputs->count;
    auto copy = [](const double *p, size_t k) {
        return p ? std::vector<double>(p, p + k) : std::vector<double>();
    };
    r->sys = *q.sys;
    if (q.sys->kind == IMPACT_AFFINE) {
        r->A = copy(q.sys->A, (size_t)n * n);
        r->B = copy(q.sys->B, (size_t)n * m);
        r->c = copy(q.sys->c, (size_t)n);
    }
    r->sys.A = r->A.empty() ? nullptr : r->A.data();
    r->sys.B = r->B.empty() ? nullptr : r->B.data();
    r->sys.c = r->c.empty() ? nullptr : r->c.data();
    r->lo = copy(q.grid->lo, n);
    r->hi = copy(q.grid->hi, n);
    r->cells.assign(q.grid->cells, q.grid->cells + n);
    r->grid = *q.grid;
    r->grid.lo = r->lo.data();
    r->grid.hi = r->hi.data();
    r->grid.cells = r->cells.data();
    r->pts = copy(q.inputs->points, (size_t)cnt * m);
    r->inputs = *q.inputs;
    r->inputs.points = r->pts.empty() ? nullptr : r->pts.data();
    r->sigma = copy(q.sigma, n);
    r->cutoff = q.cutoff;
    r->rows = B.rows;
    r->admit_bytes = align_up((int64_t)impact::batch_layout(B).total) +
                     align_up(row_bytes_of(B.rows));
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->stop) {
            delete r;
            return impact::fail(IMPACT_ERR_ARG, "server is shutting down");
        }
        r->ticket = S->next_ticket++;
        S->reqs[r->ticket] = r;
        S->waiting.push_back(r);
        *ticket = r->ticket;
    }
    S->cv_work.notify_one();
    return IMPACT_OK;
}

impact_status impact_server_poll(impact_server *S, int64_t ticket, int wait_ms, int *done,
                                 impact_csr *result, double *latency_ms)
{
    if (!S || !done) return impact::fail(IMPACT_ERR_ARG, "null argument");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || it->second->released)
        return impact::fail(IMPACT_ERR_ARG, "unknown or released ticket");
    Request *r = it->second;
    if (wait_ms != 0) {
        auto fin = [&] { return r->state == Request::DONE || r->state == Request::FAILED; };
        if (wait_ms < 0)
            S->cv_done.wait(lock, fin);
        else
            S->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), fin);
    }
    *done = (r->state == Request::DONE || r->state == Request::FAILED) ? 1 : 0;
    if (!*done) return IMPACT_OK;
    if (latency_ms) *latency_ms = ms_between(r->t_submit, r->t_done);
    if (r->state == Request::FAILED) return impact::fail(r->status, r->error);
    if (result) {
        Group *g = r->group;
        const int64_t rb = g->B.row_begin[r->index];
        memset(result, 0, sizeof(*result));
        result->rows = r->rows;
        result->nnz = r->nnz;
        result->row_ptr = g->row_ptr + rb;
        result->col = g->col;
        result->lo = g->lo;
        result->up = g->up;
        result->sink_lo = g->sink_lo + rb;
        result->sink_up = g->sink_up + rb;
        result->trunc = g->trunc + rb;
        result->row_flags = g->flags + rb;
        result->owned = 0;
    }
    return r->status;
}

impact_status impact_server_timing(impact_server *S, int64_t ticket, double *queue_ms,
                                   double *count_ms, double *emit_wait_ms, double *emit_ms)
{
    if (!S) return impact::fail(IMPACT_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return impact::fail(IMPACT_ERR_ARG, "unknown ticket");
    const Request *r = it->second;
    if (r->state != Request::DONE)
        return impact::fail(IMPACT_ERR_ARG, "the request has not finished successfully");
    if (queue_ms) *queue_ms = ms_between(r->t_submit, r->t_admit);
    if (count_ms) *count_ms = ms_between(r->t_admit, r->t_counted);
    if (emit_wait_ms) *emit_wait_ms = ms_between(r->t_counted, r->t_emit);
    if (emit_ms) *emit_ms = ms_between(r->t_emit, r->t_done);
    return IMPACT_OK;
}

impact_status impact_server_cancel(impact_server *S, int64_t ticket)
{
    if (!S) return impact::fail(IMPACT_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || it->second->released)
        return impact::fail(IMPACT_ERR_ARG, "unknown or released ticket");
    Request *r = it->second;
    if (r->state != Request::WAITING)
        return impact::fail(IMPACT_ERR_ARG, "the request has been admitted or has finished");
    for (auto w = S->waiting.begin(); w != S->waiting.end(); ++w)
        if (*w == r) {
            S->waiting.erase(w);
            break;
        }
    S->fail_request(r, IMPACT_ERR_CANCELLED, "cancelled before admission");
    return IMPACT_OK;
}

impact_status impact_server_release(impact_server *S, int64_t ticket)
{
    if (!S) return impact::fail(IMPACT_ERR_ARG, "null server");
    {
        std::lock_guard<std::mutex> lock(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return impact::fail(IMPACT_ERR_ARG, "unknown ticket");
        Request *r = it->second;
        if (r->state != Request::DONE && r->state != Request::FAILED)
            return impact::fail(IMPACT_ERR_ARG, "request still in flight");
        if (r->group && r->group->live > 0) r->group->live -= 1;
        S->reqs.erase(it);
        delete r;
    }
    S->cv_work.notify_one();
    return IMPACT_OK;
}

impact_status impact_server_stats(impact_server *S, impact_server_stats_t *stats)
{
    if (!S || !stats) return impact::fail(IMPACT_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lock(S->mu);
    stats->completed = S->completed;
    stats->pairs = S->pairs_done;
    stats->groups = S->launched_groups;
    stats->waiting = (int64_t)S->waiting.size();
    stats->bytes_in_use = S->used;
    stats->budget = S->budget;
    return IMPACT_OK;
}

impact_status impact_server_destroy(impact_server *S)
{
    if (!S) return IMPACT_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Group *g : S->groups) {
        cudaStreamSynchronize(g->stream);
        S->free_group(g);
    }
    S->groups.clear();
    for (auto &kv : S->reqs) delete kv.second;
    S->reqs.clear();
    for (cudaStream_t st : S->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    if (S->fast_stream) {
        cudaStreamSynchronize(S->fast_stream);
        cudaStreamDestroy(S->fast_stream);
    }
    delete S;
    return IMPACT_OK;
}

}  // extern "C"
