/*
 * impact.h -- C ABI of the GB300 interval-MDP abstraction builder.
 *
 * What the library computes (paper: Def. 3.1 for the bounds, Alg. 2 for the
 * row-parallel construction, Sec. 4.4 for dropping entries whose upper bound
 * is negligible, Remark 4.1 for the out-of-domain "sink"):
 *
 *   x+ = f(x, u) + w,  w ~ N(0, diag(sigma^2)),  state grid of N_d cells per
 *   dimension on the box [lo, hi], a finite list of input points u_j.
 *
 *   Row r = cell * n_inputs + j (cell id in C order, last dimension fastest).
 *   For each row, [m_lo, m_hi] is the interval image of f(., u_j) over the
 *   closed source cell, and for target cell t with edges [c_d, e_d]:
 *     g_d(m) = Phi((e_d - m)/sigma_d) - Phi((c_d - m)/sigma_d)
 *     up_t   = prod_d g_d(clamp((c_d+e_d)/2, m_lo_d, m_hi_d))   (>= T_max)
 *     lo_t   = prod_d min(g_d(m_lo_d), g_d(m_hi_d))             (<= T_min)
 *   Target t is kept iff up_t >= cutoff (ties kept; cutoff 0 keeps all).
 *   sink_lo / sink_up are the same bounds for landing outside [lo, hi];
 *   trunc is the summed upper bound of the dropped targets, so that for every
 *   row  sum(lo) + sink_lo <= 1 <= sum(up) + sink_up + trunc.
 *
 * Grid convention: edge i of dimension d is lo_d + i*(hi_d - lo_d)/N_d, and
 * edge N_d is hi_d itself. Input points are points (no input cells).
 *
 * Precisions:
 *   IMPACT_FP64_PLAIN  every factor of every pair evaluated in FP64 (erfc per
 *                      pair and dimension); lo/up stored as double.
 *   IMPACT_FP32_SOUND  factors from per-row FP32 tables with outward rounding:
 *                      lo32 <= lo64 and up32 >= up64 for the FP64 values of
 *                      the definition above; lo/up stored as float. The row
 *                      terms (sink, trunc, row checks) are combined in FP64.
 *
 * Threading: every entry point may be called from several host threads; the
 * last-error message is thread-local. Calls on one stream are ordered.
 *
 * Errors: every entry point returns an impact_status; no C++ exception
 * crosses the ABI. On failure impact_last_error() describes the cause.
 */
#ifndef IMPACT_H
#define IMPACT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IMPACT_OK = 0,
    IMPACT_ERR_ARG = 1,       /* invalid argument (sizes, pointers, ranges)          */
    IMPACT_ERR_OOM = 2,       /* a device allocation failed                          */
    IMPACT_ERR_CAPACITY = 3,  /* caller buffers too small; needed nnz written back   */
    IMPACT_ERR_CUDA = 4,      /* a CUDA runtime call or a kernel launch failed       */
    IMPACT_ERR_TIMEOUT = 5,   /* a bounded device wait gave up                       */
    IMPACT_ERR_UNSOUND = 6,   /* a row check proved a row-sum invariant violated     */
    IMPACT_ERR_CANCELLED = 7  /* a served request was cancelled before it ran        */
} impact_status;

typedef enum {
    IMPACT_AFFINE = 0,    /* f(x,u) = A x + B u + c                                   */
    IMPACT_UNICYCLE = 1,  /* n = 3, u = (v, om): x+v cos th, y+v sin th, th+om        */
    IMPACT_IMAGES = 2     /* caller supplies [m_lo, m_hi] per row and dimension       */
} impact_kind;

typedef enum {
    IMPACT_FP64_PLAIN = 0,
    IMPACT_FP32_SOUND = 1
} impact_precision;

/* Row-check bits of impact_csr.row_flags (only set when a violation is proved). */
#define IMPACT_ROW_LO_SUM_ABOVE_ONE  0x1u  /* sum(lo) + sink_lo > 1                  */
#define IMPACT_ROW_UP_SUM_BELOW_ONE  0x2u  /* sum(up) + sink_up + trunc < 1          */

/*
 * The dynamics. Host pointers, read during the call only.
 *   AFFINE:   A (n*n, row-major), B (n*m, row-major; NULL when m == 0),
 *             c (n; NULL means zero).
 *   UNICYCLE: n = 3, m = 2; A, B, c unused.
 *   IMAGES:   dev_images is a DEVICE array of rows*n*2 doubles,
 *             (m_lo, m_hi) per row and dimension, m_lo <= m_hi.
 * params is reserved and must be NULL.
 */
typedef struct {
    int kind;
    int n;
    int m;
    const double *A;
    const double *B;
    const double *c;
    const double *params;
    const double *dev_images;
} impact_system;

/* The state grid (host arrays of length n): dimension d of [lo_d, hi_d] is
 * cut into cells[d] >= 1 equal cells, lo_d < hi_d, product of cells < 2^31. */
typedef struct {
    int n;
    const double *lo;
    const double *hi;
    const int32_t *cells;
} impact_grid;

/* The input points (host, count*m doubles, row-major). count >= 1; with m == 0
 * (no input) pass count = 1 and points = NULL. */
typedef struct {
    int count;
    int m;
    const double *points;
} impact_inputs;

/*
 * The result, a CSR matrix with one row per (cell, input) and int32 target
 * cell ids in ascending order within each row. All arrays are DEVICE memory,
 * except that caller-owned col/lo/up may also be pinned host memory the
 * device can address (cudaHostAlloc / cudaHostRegister): the emit pass then
 * writes the pairs straight into host memory over the host link.
 *   rows            out: number of rows
 *   nnz             in: capacity of col/lo/up when the caller owns them;
 *                   out: number of stored pairs
 *   row_ptr         int64[rows+1]
 *   col             int32[nnz]
 *   lo, up          double[nnz] (FP64_PLAIN) or float[nnz] (FP32_SOUND)
 *   sink_lo/sink_up double[rows]
 *   trunc           double[rows]
 *   row_flags       uint32[rows] (may be NULL: then no row checks are kept)
 *   owned           set to 1 by the library when it allocated the arrays
 *   workspace       optional DEVICE scratch of workspace_bytes bytes (see
 *                   impact_workspace_bytes); NULL lets the library allocate
 *                   and free its scratch stream-ordered inside each call
 * Ownership: if col == NULL on entry to impact_build, the library allocates
 * every array stream-ordered on the given stream and impact_free releases
 * them; otherwise all arrays are the caller's and nnz is their capacity.
 */
typedef struct {
    int64_t rows;
    int64_t nnz;
    int64_t *row_ptr;
    int32_t *col;
    void *lo;
    void *up;
    double *sink_lo;
    double *sink_up;
    double *trunc;
    uint32_t *row_flags;
    int owned;
    void *workspace;
    int64_t workspace_bytes;
} impact_csr;

/*
 * impact_plan -- host-only sizing, no GPU work.
 * Writes the number of rows and an upper bound on nnz (the sum over rows of
 * the product of per-dimension window widths, Sec. 4.4 "low-cost"
 * truncation) and the device bytes that impact_build with library-owned
 * output would need at that bound. Any output pointer may be NULL.
 * Errors: IMPACT_ERR_ARG for invalid sizes or ranges.
 */
impact_status impact_plan(const impact_system *sys, const impact_grid *grid,
                          const impact_inputs *inputs, const double *sigma, double cutoff,
                          impact_precision precision, int64_t *rows, int64_t *nnz_upper_bound,
                          int64_t *bytes_upper_bound);

/*
 * impact_build -- the whole abstraction (Alg. 2) on `stream` (a cudaStream_t;
 * NULL is the legacy default stream): the count pass, the row pointers and
 * the emit pass. With caller-owned col/lo/up (capacity out->nnz) the three
 * run back to back on the device (the emit pass compares the total with the
 * capacity there); with library-owned output the library reads the total
 * after the count to allocate. The batch calls can instead run the FP32-sound
 * build into caller arrays as one pass (impact_tuning.one_pass): each row
 * counts its pairs, finds its offset from the rows before it and writes them.
 * Synchronizes `stream` once at the end (and once after the count when the
 * library allocates) to report nnz and status.
 * Errors: IMPACT_ERR_ARG, IMPACT_ERR_OOM, IMPACT_ERR_CUDA;
 *         IMPACT_ERR_CAPACITY when caller-owned col/lo/up hold fewer than the
 *         needed pairs (out->nnz then holds the needed count, row_ptr and the
 *         row terms are valid; col/lo/up are untouched, or with one_pass hold
 *         the pairs of the rows that fit);
 *         IMPACT_ERR_TIMEOUT (one_pass only) when a row's bounded wait for the
 *         offsets of the rows before it gave up (the output is incomplete; the
 *         device and the library stay usable);
 *         IMPACT_ERR_UNSOUND when row_flags != NULL and some row check failed
 *         (the output is complete; row_flags tells which rows).
 */
impact_status impact_build(const impact_system *sys, const impact_grid *grid,
                           const impact_inputs *inputs, const double *sigma, double cutoff,
                           impact_precision precision, impact_csr *out, void *stream);

/*
 * impact_workspace_bytes -- host-only: the device scratch one build uses (the
 * uploaded descriptor and tables, the scan partial sums and, for
 * IMPACT_FP32_SOUND, one 8-byte offset word per row).
 */
impact_status impact_workspace_bytes(const impact_system *sys, const impact_grid *grid,
                                     const impact_inputs *inputs, const double *sigma,
                                     double cutoff, impact_precision precision, int64_t *bytes);

/*
 * impact_count -- first half of impact_build with caller-owned arrays: writes
 * out->row_ptr (rows+1 entries), sink_lo, sink_up, trunc and row_flags, then
 * synchronizes `stream` and stores the total pair count in out->nnz.
 * col/lo/up are not touched and may be NULL. With a workspace of at least
 * impact_workspace_bytes bytes, the uploaded descriptor and tables stay in it
 * for a following impact_emit with the same arguments and the same workspace.
 * Errors as impact_build (IMPACT_ERR_TIMEOUT included).
 */
impact_status impact_count(const impact_system *sys, const impact_grid *grid,
                           const impact_inputs *inputs, const double *sigma, double cutoff,
                           impact_precision precision, impact_csr *out, void *stream);

/*
 * impact_emit -- second half: given out->row_ptr from impact_count with the
 * same arguments, writes col/lo/up (capacity out->nnz >= row_ptr[rows]).
 * Synchronizes `stream` once at the end to read the status. If
 * out->workspace is the one impact_count filled for these arguments, its
 * uploaded tables are reused; otherwise (NULL, or filled for other arguments:
 * IMPACT_ERR_ARG) pass NULL and the tables are uploaded again. Each row's factor tables are recomputed
 * on the device either way.
 * Errors: IMPACT_ERR_ARG; IMPACT_ERR_CAPACITY when row_ptr[rows] > out->nnz
 *         (nothing written); IMPACT_ERR_CUDA when row_ptr does not match the
 *         arguments (a row whose pair count differs from its row_ptr range,
 *         or a range outside [0, out->nnz)): such a row writes nothing
 *         outside its own range, and the others are complete.
 */
impact_status impact_emit(const impact_system *sys, const impact_grid *grid,
                          const impact_inputs *inputs, const double *sigma, double cutoff,
                          impact_precision precision, impact_csr *out, void *stream);

/* ------------------------------------------------------------------------
 * Batches: several independent builds in one set of launches. Rows of the
 * batch are the builds' rows concatenated in request order; build q owns the
 * global rows [row_offsets[q], row_offsets[q+1]) of one impact_csr and its
 * column ids are target cells of its own grid. Each kernel of the FP32 path
 * runs once for the whole batch (persistent launch: warps take rows of any
 * build from one counter). There is no counterpart in the paper, which builds
 * one abstraction per call (Alg. 2); the per-row arithmetic is the same.
 * ------------------------------------------------------------------------ */

/* One build of a batch: the arguments of impact_build (host pointers). */
typedef struct {
    const impact_system *sys;
    const impact_grid *grid;
    const impact_inputs *inputs;
    const double *sigma;
    double cutoff;
} impact_request;

/*
 * Launch shapes of the FP32-sound walk (impact_batch_tune picks them), and
 * fault-injection knobs for testing the failure paths without a GPU fault.
 * Zero fields take the defaults.
 *   count_warps   warps per block of the count pass and of the one-pass build,
 *                 1..8 (default 4)
 *   emit_warps    warps per block of the emit pass, 1..8 (default 4)
 *   spin_limit    one_pass: sleeps of about 0.1 us that a row's offset
 *                 look-back waits for the rows before it before the call gives
 *                 up with IMPACT_ERR_TIMEOUT (0: 2^24, far beyond any real wait)
 *   one_pass      1: the FP32-sound build into caller arrays (build, graph)
 *                 runs as one walk in which each row finds its offset by a
 *                 look-back over the rows before it; 0 (default): count, scan,
 *                 emit. Same results; the two-pass form measured faster.
 *   stall_row     r + 1: row r never publishes its pair count, so every row
 *                 after it waits until spin_limit runs out (0: off)
 *   fault_row     r + 1: row r's row check sees a lower-bound sum of 2, so it
 *                 is flagged IMPACT_ROW_LO_SUM_ABOVE_ONE and the call returns
 *                 IMPACT_ERR_UNSOUND (needs row_flags; 0: off)
 *   guard_row     r + 1: row r's walk starts with its step guard spent, as if
 *                 an invariant of the walk had broken: the call returns
 *                 IMPACT_ERR_CUDA ("internal") (FP32 walks; 0: off)
 * Shapes change speed only: results are bitwise identical for every shape.
 */
typedef struct {
    int count_warps;
    int emit_warps;
    int spin_limit;
    int one_pass;
    int64_t stall_row;
    int64_t fault_row;
    int64_t guard_row;
} impact_tuning;

/*
 * impact_batch_plan -- host-only sizing of a batch of `count` (1..65536)
 * builds. Writes row_offsets[count+1] (host array, may be NULL), the summed
 * nnz bound, the workspace bytes of the batch and the bytes each count or
 * build call copies host -> device (descriptors and tables). `tuning` may be
 * NULL; so may every output pointer.
 * Errors: IMPACT_ERR_ARG (the message names the failing request).
 */
impact_status impact_batch_plan(const impact_request *reqs, int count, impact_precision precision,
                                const impact_tuning *tuning, int64_t *row_offsets,
                                int64_t *nnz_upper_bound, int64_t *workspace_bytes,
                                int64_t *upload_bytes);

/* impact_count / impact_emit / impact_build for a batch: the same contracts
 * with `out` covering every row of the batch (out->rows = total rows). */
impact_status impact_batch_count(const impact_request *reqs, int count,
                                 impact_precision precision, const impact_tuning *tuning,
                                 impact_csr *out, void *stream);
impact_status impact_batch_emit(const impact_request *reqs, int count,
                                impact_precision precision, const impact_tuning *tuning,
                                impact_csr *out, void *stream);
impact_status impact_batch_build(const impact_request *reqs, int count,
                                 impact_precision precision, const impact_tuning *tuning,
                                 impact_csr *out, void *stream);

/*
 * CUDA graph of a batch's whole pipeline (setup, count, scan and emit, or the
 * one-pass build with impact_tuning.one_pass) into fixed
 * caller-owned arrays: out->col/lo/up with capacity out->nnz and the row
 * arrays, all DEVICE memory that must outlive the graph. The descriptors and
 * tables are uploaded once here (into out->workspace when given, else into
 * scratch the graph owns); each impact_graph_launch replays the build
 * asynchronously on `stream`. After synchronizing that stream,
 * impact_graph_result returns the launch's status and nnz (IMPACT_ERR_CAPACITY
 * when the capacity was short: then col/lo/up are untouched, or with one_pass
 * hold the pairs of the rows that fit). The request
 * arguments are read during impact_graph_create only.
 */
typedef struct impact_graph impact_graph;
impact_status impact_graph_create(const impact_request *reqs, int count,
                                  impact_precision precision, const impact_tuning *tuning,
                                  const impact_csr *out, void *stream, impact_graph **graph);
impact_status impact_graph_launch(impact_graph *graph, void *stream);
impact_status impact_graph_result(impact_graph *graph, int64_t *nnz);
impact_status impact_graph_destroy(impact_graph *graph);

/*
 * impact_batch_tune -- the autotuner: times the count pass over 2, 4, 6 and 8
 * warps per block, then (unless out->col == NULL) the emit pass over the
 * same, each the best of `reps` runs on this batch, and writes the fastest
 * shape to *best and the sum of the two best times to *best_ms (may be NULL). `out` as for impact_batch_emit with the capacity of
 * a previous count. Synchronizes `stream`; its own scratch is allocated and
 * freed stream-ordered. FP32_SOUND only.
 */
impact_status impact_batch_tune(const impact_request *reqs, int count,
                                impact_precision precision, impact_csr *out, int reps,
                                void *stream, impact_tuning *best, double *best_ms);

/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching. Builds are submitted from
 * any host thread and run asynchronously: a scheduler thread admits waiting
 * requests in arrival order while their workspace and row arrays fit the
 * device-memory budget, runs them together as one batch count, emits each
 * counted group as soon as its exact output fits the budget, and overlaps
 * groups on a pool of streams, so requests that arrive while others are on
 * the device join the next group. Small groups (at most 2^18 rows) run on a
 * high-priority stream; larger ones run each pass in launches of 2^18 rows,
 * so the SMs they free between launches go to the small groups first.
 * Results stay on the device until released.
 * Each result is bitwise the same alone and in any mix (same kernels and
 * launch shapes per row). The paper has no counterpart (it builds one
 * abstraction per program run).
 * ------------------------------------------------------------------------ */

typedef struct {
    int64_t memory_budget;       /* device bytes for requests in flight and kept
                                    results (0: 80% of free memory at creation) */
    int max_batch;               /* builds per group (0: 64)                  */
    int64_t max_group_rows;      /* rows per group, past its first build
                                    (0: 2^22)                                 */
    int streams;                 /* streams groups overlap on, 0..8 (0: 2)    */
    impact_precision precision;
} impact_server_config;

typedef struct {
    int64_t completed;           /* requests finished                          */
    int64_t pairs;               /* pairs of the finished requests             */
    int64_t groups;              /* groups launched                            */
    int64_t waiting;             /* requests not yet admitted                  */
    int64_t bytes_in_use;        /* device bytes held now                      */
    int64_t budget;              /* the memory budget in force                 */
} impact_server_stats_t;

typedef struct impact_server impact_server;

/* Starts the scheduler thread on the current device. */
impact_status impact_server_create(const impact_server_config *config, impact_server **server);

/* Checks the request (host only), copies its host arrays and queues it;
 * *ticket identifies it. Errors: IMPACT_ERR_ARG. */
impact_status impact_server_submit(impact_server *server, const impact_request *request,
                                   int64_t *ticket);

/*
 * impact_server_poll -- *done = 1 once the request finished. wait_ms > 0
 * waits up to that many milliseconds for it (< 0: without limit, 0: not at
 * all); *done = 0 when it is still in flight. Once done, *latency_ms (may be
 * NULL) is the time from submission to completion, and *result (may be NULL) describes the device result: rows,
 * nnz, row_ptr (rows+1 entries whose values index col/lo/up directly; the
 * first is not necessarily 0), col/lo/up, sink_lo/sink_up/trunc/row_flags.
 * The arrays belong to the server (owned = 0) and stay valid until
 * impact_server_release. Returns the request's status (IMPACT_ERR_OOM when it
 * can never fit the budget).
 */
impact_status impact_server_poll(impact_server *server, int64_t ticket, int wait_ms, int *done,
                                 impact_csr *result, double *latency_ms);

/*
 * impact_server_timing -- where a finished request's latency went, as seen
 * by the scheduler thread (any pointer may be NULL): queue_ms from submission
 * until its group was launched, count_ms until the group's count pass was
 * seen finished, emit_wait_ms until its emit pass was launched (waiting for
 * output memory or for earlier groups), emit_ms until the emit was seen
 * finished. The four add up to the latency of impact_server_poll.
 * Errors: IMPACT_ERR_ARG for an unknown, released, failed or unfinished
 * request.
 */
impact_status impact_server_timing(impact_server *server, int64_t ticket, double *queue_ms,
                                   double *count_ms, double *emit_wait_ms, double *emit_ms);

/*
 * impact_server_cancel -- withdraws a request that is still waiting for
 * admission: it never reaches the device, and impact_server_poll then reports
 * it done with IMPACT_ERR_CANCELLED (release it as any finished request).
 * A request already admitted runs to completion.
 * Errors: IMPACT_ERR_ARG for an unknown or released ticket, or a request that
 * has been admitted or has finished.
 */
impact_status impact_server_cancel(impact_server *server, int64_t ticket);

/* Frees a finished request's result (its group's memory goes once every
 * request of the group is released). Errors: IMPACT_ERR_ARG when in flight. */
impact_status impact_server_release(impact_server *server, int64_t ticket);

impact_status impact_server_stats(impact_server *server, impact_server_stats_t *stats);

/* Waits for every submitted request, then frees everything. */
impact_status impact_server_destroy(impact_server *server);

/* ------------------------------------------------------------------------
 * Controller synthesis on a built IMDP (paper: Sec. 5 and Alg. 3/4, the LP of
 * Sec. 5 solved by the sorting method of Sec. 6.2); impact_synthesize_ex
 * (below) adds the optimistic policy, a finite horizon, disturbances and
 * region vectors.
 * ------------------------------------------------------------------------ */

typedef enum {
    IMPACT_REACH_AVOID = 0,   /* reach a target cell, never an avoid cell or the sink */
    IMPACT_SAFETY = 1         /* never reach an avoid cell or the sink             */
} impact_spec;

/*
 * impact_synthesize -- interval iteration on the IMDP `imdp` (a result of
 * impact_build for one build: rows = cells * n_inputs, all arrays on the
 * device; FP32 or FP64 values per `precision`). labels: DEVICE uint8[cells],
 * 0 free, 1 target, 2 avoid. The successors of a row are its kept targets
 * [lo, up], the sink [sink_lo, sink_up] and the truncated mass [0, trunc]
 * (valued at its worst end: 0 in a min LP, 1 in a max LP). Phase 1 iterates
 * V0 (from 0) and V1 (from 1) with the best input per cell (reach-avoid:
 * max over inputs of the min LP; safety: min over inputs of the max LP of
 * reaching an avoid cell or the sink) until max |V1 - V0| <= eps, and fixes
 * that input as the policy; phase 2 iterates the opposite LP under the policy.
 * Writes p_min, p_max (DEVICE double[cells]: reach-avoid V0 of phase 1 and V1
 * of phase 2; safety 1 - V1 of phase 1 and 1 - V0 of phase 2) and policy
 * (DEVICE int32[cells], input index; 0 on labelled cells), and the iterations
 * of each phase to iterations[2] (host, may be NULL). A phase that reaches
 * max_iters stops there (its interval is then wider than eps). Synchronizes
 * `stream` once per iteration. Same as impact_synthesize_ex with a
 * pessimistic policy, no horizon, one disturbance point and no region
 * vectors. Errors: IMPACT_ERR_ARG, IMPACT_ERR_OOM, IMPACT_ERR_CUDA.
 */
impact_status impact_synthesize(const impact_csr *imdp, impact_precision precision,
                                int64_t cells, int n_inputs, const uint8_t *labels, int spec,
                                double eps, int max_iters, double *p_min, double *p_max,
                                int32_t *policy, int *iterations, void *stream);

/*
 * impact_build_mc -- impact_build for a noise given by draws instead of the
 * diagonal Gaussian (paper: Sec. 4.1, a full covariance matrix or a custom
 * distribution, integrated by Monte-Carlo sampling). samples: DEVICE
 * double[n][n_samples], dimension-major (draw s of coordinate d at
 * d * n_samples + s); for a covariance C pass L z with C = L L^T and z
 * standard normal. The draws are the caller's: the library draws nothing.
 * With the row's interval image M (as in impact_build) and draw w_s moving it
 * to w_s + M, and cells half-open (edge_i <= y < edge_{i+1}, the last one
 * closed):
 *   up  = fraction of draws whose moved box meets the target cell,
 *   lo  = fraction of draws whose moved box lies in the target cell,
 *   sink_up / sink_lo = fraction that leaves the domain in part / whole,
 * Monte-Carlo estimates of P(w + M meets t), an upper bound of the maximum
 * over the cell, and of P(w + M inside t), a lower bound of the minimum.
 * A target is kept iff up >= cutoff (cutoff 0: every cell); trunc is the
 * dropped up mass. Values are count / n_samples (FP64 exactly as divided;
 * FP32: lo rounded down, up rounded up). sys, grid and inputs as for
 * impact_build (sigma is not used); n_samples in [1, 2^24], every draw
 * finite. The cells within reach of a row's moved boxes must number at most
 * 12288, and at most 64 along one dimension (IMPACT_ERR_ARG otherwise).
 * Ownership, capacity and errors as impact_build; synchronizes `stream`
 * once between the passes.
 */
impact_status impact_build_mc(const impact_system *sys, const impact_grid *grid,
                              const impact_inputs *inputs, const double *samples,
                              int64_t n_samples, double cutoff, impact_precision precision,
                              impact_csr *out, void *stream);

/* ------------------------------------------------------------------------
 * Target and avoid regions (paper: Sec. 3.1 and Alg. 1 for the labels and
 * the vectors R and A, Remark 4.1 for the sink inside A).
 * ------------------------------------------------------------------------ */

#define IMPACT_REGION_MAX_BOXES 16

typedef enum {
    IMPACT_LABEL_FREE = 0,
    IMPACT_LABEL_TARGET = 1,
    IMPACT_LABEL_AVOID = 2
} impact_label;

typedef enum {
    IMPACT_REGION_BOX = 0,        /* one relaxation per region box (tighter)          */
    IMPACT_REGION_CELL_SUM = 1    /* the paper's sums of per-cell bounds (Alg. 1)     */
} impact_region_mode;

/*
 * Regions as axis-aligned boxes in state coordinates: HOST arrays of
 * [count][n] lower and upper corners (lo <= hi, finite). A box labels the
 * cells whose centre (the midpoint of the cell's two edges, edges as in
 * impact_grid) lies in the closed box, so every box stands for a block of
 * whole cells. n_target + n_avoid <= IMPACT_REGION_MAX_BOXES; a box that
 * contains no centre is ignored.
 */
typedef struct {
    int n_target;
    int n_avoid;
    const double *target_lo, *target_hi;   /* host [n_target][n] */
    const double *avoid_lo, *avoid_hi;     /* host [n_avoid][n]  */
} impact_regions;

/*
 * impact_label_cells -- labels of every cell (Alg. 1, labelling step):
 * IMPACT_LABEL_AVOID if the cell's centre lies in an avoid box, else
 * IMPACT_LABEL_TARGET if it lies in a target box, else IMPACT_LABEL_FREE
 * (boxes may overlap; avoid wins). labels: DEVICE uint8[total cells], C
 * order, written stream-ordered on `stream`. Errors: IMPACT_ERR_ARG.
 */
impact_status impact_label_cells(const impact_grid *grid, const impact_regions *regions,
                                 uint8_t *labels, void *stream);

/*
 * impact_region_vectors -- per row r = cell * n_inputs + j the bounds
 * [R_min, R_max] of the probability of landing in the target cells and
 * [A_min, A_max] of landing in an avoid cell or outside the domain.
 *   IMPACT_REGION_CELL_SUM: the paper's vectors, sums of the per-cell
 *     bounds of impact_build (Def. 3.1 relaxation, every cell, no cutoff)
 *     over the labelled cells;
 *   IMPACT_REGION_BOX: each box, as the block of its cells, bounded like one
 *     large target cell (clamped-midpoint maximum, endpoint minimum per
 *     dimension), summed over the boxes. Lies inside the cell sums.
 * Both add the sink bounds of the row to A. The boxes must cover pairwise
 * disjoint sets of cells (IMPACT_ERR_ARG otherwise). IMPACT_FP64_PLAIN
 * evaluates in round-to-nearest FP64; IMPACT_FP32_SOUND uses the outward
 * image and widens every factor by its error bound, with directed rounding,
 * so the vectors enclose the exact ones. r_lo, r_up, a_lo, a_up: DEVICE
 * double[rows], written stream-ordered on `stream`. Errors: IMPACT_ERR_ARG,
 * IMPACT_ERR_OOM, IMPACT_ERR_CUDA.
 */
impact_status impact_region_vectors(const impact_system *sys, const impact_grid *grid,
                                    const impact_inputs *inputs, const double *sigma,
                                    const impact_regions *regions, impact_region_mode mode,
                                    impact_precision precision, double *r_lo, double *r_up,
                                    double *a_lo, double *a_up, void *stream);

/*
 * Options of impact_synthesize_ex.
 *   spec        IMPACT_REACH_AVOID or IMPACT_SAFETY
 *   optimistic  0: the policy is optimised on the lower bound P_min
 *               (pessimistic), 1: on the upper bound P_max (optimistic); the
 *               other bound follows with the policy fixed (Sec. 5)
 *   horizon     0: iterate until max |V1 - V0| <= eps (or max_iters);
 *               K > 0: exactly K steps from V0 = V1 = 0 on the free cells
 *               (Remark 5.1; eps and max_iters are then unused)
 *   n_disturb   disturbance points per input (>= 1): the rows are
 *               r = (cell * n_inputs + j) * n_disturb + k, i.e. the build's
 *               input points are the (input, disturbance) pairs with the
 *               disturbance fastest. The disturbance is the adversary:
 *               it minimises satisfaction, the input maximises it (Sec. 5)
 *   r_lo..a_up  NULL (the labelled cells stay successors and the sink is
 *               one more) or the four DEVICE double[rows] vectors of
 *               impact_region_vectors: the labelled cells then leave every
 *               row and the regions enter as two successors
 */
typedef struct {
    int spec;
    int optimistic;
    int horizon;
    int n_disturb;
    double eps;
    int max_iters;
    const double *r_lo, *r_up, *a_lo, *a_up;
} impact_synth_options;

/*
 * impact_synthesize_ex -- impact_synthesize with the options above. The
 * reported ends: reach-avoid P_min = V0 of the min-LP phase and P_max = V1
 * of the max-LP phase; safety P_min = 1 - V1 of the max-LP phase and
 * P_max = 1 - V0 of the min-LP phase. The policy is phase 1's choice on the
 * vector whose end phase 1 reports (ties: the lowest input index).
 * rows of imdp must equal cells * n_inputs * n_disturb. Synchronizes
 * `stream` once per iteration (once per phase with a horizon). Errors:
 * IMPACT_ERR_ARG, IMPACT_ERR_OOM, IMPACT_ERR_CUDA.
 */
impact_status impact_synthesize_ex(const impact_csr *imdp, impact_precision precision,
                                   int64_t cells, int n_inputs, const uint8_t *labels,
                                   const impact_synth_options *options, double *p_min,
                                   double *p_max, int32_t *policy, int *iterations,
                                   void *stream);

/* Release library-owned arrays of a result (no-op for caller-owned ones). */
impact_status impact_free(impact_csr *out);

/* Message of the last failing call on this host thread ("" if none). */
const char *impact_last_error(void);

/* Library ABI version (major*100 + minor). */
int impact_version(void);

/* ------------------------------------------------------------------------
 * Failure injection for tests of the out-of-memory paths: the failure is
 * made on the host, so no GPU is exhausted or faulted. The paper has no
 * counterpart (its tool has no failure handling to test).
 * ------------------------------------------------------------------------ */

/*
 * impact_debug_fail_alloc -- the n-th device or pinned-host allocation the
 * library makes from now on (counting across all threads) fails as if the
 * device were out of memory, without allocating; the entry point that made it
 * returns IMPACT_ERR_OOM after releasing everything it took. n = 0 turns the
 * injection off; after the failure it is off again.
 * Errors: IMPACT_ERR_ARG when n < 0.
 */
impact_status impact_debug_fail_alloc(int64_t n);

/*
 * impact_debug_live_bytes -- bytes of device and of pinned host memory the
 * library currently holds through its own allocations (workspaces, scratch,
 * library-owned results, server groups; not the caller's arrays, and not the
 * fixed scratch of impact_scan_rows_static). Either pointer may be NULL.
 */
impact_status impact_debug_live_bytes(int64_t *device_bytes, int64_t *host_bytes);

/* Largest `rows` that impact_scan_rows_static accepts. */
#define IMPACT_SCAN_STATIC_MAX_ROWS (1LL << 27)

/*
 * impact_scan_rows_static -- the row-pointer scan (the one the FP64-plain count
 * pass and impact_build_mc run), for callers that must not allocate device
 * memory. The paper has no counterpart: this is
 * a deployment convenience, not part of the method.
 *
 * Who needs it: code that cannot call cudaMalloc (or cudaMallocAsync) at the
 * point where it builds row pointers -- for example a host program whose
 * device memory is all reserved up front by its own arena allocator and may
 * not grow afterwards (a real-time controller that forbids allocation after
 * start-up), or a plugin whose host framework owns every device allocation.
 * Such a caller can count pairs into its own buffer and turn the counts into
 * CSR row pointers here without the library allocating anything.
 *
 * Arguments: row_ptr is a DEVICE array of rows+1 int64. On entry
 * row_ptr[0..rows) holds the per-row pair counts; on return (stream-ordered
 * on `stream`, a cudaStream_t or NULL) row_ptr[r] is the exclusive prefix sum
 * and row_ptr[rows] the total. Nothing is allocated or freed, no library
 * routine that allocates is called, and the call does not synchronize.
 *
 * Scratch: a fixed device array of IMPACT_SCAN_STATIC_MAX_ROWS/4096 + 1 int64
 * (256 KiB), declared at file scope in the library, so every GPU that loads
 * the library holds it until the process exits. The first call on a device
 * looks up that array's device address (with the device current); make that
 * first call before any stream capture. All calls share the array and every
 * call overwrites the part it uses before reading it: calls whose work
 * overlaps on the GPU (different streams, or different host threads on one
 * device) race and must be serialized by the caller.
 *
 * Errors: IMPACT_ERR_ARG when rows < 1, rows > IMPACT_SCAN_STATIC_MAX_ROWS or
 * row_ptr is not device (or managed) memory (checked with
 * cudaPointerGetAttributes, which allocates nothing); IMPACT_ERR_CUDA when the
 * address lookup or a launch fails.
 */
impact_status impact_scan_rows_static(int64_t *row_ptr, int64_t rows, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* IMPACT_H */
