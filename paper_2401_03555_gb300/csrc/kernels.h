// kernels.h -- launchers the host planner (api.cu) uses; internal interface.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "impact_desc.h"

#define IMPACT_TABLE_MAX 512              // FP64: window factors a warp stages (wider: re-evaluated)
#define IMPACT_WALK_CAP 64                // FP32 walk: nodes per level list (one chunk)
#define IMPACT_LEAF_STAGE 256             // FP32 walk: leaf-table entries a warp stages
#define IMPACT_WALK_SMEM_MAX (200 * 1024) // FP32 walk: shared memory of one warp at most
#define IMPACT_TREE_WARPS 4               // FP32 walk: warps per block (default)
#define IMPACT_TREE_WARPS_MAX 8
#define IMPACT_STATUS_TABLE_OVERFLOW 0x1u // a row's window exceeded the planner's bound
#define IMPACT_STATUS_UNSOUND 0x2u        // some row check proved a violation
#define IMPACT_STATUS_CAPACITY 0x4u       // emit skipped: output capacity too small
#define IMPACT_STATUS_EMIT_MISMATCH 0x8u  // emit found a different pair count than count
#define IMPACT_STATUS_TIMEOUT 0x20u       // a bounded look-back wait gave up
#define IMPACT_STATUS_INTERNAL 0x40u      // the walk's step guard ran out (broken invariant)

namespace impact {

struct RowOutputs {
    int64_t *row_ptr;   // count pass: per-row counts out; emit pass: row offsets in
    int32_t *col;
    void *lo;
    void *up;
    double *sink_lo;
    double *sink_up;
    double *trunc;
    uint32_t *flags;
    uint32_t *status;
    int64_t capacity;   // emit: pairs the col/lo/up arrays hold (< 0: unchecked)
    int64_t total_at;   // emit: index of the total count in row_ptr (rows)
};

cudaError_t launch_rows(const ImpactDesc *d_desc, int prec, bool emit, int64_t row_begin,
                        int64_t row_end, const RowOutputs &o, cudaStream_t stream);

int64_t scan_scratch_elems(int64_t n);

// Sets the message impact_last_error() returns on this host thread.
void set_last_error(const std::string &msg);

// Region boxes as blocks of whole cells (impact_regions after the host has
// found the cells whose centre lies in each box): targets first.
#define IMPACT_REGION_BOXES 16
struct RegionBoxes {
    int count;                                      // boxes in use
    int n_target;                                   // boxes [0, n_target) are targets
    int n;                                          // dimensions
    int cells[IMPACT_MAX_DIM];                      // grid cells per dimension
    int first[IMPACT_REGION_BOXES][IMPACT_MAX_DIM];   // first cell index per dimension
    int last[IMPACT_REGION_BOXES][IMPACT_MAX_DIM];    // last cell index per dimension
};

// Sampled noise (Monte-Carlo integration): per-call tables (the draws'
// order-preserving integer keys, their per-dimension range, the values u / S,
// a flag for non-finite draws), then the count and emit passes over a
// per-row histogram of the cells the moved image box meets / lies in.
// Draws: dimension-major [n][S].
#define IMPACT_MC_HIST_MAX 12288          // window cells one block's histogram holds
#define IMPACT_MC_EDGES_MAX 64            // window cells per dimension
#define IMPACT_STATUS_MC_WINDOW 0x10u     // some row's window exceeded the limits above
cudaError_t launch_mc_prep(const double *samples, int n, int64_t S, long long *keys,
                           double *val, float *val_dn, float *val_up, unsigned *bad,
                           double *range, cudaStream_t stream);
cudaError_t launch_mc_rows(const ImpactDesc *d_desc, bool emit, int64_t rows,
                           const long long *keys, int64_t S, const double *range,
                           const double *val, const float *val_dn, const float *val_up,
                           unsigned kmin, const RowOutputs &o, cudaStream_t stream);

// Labels of every cell (0 free, 1 target, 2 avoid; avoid wins).
cudaError_t launch_labels(const RegionBoxes &boxes, int64_t total_cells, uint8_t *labels,
                          cudaStream_t stream);
// Region vectors of rows [0, rows) of the build described by d_desc (FP64
// tables): cell_sum selects the paper's sums of per-cell bounds, else one
// relaxation per box; sound selects the enclosing evaluation.
cudaError_t launch_regions(const ImpactDesc *d_desc, int64_t rows, const RegionBoxes &boxes,
                           bool cell_sum, bool sound, double *r_lo, double *r_up, double *a_lo,
                           double *a_up, cudaStream_t stream);

// FP32-sound path (walk_fp32.cu). The setup kernel writes one record per
// row (record_stride bytes: per-dimension entries, then the window tables)
// and, when the row arrays are given, the sink bounds and the mass outside
// the window box; the walk kernels read the records. A walk launch covers
// the global rows [row_begin, row_end) of a batch (the pass's row counter
// zeroed before each launch; launches of one pass in row order on one
// stream). A warp's shared memory holds two record buffers of `rec_max`
// bytes (the largest record_stride of the batch: the row being walked and the
// next one, prefetched) and work space: `work_max` = the largest
// walk_work_bytes of the batch for the emit pass [0] and the passes that
// count [1]; `lb`: one
// 8-byte look-back word per row, zeroed before the first launch of a FUSED
// pass. COUNT writes per-row counts (a scan makes them row pointers), FUSED
// the row pointers themselves.
enum { WALK_COUNT = 0, WALK_EMIT = 1, WALK_FUSED = 2 };
struct WalkFaults {
    int spin_limit = 0;        // look-back sleeps before giving up (0: the default)
    int64_t stall_row = -1;    // this row never publishes its count (-1: none)
    int64_t fault_row = -1;    // this row's checks see an impossible sum (-1: none)
    int64_t guard_row = -1;    // this row's walk starts with its step guard spent (-1: none)
};
int64_t record_stride(int n, int tsum_cap);
int walk_core_bytes(int n, int tsum_cap, int leaf_cap);   // both buffers and the work space
int walk_work_bytes(int n, int leaf_cap, bool count);
cudaError_t launch_setup_fp32(const BatchIndex *d_index, int64_t units, uint32_t *status,
                              double *sink_lo, double *sink_up, double *trunc, cudaStream_t stream);
cudaError_t launch_walk_fp32(const BatchIndex *d_index, int64_t row_begin, int64_t row_end,
                             int rec_max, const int work_max[2], int warps, int mode,
                             const RowOutputs &o,
                             unsigned long long *lb, const WalkFaults &f, cudaStream_t stream);
cudaError_t launch_scan(int64_t *row_ptr, int64_t n, int64_t *scratch, cudaStream_t stream);

}  // namespace impact
