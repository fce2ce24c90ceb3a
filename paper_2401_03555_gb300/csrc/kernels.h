// kernels.h -- launchers the host planner (api.cu) uses; internal interface.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "impact_desc.h"

#define IMPACT_TABLE_MAX 512              // factor entries staged per row (all dims), FP64
#define IMPACT_WINDOW_MAX 64              // FP32 path: window cells per (row, dim)
#define IMPACT_TSUM_MAX 256               // FP32 path: factor entries per row record
#define IMPACT_TREE_SEG 512               // FP32 path: pairs staged per leaf batch
#define IMPACT_TREE_HDR 256               // FP32 path: per-row scalars per warp (bytes)
#define IMPACT_TREE_SMEM_COUNT 6144       // FP32 path: per-warp shared memory aimed for, count (default)
#define IMPACT_TREE_SMEM_EMIT 8192        // FP32 path: per-warp shared memory aimed for, emit (default)
#define IMPACT_TREE_WARPS 4               // FP32 path: warps per block of the walk (default)
#define IMPACT_TREE_WARPS_MAX 8
#define IMPACT_STATUS_TABLE_OVERFLOW 0x1u // some row's windows exceeded IMPACT_TABLE_MAX
#define IMPACT_STATUS_UNSOUND 0x2u        // some row check proved a violation
#define IMPACT_STATUS_CAPACITY 0x4u       // emit skipped: output capacity too small
#define IMPACT_STATUS_EMIT_MISMATCH 0x8u  // emit found a different pair count than count

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

// FP32-sound table path (tree_fp32.cu), every launch over a whole batch.
int64_t record_stride(int n, int tsum_cap);
int tree_smem_bytes(int tsum_cap, int pool_cap, bool emit);
// `units`: warp units of the batch (BatchIndex::units); the row outputs may
// be null (records rebuilt for an emit pass).
cudaError_t launch_setup_fp32(const BatchIndex *d_index, int64_t units, uint32_t *status,
                              double *sink_lo, double *sink_up, double *trunc, cudaStream_t stream);
// `warp_smem`: shared-memory bytes of one warp (the largest of the batch);
// `warps`: warps per block (1..8).
cudaError_t launch_tree_fp32(const BatchIndex *d_index, int64_t rows, int warp_smem, int warps,
                             bool emit, const RowOutputs &o, cudaStream_t stream);
cudaError_t launch_scan(int64_t *row_ptr, int64_t n, int64_t *scratch, cudaStream_t stream);

}  // namespace impact
