// pipeline.h -- a batch of builds, its device workspace and the count /
// emit pipeline (api.cu), shared with the serving runtime (server.cu);
// internal.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/impact.h"
#include "impact_desc.h"
#include "kernels.h"
#include "plan.h"

namespace impact {

struct Batch {
    std::vector<Plan> plans;
    std::vector<const double *> images;   // per build: device images (IMAGES kind)
    std::vector<int64_t> row_begin;       // [count + 1] first global row of each build
    std::vector<int64_t> unit_begin;      // [count + 1] first setup unit (32/n rows)
    int64_t rows = 0, units = 0, nnz_bound = 0;
    int prec = 0;
    int rec_max = 0;                      // FP32 walk: largest record of the batch
    int work_max[2] = {0, 0};             // FP32 walk: largest work space, emit / count
    Tuning tune;
    uint64_t hash = 0;
    int count() const { return (int)plans.size(); }
};

impact_status make_batch(const impact_request *reqs, int count, impact_precision precision,
                         const impact_tuning *tuning, Batch &B);

// Offsets (bytes, 256-aligned) of everything in the device workspace.
struct BatchLayout {
    size_t index = 0, row_begin = 0, unit_begin = 0, descs = 0, recs = 0;
    std::vector<size_t> tables;            // per build: its descriptor and tables
    std::vector<impact::TableLayout> tl;
    size_t upload_end = 0;                 // [0, upload_end) is copied from the host
    size_t status = 0, counter = 0, scan = 0;
    size_t lb = 0;                         // FP32: one look-back word per row
    std::vector<size_t> rec;               // per build: FP32 per-row records
    size_t total = 0;
};

BatchLayout batch_layout(const Batch &B);

// The device workspace of one call.
struct Work {
    unsigned char *base = nullptr;
    BatchLayout L;
    bool owned = false;
    const BatchIndex *index() const { return (const BatchIndex *)(base + L.index); }
    uint32_t *status() const { return (uint32_t *)(base + L.status); }
    unsigned long long *counter() const { return (unsigned long long *)(base + L.counter); }
    int64_t *scan() const { return (int64_t *)(base + L.scan); }
    unsigned long long *lb() const { return (unsigned long long *)(base + L.lb); }
    const ImpactDesc *desc(int q) const
    {
        return (const ImpactDesc *)(base + L.tables[q] + L.tl[q].desc);
    }
};

// Copies the batch index, the descriptors and the tables into W (stream-ordered).
impact_status upload(const Batch &B, Work &W, cudaStream_t st);
// The passes below launch the FP32 walk over all rows at once, or in chunks
// of `chunk_rows` rows one after another on `st` (so that work on other
// streams can take SMs between chunks); the FP64 kernels ignore chunk_rows.
// count pass into out's row arrays (row pointers included).
impact_status run_count(const Batch &B, const Work &W, const impact_csr *out, cudaStream_t st,
                        int64_t chunk_rows = 0);
// emit pass into out's pair arrays at the row pointers of a count pass
// (`records_ready`: W holds the FP32 row records of that count pass).
impact_status run_emit(const Batch &B, const Work &W, const impact_csr *out, int64_t capacity,
                       bool records_ready, cudaStream_t st, int64_t chunk_rows = 0);
// FP32: count and emit in one pass (capacity known); FP64: count, scan, emit.
impact_status run_fused(const Batch &B, const Work &W, const impact_csr *out, int64_t capacity,
                        cudaStream_t st, int64_t chunk_rows = 0);
// Maps the device status word of a finished pipeline to a status code.
impact_status status_result(uint32_t status);
void configure_pool_once();

}  // namespace impact
