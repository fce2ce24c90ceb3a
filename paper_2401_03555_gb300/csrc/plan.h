// plan.h -- host planner interface (plan.cu) shared with the entry points
// (api.cu); internal.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/impact.h"
#include "impact_desc.h"
#include "kernels.h"

namespace impact {

// Sets the thread's last-error message and returns `s` (api.cu).
impact_status fail(impact_status s, const std::string &msg);

// Launch shapes of the FP32 walk (impact_tuning with the defaults filled in)
// and its fault-injection knobs.
struct Tuning {
    int count_warps = IMPACT_TREE_WARPS;
    int emit_warps = IMPACT_TREE_WARPS;
    bool one_pass = false;   // FP32 build into caller arrays: one walk with look-back
    WalkFaults faults;
};

struct Plan {
    ImpactDesc desc;
    std::vector<double> edges, term_rn, term_dn, term_up, off_rn, off_dn, off_up, uni_rn,
        uni_sd, inputs;
    // FP32-sound table path
    std::vector<float2> ea, ta_lo, ta_hi, oa, ua, oma;
    std::vector<float> mu_lo, mu_hi, mo, um, omm;
    int64_t rows = 0;
    int64_t nnz_bound = 0;
    int table_need = 0;   // upper bound of the staged entries per row (-1: unknown)
    uint64_t hash = 0;    // identifies the arguments (workspace reuse check)
};

// Offsets (in bytes, 256-aligned) of the descriptor and tables of one build.
struct TableLayout {
    size_t desc, edges, term_rn, term_dn, term_up, off_rn, off_dn, off_up, uni_rn, uni_sd,
        inputs, ea, ta_lo, ta_hi, oa, ua, oma, mu_lo, mu_hi, mo, um, omm, total;
};

size_t align256(size_t x);
TableLayout table_layout(const Plan &p);

impact_status make_plan(const impact_system *sys, const impact_grid *grid,
                        const impact_inputs *inputs, const double *sigma, double cutoff,
                        impact_precision precision, Plan &P);

// Writes the descriptor and tables of P into `host` (table_layout(P).total
// bytes) with every pointer set for the copy that will sit at `dev_base`.
void pack_tables(const Plan &P, unsigned char *host, unsigned char *dev_base,
                 const double *dev_images);

}  // namespace impact
