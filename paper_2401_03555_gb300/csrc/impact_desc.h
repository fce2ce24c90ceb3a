// impact_desc.h -- the per-build descriptor the host planner uploads once and
// every kernel of the build reads. Plain data, shared by host and device code.
#pragma once
#include <stdint.h>

#define IMPACT_MAX_DIM 8
#define IMPACT_MAX_M 8

// Per-dimension constants (computed on the host in FP64).
struct ImpactDim {
    double lo, hi;        // domain [lo, hi]
    double h;             // (hi - lo) / N, the nominal cell width
    double inv_h;         // RN(1 / h)
    double sigma;         // noise standard deviation
    double inv_s;         // RN(1 / (sigma * sqrt 2))
    double kappa;         // RN(h * inv_s): cell width in erf-argument units
    double delta;         // window margin sigma * z_c (+inf when cutoff == 0)
    float kappa_hi, kappa_lo;   // kappa as an FP32 pair (hi + lo)
    float edge_err;       // bound on |(E_i - E_a)*inv_s - (i-a)*kappa| (erf units)
    float plateau_hi;     // FP32 upper bound of erf(h_max * inv_s / 2), the max factor
    float qmin_lo;        // FP32 lower bound of the least out-of-domain mass 2*T(halfwidth)
    int N;                // number of cells
    int stride;           // C-order column stride
    int edge_off;         // offset of this dim's N+1 FP64 edges in the edge table
    int wcap;             // largest window (cells) of a row in this dim
    int rec_off;          // FP32 path: first entry of this dim's table in a row record
    float delta_cells;    // delta / h
    uint32_t div_m;       // fast division by N: q = (umulhi(x, div_m) + x) >> div_s
    int div_s;
};

// Kinds (match impact_kind) and precisions (match impact_precision).
enum { KIND_AFFINE = 0, KIND_UNICYCLE = 1, KIND_IMAGES = 2 };
enum { PREC_FP64_PLAIN = 0, PREC_FP32_SOUND = 1 };

struct ImpactDesc {
    int n;                // state dimension
    int m;                // input dimension
    int kind;
    int prec;
    int n_inputs;
    int n_in_split_min;   // inner enumeration block: grow inner dims until >= this
    int64_t rows;         // rows = cells * n_inputs
    int64_t cells;        // total cells
    double cutoff;        // keep iff up >= cutoff
    float cutoff32;       // smallest float >= cutoff (FP32 keep test)
    int table_max;        // per-row window entries the kernel can stage
    ImpactDim dim[IMPACT_MAX_DIM];

    // Device pointers into the same allocation (set by the planner).
    const double *edges;      // per dim N_d + 1 edges (oracle definition)
    // AFFINE: per (d, k, i) image terms of A_dk * x_k over cell i of dim k.
    //   term_rn[d][k][i]  = min/max in round-to-nearest, lo then hi (2 doubles)
    //   term_dn[d][k][i]  = lower bound (directed), term_up = upper bound
    const double *term_rn;    // [n][n][Nmax][2]
    const double *term_dn;    // [n][n][Nmax]
    const double *term_up;    // [n][n][Nmax]
    // AFFINE: per input j, offset c_d + sum_k B_dk u_k: RN, and a bracket.
    const double *off_rn;     // [n_inputs][n]
    const double *off_dn;     // [n_inputs][n]
    const double *off_up;     // [n_inputs][n]
    // UNICYCLE: per (heading cell i, input j): range of v cos th and v sin th
    //   over the heading cell, RN [4] = (cos lo, cos hi, sin lo, sin hi) and a
    //   bracketing version.
    const double *uni_rn;     // [N_th][n_inputs][4]
    const double *uni_sd;     // [N_th][n_inputs][4] outward
    const double *inputs;     // [n_inputs][m]
    const double *images;     // IMAGES: [rows][n][2], caller's device array
    int n_max;                // max N_d
    int pad1;

    // FP32-sound table path. Values "in erf units" of dimension d are
    // multiplied by 1/(sigma_d sqrt2) on the host in FP64 and stored as FP32
    // pairs (hi + lo); values "in cells" are divided by h_d (FP32, used only
    // to place the windows, with slack).
    uint32_t inp_div_m;       // fast division by n_inputs
    int inp_div_s;
    int tsum_cap;             // window targets of a row, all dims (at most)
    int rec_stride;           // bytes per row record in the workspace
    int leaf_cap;             // leaf-table entries a warp of the walk stages
    int walk_core;            // shared-memory bytes of one warp of the walk
    const float2 *ea;         // per dim: N+1 edges in erf units, offset edge_off
    const float2 *ta_lo;      // AFFINE [n][n][Nmax]: min term A_dk x_k in erf units of d
    const float2 *ta_hi;      //                      max term
    const float *mu_lo;       // AFFINE [n][n][Nmax]: min term divided by h_d
    const float *mu_hi;       //                      max term divided by h_d
    const float2 *oa;         // AFFINE [n_inputs][n]: offset c + B u in erf units
    const float *mo;          // AFFINE [n_inputs][n]: (offset - lo_d) / h_d
    const float2 *ua;         // UNICYCLE [N_th][n_inputs][4]: v cos / v sin ranges, erf units
    const float *um;          // UNICYCLE [N_th][n_inputs][4]: the same in cells
    const float2 *oma;        // UNICYCLE [n_inputs]: om in erf units of the heading
    const float *omm;         // UNICYCLE [n_inputs]: om in heading cells
};

// Several builds handled by one launch of each FP32 kernel: problem q owns the
// global rows [row_begin[q], row_begin[q+1]) of the concatenated output and
// the setup units [unit_begin[q], unit_begin[q+1]) (a unit is the 32/n rows
// one warp prepares); a single build is a batch of one.
struct BatchIndex {
    int count;                          // problems
    int64_t rows;                       // total rows
    int64_t units;                      // setup work units: 32/n rows of one problem
    const int64_t *row_begin;           // [count + 1]
    const int64_t *unit_begin;          // [count + 1]
    const ImpactDesc *const *desc;      // [count] device descriptors
    unsigned char *const *rec;          // [count] FP32 per-row records
    unsigned long long *next_row;       // [2] row counters of the count / emit walk
};
