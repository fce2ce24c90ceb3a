/*
 * impact_oracle.c -- plain, slow FP64 CPU oracle for the interval-MDP (IMDP)
 * abstraction of x+ = f(x,u) + w with diagonal Gaussian w.
 *
 * TEST INFRASTRUCTURE. This file is the reference that the CUDA path is checked
 * against; it is not part of the product. Only tests/, __graft_entry__.smoke()
 * and bench.py's cpu_baseline leg may load it. It shares no code, header,
 * table or constant with the CUDA library, and never calls it.
 *
 * What it computes (paper: Def. 3.1, Alg. 1, Sec. 4.4 and Remark 4.1), with
 * the sound box relaxation of the per-cell min/max that the hot path uses:
 *
 *   for every row r = cell * n_inputs + j (cell id in C order, last dim fastest)
 *     [m_lo, m_hi]  = coordinate-wise range of f(., u_j) over the closed cell
 *     for EVERY target cell t (dense, no windows, no tables):
 *       g_d(m)   = Phi((e_d - m)/sigma_d) - Phi((c_d - m)/sigma_d)
 *       up_t     = prod_d g_d(clamp((c_d + e_d)/2, m_lo_d, m_hi_d))
 *       lo_t     = prod_d min(g_d(m_lo_d), g_d(m_hi_d))
 *       keep t   iff up_t >= cutoff          (the "low-cost" rule, Sec. 4.4)
 *     trunc      = sum of up_t over the dropped targets (Neumaier summation)
 *     sink_lo    = 1 - prod_d G_d(clamp(mid of domain_d, m_lo_d, m_hi_d))
 *     sink_up    = 1 - prod_d min(G_d(m_lo_d), G_d(m_hi_d))
 *                  with G_d the same factor over the domain interval
 *                  [lo_d, hi_d] (Remark 4.1: leaving the domain is the
 *                  complement of landing inside it).
 *
 * Grid: dimension d of the domain [lo_d, hi_d] is cut into N_d equal cells;
 * edge i is lo_d + i*h_d with h_d = (hi_d - lo_d)/N_d, except that edge N_d is
 * hi_d itself. Cell i is [edge i, edge i+1]. Inputs are points.
 *
 * Build with -ffp-contract=off so every expression is evaluated as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_DIM 8

enum { ORACLE_AFFINE = 0, ORACLE_UNICYCLE = 1, ORACLE_IMAGES = 2 };

typedef struct {
    int kind;               /* ORACLE_AFFINE, ORACLE_UNICYCLE or ORACLE_IMAGES */
    int n;                  /* state dimension, 1..8 */
    int m;                  /* input dimension */
    const double *A;        /* affine: n*n, row-major */
    const double *B;        /* affine: n*m, row-major (may be NULL when m == 0) */
    const double *c;        /* affine: n (may be NULL: zero) */
    const double *images;   /* images: rows*n*2, (m_lo, m_hi) per row and dim */
    const double *lo;       /* n: domain lower corner */
    const double *hi;       /* n: domain upper corner */
    const int32_t *cells;   /* n: cells per dimension */
    int n_inputs;           /* number of input points (>= 1) */
    const double *inputs;   /* n_inputs*m, row-major */
    const double *sigma;    /* n: noise standard deviations */
    double cutoff;          /* keep a target iff its upper bound >= cutoff */
} oracle_problem;

/*
 * g(c, e; m) = Phi((e-m)/s) - Phi((c-m)/s): the probability that m + w lands
 * in [c, e] for w ~ N(0, s^2) (the Gaussian kernel T of Def. 2.2 restricted to
 * one dimension). Evaluated in the form that avoids subtracting two numbers
 * close to 1: both tails on the same side use erfc of non-negative arguments.
 */
double oracle_phi_diff(double c, double e, double m, double s)
{
    double a = (c - m) / s;
    double b = (e - m) / s;
    if (a >= 0.0)
        return 0.5 * (erfc(a * M_SQRT1_2) - erfc(b * M_SQRT1_2));
    if (b <= 0.0)
        return 0.5 * (erfc(-b * M_SQRT1_2) - erfc(-a * M_SQRT1_2));
    return 1.0 - 0.5 * erfc(-a * M_SQRT1_2) - 0.5 * erfc(b * M_SQRT1_2);
}

/* Edge i of dimension d (0 <= i <= N_d). */
double oracle_edge(const oracle_problem *p, int d, int i)
{
    int N = p->cells[d];
    if (i >= N) return p->hi[d];
    double h = (p->hi[d] - p->lo[d]) / (double)N;
    return p->lo[d] + (double)i * h;
}

static int64_t total_cells(const oracle_problem *p)
{
    int64_t t = 1;
    for (int d = 0; d < p->n; ++d) t *= p->cells[d];
    return t;
}

/* Cell index of dimension d for a C-order cell id. */
static int cell_digit(const oracle_problem *p, int64_t cell, int d)
{
    int64_t stride = 1;
    for (int k = d + 1; k < p->n; ++k) stride *= p->cells[k];
    return (int)((cell / stride) % p->cells[d]);
}

/* Range of cos over [a, b]: the endpoint values, widened to +1 where an even
 * multiple of pi lies inside and to -1 where an odd multiple does. */
static void cos_range(double a, double b, double *lo, double *hi)
{
    double ca = cos(a), cb = cos(b);
    *lo = ca < cb ? ca : cb;
    *hi = ca < cb ? cb : ca;
    for (long k = (long)ceil(a / M_PI); (double)k * M_PI <= b; ++k) {
        if (k % 2 == 0) *hi = 1.0; else *lo = -1.0;
    }
}

/* Range of sin over [a, b]: extrema at pi/2 + k*pi (+1 for even k, -1 for odd). */
static void sin_range(double a, double b, double *lo, double *hi)
{
    double sa = sin(a), sb = sin(b);
    *lo = sa < sb ? sa : sb;
    *hi = sa < sb ? sb : sa;
    for (long k = (long)ceil((a - M_PI_2) / M_PI); M_PI_2 + (double)k * M_PI <= b; ++k) {
        if (k % 2 == 0) *hi = 1.0; else *lo = -1.0;
    }
}

/*
 * Interval image [m_lo, m_hi] of f(., u_j) over the source cell of `row`: the
 * exact coordinate-wise range (the box that the per-cell min/max of Def. 3.1
 * is relaxed over).
 *   affine:   f(x,u) = A x + B u + c; each term A_dk x_k ranges over
 *             [min, max] of its two endpoint products.
 *   unicycle: x+ = x + v cos(th), y+ = y + v sin(th), th+ = th + om, inputs
 *             (v, om); th is not wrapped.
 *   images:   read from the caller's array.
 */
void oracle_image(const oracle_problem *p, int64_t row, double *m_lo, double *m_hi)
{
    int n = p->n;
    int64_t cell = row / p->n_inputs;
    int j = (int)(row % p->n_inputs);
    const double *u = p->inputs + (int64_t)j * p->m;
    double xlo[ORACLE_MAX_DIM], xhi[ORACLE_MAX_DIM];
    for (int d = 0; d < n; ++d) {
        int i = cell_digit(p, cell, d);
        xlo[d] = oracle_edge(p, d, i);
        xhi[d] = oracle_edge(p, d, i + 1);
    }
    if (p->kind == ORACLE_AFFINE) {
        for (int d = 0; d < n; ++d) {
            double off = p->c ? p->c[d] : 0.0;
            for (int k = 0; k < p->m; ++k) off += p->B[d * p->m + k] * u[k];
            double s_lo = 0.0, s_hi = 0.0;
            for (int k = 0; k < n; ++k) {
                double a = p->A[d * n + k] * xlo[k];
                double b = p->A[d * n + k] * xhi[k];
                s_lo += a < b ? a : b;
                s_hi += a < b ? b : a;
            }
            m_lo[d] = s_lo + off;
            m_hi[d] = s_hi + off;
        }
    } else if (p->kind == ORACLE_UNICYCLE) {
        double v = u[0], om = u[1];
        double cl, ch, sl, sh;
        cos_range(xlo[2], xhi[2], &cl, &ch);
        sin_range(xlo[2], xhi[2], &sl, &sh);
        double vc1 = v * cl, vc2 = v * ch, vs1 = v * sl, vs2 = v * sh;
        m_lo[0] = xlo[0] + (vc1 < vc2 ? vc1 : vc2);
        m_hi[0] = xhi[0] + (vc1 < vc2 ? vc2 : vc1);
        m_lo[1] = xlo[1] + (vs1 < vs2 ? vs1 : vs2);
        m_hi[1] = xhi[1] + (vs1 < vs2 ? vs2 : vs1);
        m_lo[2] = xlo[2] + om;
        m_hi[2] = xhi[2] + om;
    } else {
        for (int d = 0; d < n; ++d) {
            m_lo[d] = p->images[(row * n + d) * 2 + 0];
            m_hi[d] = p->images[(row * n + d) * 2 + 1];
        }
    }
}

static double clamp(double x, double lo, double hi)
{
    if (x < lo) return lo;
    if (x > hi) return hi;
    return x;
}

/*
 * Dense bounds of one row over every target cell (Def. 3.1 with the box
 * relaxation): up[t], lo[t] for t = 0 .. total_cells-1, plus the sink bounds
 * of Remark 4.1.
 */
void oracle_row_dense(const oracle_problem *p, int64_t row, double *up, double *lo,
                      double *sink_lo, double *sink_up)
{
    int n = p->n;
    double m_lo[ORACLE_MAX_DIM], m_hi[ORACLE_MAX_DIM];
    oracle_image(p, row, m_lo, m_hi);

    int64_t T = total_cells(p);
    for (int64_t t = 0; t < T; ++t) {
        double u_t = 1.0, l_t = 1.0;
        for (int d = 0; d < n; ++d) {
            int i = cell_digit(p, t, d);
            double c = oracle_edge(p, d, i);
            double e = oracle_edge(p, d, i + 1);
            double s = p->sigma[d];
            double mid = 0.5 * (c + e);
            double g_max = oracle_phi_diff(c, e, clamp(mid, m_lo[d], m_hi[d]), s);
            double g_a = oracle_phi_diff(c, e, m_lo[d], s);
            double g_b = oracle_phi_diff(c, e, m_hi[d], s);
            u_t *= g_max;
            l_t *= g_a < g_b ? g_a : g_b;
        }
        up[t] = u_t;
        lo[t] = l_t;
    }

    double in_max = 1.0, in_min = 1.0;
    for (int d = 0; d < n; ++d) {
        double s = p->sigma[d];
        double mid = 0.5 * (p->lo[d] + p->hi[d]);
        double G_max = oracle_phi_diff(p->lo[d], p->hi[d], clamp(mid, m_lo[d], m_hi[d]), s);
        double G_a = oracle_phi_diff(p->lo[d], p->hi[d], m_lo[d], s);
        double G_b = oracle_phi_diff(p->lo[d], p->hi[d], m_hi[d], s);
        in_max *= G_max;
        in_min *= G_a < G_b ? G_a : G_b;
    }
    *sink_lo = 1.0 - in_max;
    *sink_up = 1.0 - in_min;
}

/* ---- batch driver: rows -> CSR, two calls (run, then fetch) ---------------- */

typedef struct {
    int64_t count;
    int32_t *col;
    double *lo, *up;
    double sink_lo, sink_up, trunc;
} oracle_row_result;

typedef struct {
    int64_t nrows;
    oracle_row_result *r;
} oracle_batch;

/* Neumaier's compensated summation step. */
static void neumaier_add(double *sum, double *comp, double x)
{
    double t = *sum + x;
    if (fabs(*sum) >= fabs(x)) *comp += (*sum - t) + x;
    else *comp += (x - t) + *sum;
    *sum = t;
}

/*
 * Build the CSR rows listed in `rows` (any order, any subset). Keeps target t
 * iff up_t >= cutoff (ties kept, cutoff 0 keeps everything), columns ascend,
 * trunc = Neumaier sum of the dropped up_t. Returns an opaque handle; *nnz is
 * the total number of kept pairs. threads <= 0 uses the OpenMP default.
 */
void *oracle_run(const oracle_problem *p, const int64_t *rows, int64_t nrows, int threads,
                 int64_t *nnz)
{
    oracle_batch *b = (oracle_batch *)calloc(1, sizeof(oracle_batch));
    b->nrows = nrows;
    b->r = (oracle_row_result *)calloc((size_t)(nrows > 0 ? nrows : 1), sizeof(oracle_row_result));
    int64_t T = total_cells(p);
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel
    {
        double *up = (double *)malloc(sizeof(double) * (size_t)T);
        double *lo = (double *)malloc(sizeof(double) * (size_t)T);
#pragma omp for schedule(dynamic, 1)
        for (int64_t k = 0; k < nrows; ++k) {
            oracle_row_result *res = &b->r[k];
            oracle_row_dense(p, rows[k], up, lo, &res->sink_lo, &res->sink_up);
            int64_t cnt = 0;
            double s = 0.0, comp = 0.0;
            for (int64_t t = 0; t < T; ++t) {
                if (up[t] >= p->cutoff) ++cnt;
                else neumaier_add(&s, &comp, up[t]);
            }
            res->trunc = s + comp;
            res->count = cnt;
            res->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1));
            res->lo = (double *)malloc(sizeof(double) * (size_t)(cnt > 0 ? cnt : 1));
            res->up = (double *)malloc(sizeof(double) * (size_t)(cnt > 0 ? cnt : 1));
            int64_t w = 0;
            for (int64_t t = 0; t < T; ++t) {
                if (up[t] >= p->cutoff) {
                    res->col[w] = (int32_t)t;
                    res->lo[w] = lo[t];
                    res->up[w] = up[t];
                    ++w;
                }
            }
        }
        free(up);
        free(lo);
    }
    int64_t total = 0;
    for (int64_t k = 0; k < nrows; ++k) total += b->r[k].count;
    *nnz = total;
    return b;
}

/* Copy a batch out (row_ptr has nrows+1 entries) and keep the handle. */
void oracle_fetch(void *handle, int64_t *row_ptr, int32_t *col, double *lo, double *up,
                  double *sink_lo, double *sink_up, double *trunc)
{
    oracle_batch *b = (oracle_batch *)handle;
    int64_t off = 0;
    for (int64_t k = 0; k < b->nrows; ++k) {
        oracle_row_result *res = &b->r[k];
        row_ptr[k] = off;
        memcpy(col + off, res->col, sizeof(int32_t) * (size_t)res->count);
        memcpy(lo + off, res->lo, sizeof(double) * (size_t)res->count);
        memcpy(up + off, res->up, sizeof(double) * (size_t)res->count);
        sink_lo[k] = res->sink_lo;
        sink_up[k] = res->sink_up;
        trunc[k] = res->trunc;
        off += res->count;
    }
    row_ptr[b->nrows] = off;
}

void oracle_release(void *handle)
{
    oracle_batch *b = (oracle_batch *)handle;
    if (!b) return;
    for (int64_t k = 0; k < b->nrows; ++k) {
        free(b->r[k].col);
        free(b->r[k].lo);
        free(b->r[k].up);
    }
    free(b->r);
    free(b);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- target / avoid regions (Sec. 3.1, Alg. 1, Remark 4.1) --------------- */

enum { ORACLE_FREE = 0, ORACLE_TARGET = 1, ORACLE_AVOID = 2 };

/* Centre of cell i of dimension d. */
static double cell_centre(const oracle_problem *p, int d, int i)
{
    return 0.5 * (oracle_edge(p, d, i) + oracle_edge(p, d, i + 1));
}

/*
 * Cells of one region box: in every dimension the cells whose centre lies in
 * the closed interval [box_lo_d, box_hi_d] (a contiguous index range). Writes
 * the first and last index per dimension; returns 0 when no cell qualifies.
 */
int oracle_box_cells(const oracle_problem *p, const double *box_lo, const double *box_hi,
                     int *first, int *last)
{
    for (int d = 0; d < p->n; ++d) {
        first[d] = -1;
        last[d] = -2;
        for (int i = 0; i < p->cells[d]; ++i) {
            double c = cell_centre(p, d, i);
            if (c >= box_lo[d] && c <= box_hi[d]) {
                if (first[d] < 0) first[d] = i;
                last[d] = i;
            }
        }
        if (first[d] < 0) return 0;
    }
    return 1;
}

/*
 * Labels of every cell (Sec. 3.1: target and avoid states are absorbing): a
 * cell is avoid if its centre lies in an avoid box, else target if it lies in
 * a target box, else free. Boxes: [count][n] lower and upper corners.
 */
void oracle_labels(const oracle_problem *p, int n_target, const double *t_lo, const double *t_hi,
                   int n_avoid, const double *a_lo, const double *a_hi, uint8_t *labels)
{
    int64_t T = total_cells(p);
    for (int64_t t = 0; t < T; ++t) {
        uint8_t lab = ORACLE_FREE;
        for (int k = 0; k < n_target + n_avoid; ++k) {
            int avoid = k >= n_target;
            const double *lo = avoid ? a_lo + (k - n_target) * p->n : t_lo + k * p->n;
            const double *hi = avoid ? a_hi + (k - n_target) * p->n : t_hi + k * p->n;
            int in = 1;
            for (int d = 0; d < p->n && in; ++d) {
                double c = cell_centre(p, d, cell_digit(p, t, d));
                in = c >= lo[d] && c <= hi[d];
            }
            if (in && avoid) lab = ORACLE_AVOID;
            else if (in && lab == ORACLE_FREE) lab = ORACLE_TARGET;
        }
        labels[t] = lab;
    }
}

/*
 * Region vectors of one row: out = (R_min, R_max, A_min, A_max).
 *   mode 1 (the paper's sums, Alg. 1): R = sum over the target-labelled
 *     cells of the per-cell bounds [lo_t, up_t] (every cell, no cutoff);
 *     A = the same over the avoid cells plus the sink bounds (Remark 4.1).
 *   mode 0 (one relaxation per region box): each box is replaced by the
 *     union of its cells, [edge first_d, edge last_d + 1] per dimension, and
 *     bounded like one big target cell: up = prod_d g_d(clamp(mid_d)),
 *     lo = prod_d min(g_d(m_lo_d), g_d(m_hi_d)); R and A sum their boxes,
 *     A adds the sink.
 * `labels` (mode 1) comes from oracle_labels; the boxes (mode 0) must cover
 * pairwise disjoint sets of cells (checked by the caller).
 */
void oracle_region_row(const oracle_problem *p, int64_t row, int mode, const uint8_t *labels,
                       int n_target, const double *t_lo, const double *t_hi, int n_avoid,
                       const double *a_lo, const double *a_hi, double *out)
{
    int n = p->n;
    int64_t T = total_cells(p);
    double *up = (double *)malloc(sizeof(double) * (size_t)T);
    double *lo = (double *)malloc(sizeof(double) * (size_t)T);
    double sl, su;
    oracle_row_dense(p, row, up, lo, &sl, &su);
    double r_lo = 0.0, r_up = 0.0, x_lo = 0.0, x_up = 0.0;
    if (mode == 1) {
        for (int64_t t = 0; t < T; ++t) {
            if (labels[t] == ORACLE_TARGET) { r_lo += lo[t]; r_up += up[t]; }
            if (labels[t] == ORACLE_AVOID) { x_lo += lo[t]; x_up += up[t]; }
        }
    } else {
        double m_lo[ORACLE_MAX_DIM], m_hi[ORACLE_MAX_DIM];
        oracle_image(p, row, m_lo, m_hi);
        for (int k = 0; k < n_target + n_avoid; ++k) {
            int avoid = k >= n_target;
            const double *blo = avoid ? a_lo + (k - n_target) * n : t_lo + k * n;
            const double *bhi = avoid ? a_hi + (k - n_target) * n : t_hi + k * n;
            int first[ORACLE_MAX_DIM], last[ORACLE_MAX_DIM];
            if (!oracle_box_cells(p, blo, bhi, first, last)) continue;
            double b_up = 1.0, b_lo = 1.0;
            for (int d = 0; d < n; ++d) {
                double left = oracle_edge(p, d, first[d]);
                double right = oracle_edge(p, d, last[d] + 1);
                double sd = p->sigma[d];
                double centre = 0.5 * (left + right);
                double r_max = oracle_phi_diff(left, right, clamp(centre, m_lo[d], m_hi[d]), sd);
                double r_a = oracle_phi_diff(left, right, m_lo[d], sd);
                double r_b = oracle_phi_diff(left, right, m_hi[d], sd);
                b_up *= r_max;
                b_lo *= r_a < r_b ? r_a : r_b;
            }
            if (avoid) { x_lo += b_lo; x_up += b_up; }
            else { r_lo += b_lo; r_up += b_up; }
        }
    }
    out[0] = r_lo;
    out[1] = r_up;
    out[2] = sl + x_lo;
    out[3] = su + x_up;
    free(up);
    free(lo);
}

/* oracle_region_row over a list of rows (OpenMP), out: [nrows][4]. */
void oracle_region_rows(const oracle_problem *p, const int64_t *rows, int64_t nrows, int mode,
                        const uint8_t *labels, int n_target, const double *t_lo,
                        const double *t_hi, int n_avoid, const double *a_lo, const double *a_hi,
                        double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nrows; ++k)
        oracle_region_row(p, rows[k], mode, labels, n_target, t_lo, t_hi, n_avoid, a_lo, a_hi,
                          out + 4 * k);
}

/* ---- sampled noise (Sec. 4.1: full covariance or a custom distribution,
 * integrated by Monte-Carlo sampling) ------------------------------------- */

/*
 * Cell of dimension d that holds the coordinate y: -1 below the domain, N
 * above it, else the i with edge i <= y < edge i+1 (the last cell also holds
 * y == hi).
 */
int oracle_cell_of(const oracle_problem *p, int d, double y)
{
    int N = p->cells[d];
    if (y < oracle_edge(p, d, 0)) return -1;
    if (y > oracle_edge(p, d, N)) return N;
    for (int i = 0; i < N; ++i)
        if (y < oracle_edge(p, d, i + 1)) return i;
    return N - 1;
}

/*
 * Sample counts of one row. With the image box M = [m_lo, m_hi] of the row
 * and the noise samples w_s (samples[d * S + s], dimension-major), sample s
 * moves the box to w_s + M:
 *   up[t]    += 1 for every target cell t the moved box meets,
 *   lo[t]    += 1 for the one cell t that holds the whole moved box,
 *   sink_up  += 1 when the moved box is not inside the domain,
 *   sink_lo  += 1 when it lies entirely outside.
 * Divided by S these estimate P(w + M meets t) >= max over m in M of
 * P(m + w in t) and P(w + M inside t) <= the min (Def. 3.1 for a noise whose
 * cell masses have no closed form).
 */
void oracle_mc_row(const oracle_problem *p, int64_t row, const double *samples, int64_t S,
                   uint32_t *up, uint32_t *lo, int64_t *sink_lo, int64_t *sink_up)
{
    int n = p->n;
    double m_lo[ORACLE_MAX_DIM], m_hi[ORACLE_MAX_DIM];
    oracle_image(p, row, m_lo, m_hi);
    int64_t T = total_cells(p);
    memset(up, 0, sizeof(uint32_t) * (size_t)T);
    memset(lo, 0, sizeof(uint32_t) * (size_t)T);
    *sink_lo = 0;
    *sink_up = 0;
    for (int64_t s = 0; s < S; ++s) {
        int a[ORACLE_MAX_DIM], b[ORACLE_MAX_DIM];
        int inside = 1, outside = 0, single = 1;
        for (int d = 0; d < n; ++d) {
            double w = samples[(int64_t)d * S + s];
            a[d] = oracle_cell_of(p, d, w + m_lo[d]);
            b[d] = oracle_cell_of(p, d, w + m_hi[d]);
            if (a[d] < 0 || b[d] > p->cells[d] - 1) inside = 0;
            if (b[d] < 0 || a[d] > p->cells[d] - 1) outside = 1;
            if (a[d] != b[d]) single = 0;
        }
        if (!inside) ++*sink_up;
        if (outside) {
            ++*sink_lo;
            continue;
        }
        /* every target cell t: does the moved box meet it, hold it whole? */
        for (int64_t t = 0; t < T; ++t) {
            int meets = 1;
            for (int d = 0; d < n && meets; ++d) {
                int i = cell_digit(p, t, d);
                meets = a[d] <= i && i <= b[d];
            }
            if (meets) {
                ++up[t];
                if (single) ++lo[t];
            }
        }
    }
}

/* Build the rows listed from sampled noise (same layout and rules as
 * oracle_run: keep t iff up_t >= cutoff, trunc = dropped up mass), values
 * count / S. */
void *oracle_run_mc(const oracle_problem *p, const int64_t *rows, int64_t nrows,
                    const double *samples, int64_t S, int threads, int64_t *nnz)
{
    oracle_batch *b = (oracle_batch *)calloc(1, sizeof(oracle_batch));
    b->nrows = nrows;
    b->r = (oracle_row_result *)calloc((size_t)(nrows > 0 ? nrows : 1), sizeof(oracle_row_result));
    int64_t T = total_cells(p);
    const double dS = (double)S;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel
    {
        uint32_t *up = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)T);
        uint32_t *lo = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)T);
#pragma omp for schedule(dynamic, 1)
        for (int64_t k = 0; k < nrows; ++k) {
            oracle_row_result *res = &b->r[k];
            int64_t sl, su, cnt = 0, dropped = 0;
            oracle_mc_row(p, rows[k], samples, S, up, lo, &sl, &su);
            for (int64_t t = 0; t < T; ++t) {
                if ((double)up[t] / dS >= p->cutoff) ++cnt;
                else dropped += up[t];
            }
            res->sink_lo = (double)sl / dS;
            res->sink_up = (double)su / dS;
            res->trunc = (double)dropped / dS;
            res->count = cnt;
            res->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1));
            res->lo = (double *)malloc(sizeof(double) * (size_t)(cnt > 0 ? cnt : 1));
            res->up = (double *)malloc(sizeof(double) * (size_t)(cnt > 0 ? cnt : 1));
            int64_t w = 0;
            for (int64_t t = 0; t < T; ++t) {
                if ((double)up[t] / dS >= p->cutoff) {
                    res->col[w] = (int32_t)t;
                    res->lo[w] = (double)lo[t] / dS;
                    res->up[w] = (double)up[t] / dS;
                    ++w;
                }
            }
        }
        free(up);
        free(lo);
    }
    int64_t total = 0;
    for (int64_t k = 0; k < nrows; ++k) total += b->r[k].count;
    *nnz = total;
    return b;
}
