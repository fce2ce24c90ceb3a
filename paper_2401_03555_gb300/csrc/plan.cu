// plan.cu -- the host planner: validates one build's arguments and computes,
// in FP64 on the host, every per-build constant the kernels read (grid edges,
// per-term image tables, input offsets, window margins, plateau and
// out-of-domain constants, FP32 pair tables, the walk's shared-memory sizes),
// and packs them with the descriptor into the layout of the device tables.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "plan.h"

namespace impact {

namespace {

double next_down(double x) { return nextafter(x, -INFINITY); }
double next_up(double x) { return nextafter(x, INFINITY); }

// Smallest float >= x (x finite, representable range).
float f32_up(double x)
{
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}

float f32_down(double x)
{
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return f;
}

// Range of cos / sin over [a, b]: endpoint values, widened to +-1 where an
// extremum (k pi for cos, pi/2 + k pi for sin) lies inside. `slack` > 0 widens
// the interval used for the extremum test and the endpoint values (outward).
void trig_range(bool is_cos, double a, double b, double slack, double &lo, double &hi)
{
    double fa = is_cos ? cos(a) : sin(a);
    double fb = is_cos ? cos(b) : sin(b);
    lo = fa < fb ? fa : fb;
    hi = fa < fb ? fb : fa;
    double shift = is_cos ? 0.0 : M_PI_2;
    double a2 = a - slack, b2 = b + slack;
    for (long k = (long)ceil((a2 - shift) / M_PI); shift + (double)k * M_PI <= b2; ++k) {
        if (k % 2 == 0) hi = 1.0; else lo = -1.0;
    }
    if (slack > 0.0) {
        lo = std::max(-1.0, lo - 8.0 * 2.220446049250313e-16);
        hi = std::min(1.0, hi + 8.0 * 2.220446049250313e-16);
    }
}

// Fast division by N for x < 2^31: q = (umulhi(x, m) + x) >> s.
void div_magic(uint32_t N, uint32_t &m, int &s)
{
    int l = 0;
    while (((uint64_t)1 << l) < N) ++l;
    m = (uint32_t)(((((uint64_t)1 << l) - N) << 32) / N + 1);
    s = l;
}

float2 pair_of(double v)
{
    float hi = (float)v;
    float lo = (float)(v - (double)hi);
    return make_float2(hi, lo);
}

uint64_t fnv(uint64_t h, const void *p, size_t bytes)
{
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < bytes; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}


}  // namespace



size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

TableLayout table_layout(const Plan &p)
{
    TableLayout L;
    size_t o = 0;
    auto put = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    L.desc = put(sizeof(ImpactDesc));
    L.edges = put(p.edges.size() * 8);
    L.term_rn = put(p.term_rn.size() * 8);
    L.term_dn = put(p.term_dn.size() * 8);
    L.term_up = put(p.term_up.size() * 8);
    L.off_rn = put(p.off_rn.size() * 8);
    L.off_dn = put(p.off_dn.size() * 8);
    L.off_up = put(p.off_up.size() * 8);
    L.uni_rn = put(p.uni_rn.size() * 8);
    L.uni_sd = put(p.uni_sd.size() * 8);
    L.inputs = put(p.inputs.size() * 8);
    L.ea = put(p.ea.size() * 8);
    L.ta_lo = put(p.ta_lo.size() * 8);
    L.ta_hi = put(p.ta_hi.size() * 8);
    L.oa = put(p.oa.size() * 8);
    L.ua = put(p.ua.size() * 8);
    L.oma = put(p.oma.size() * 8);
    L.mu_lo = put(p.mu_lo.size() * 4);
    L.mu_hi = put(p.mu_hi.size() * 4);
    L.mo = put(p.mo.size() * 4);
    L.um = put(p.um.size() * 4);
    L.omm = put(p.omm.size() * 4);
    L.total = o;
    return L;
}


// z with P(Z >= z) = erfc(z/sqrt2)/2 <= p for a standard normal Z (bisection).
double normal_quantile_upper(double p)
{
    double lo = 0.0, hi = 40.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (0.5 * erfc(mid * M_SQRT1_2) <= p) hi = mid; else lo = mid;
    }
    return hi;
}

impact_status make_plan(const impact_system *sys, const impact_grid *grid,
                        const impact_inputs *inputs, const double *sigma, double cutoff,
                        impact_precision precision, Plan &P)
{
    if (!sys || !grid || !inputs || !sigma) return fail(IMPACT_ERR_ARG, "null argument");
    const int n = grid->n;
    if (n < 1 || n > IMPACT_MAX_DIM) return fail(IMPACT_ERR_ARG, "grid.n must be in [1, 8]");
    if (sys->n != n) return fail(IMPACT_ERR_ARG, "system.n != grid.n");
    if (!grid->lo || !grid->hi || !grid->cells) return fail(IMPACT_ERR_ARG, "null grid array");
    if (sys->kind < IMPACT_AFFINE || sys->kind > IMPACT_IMAGES)
        return fail(IMPACT_ERR_ARG, "unknown system kind");
    if (precision != IMPACT_FP64_PLAIN && precision != IMPACT_FP32_SOUND)
        return fail(IMPACT_ERR_ARG, "unknown precision");
    if (!(cutoff >= 0.0 && cutoff < 1.0)) return fail(IMPACT_ERR_ARG, "cutoff must be in [0, 1)");
    if (sys->params) return fail(IMPACT_ERR_ARG, "system.params is reserved and must be NULL");
    const int m = inputs->m;
    if (inputs->count < 1) return fail(IMPACT_ERR_ARG, "inputs.count must be >= 1");
    if (m < 0 || m > IMPACT_MAX_M) return fail(IMPACT_ERR_ARG, "inputs.m must be in [0, 8]");
    if (m > 0 && !inputs->points) return fail(IMPACT_ERR_ARG, "null input points");
    if (sys->kind == IMPACT_AFFINE) {
        if (!sys->A) return fail(IMPACT_ERR_ARG, "affine system needs A");
        if (sys->m != m) return fail(IMPACT_ERR_ARG, "system.m != inputs.m");
        if (m > 0 && !sys->B) return fail(IMPACT_ERR_ARG, "affine system with inputs needs B");
    } else if (sys->kind == IMPACT_UNICYCLE) {
        if (n != 3 || m != 2) return fail(IMPACT_ERR_ARG, "unicycle needs n = 3, m = 2");
    } else {
        if (!sys->dev_images) return fail(IMPACT_ERR_ARG, "images system needs dev_images");
    }
    int64_t cells = 1;
    for (int d = 0; d < n; ++d) {
        if (grid->cells[d] < 1) return fail(IMPACT_ERR_ARG, "cells must be >= 1");
        if (!(grid->lo[d] < grid->hi[d]) || !isfinite(grid->lo[d]) || !isfinite(grid->hi[d]))
            return fail(IMPACT_ERR_ARG, "grid needs finite lo < hi");
        if (!(sigma[d] > 0.0) || !isfinite(sigma[d]))
            return fail(IMPACT_ERR_ARG, "sigma must be finite and > 0");
        cells *= grid->cells[d];
        if (cells >= ((int64_t)1 << 31)) return fail(IMPACT_ERR_ARG, "more than 2^31-1 cells");
    }
    const int n_inputs = inputs->count;
    const int64_t rows = cells * n_inputs;

    ImpactDesc &D = P.desc;
    memset(&D, 0, sizeof(D));
    D.n = n;
    D.m = m;
    D.kind = sys->kind;
    D.prec = precision;
    D.n_inputs = n_inputs;
    D.n_in_split_min = 24;
    D.rows = rows;
    D.cells = cells;
    D.cutoff = cutoff;
    D.cutoff32 = f32_up(cutoff);
    D.table_max = IMPACT_TABLE_MAX;
    P.rows = rows;

    // grid edges (E_i = lo + i*h, E_N = hi), per-dimension constants
    int nmax = 0;
    int64_t stride = 1;
    for (int d = n - 1; d >= 0; --d) {
        D.dim[d].stride = (int)stride;
        stride *= grid->cells[d];
    }
    const double zc = cutoff > 0.0 ? normal_quantile_upper(0.5 * cutoff) : INFINITY;
    for (int d = 0; d < n; ++d) {
        ImpactDim &g = D.dim[d];
        const int N = grid->cells[d];
        nmax = std::max(nmax, N);
        g.lo = grid->lo[d];
        g.hi = grid->hi[d];
        g.N = N;
        g.h = (g.hi - g.lo) / (double)N;
        g.inv_h = 1.0 / g.h;
        g.sigma = sigma[d];
        g.inv_s = 1.0 / (sigma[d] * M_SQRT2);
        g.kappa = g.h * g.inv_s;
        g.kappa_hi = (float)g.kappa;
        g.kappa_lo = (float)(g.kappa - (double)g.kappa_hi);
        g.delta = isfinite(zc) ? sigma[d] * zc * (1.0 + 1e-9) : INFINITY;
        g.edge_off = (int)P.edges.size();
        double hmax = 0.0;
        for (int i = 0; i <= N; ++i) {
            double e = (i == N) ? g.hi : g.lo + (double)i * g.h;
            P.edges.push_back(e);
            if (i > 0) hmax = std::max(hmax, e - P.edges[P.edges.size() - 2]);
        }
        double mag = std::max(fabs(g.lo), fabs(g.hi));
        double dev = ldexp(mag + fabs(g.hi - g.lo), -51) + fabs(g.hi - (g.lo + (double)N * g.h)) +
                     ldexp(fabs(g.hi), -50);
        g.edge_err = f32_up(dev * g.inv_s * (1.0 + 1e-9) + 1e-300);
        double xp = hmax * g.inv_s * 0.5 * (1.0 + 1e-12);
        g.plateau_hi = std::min(1.0f, f32_up(erf(xp) + 4e-16));
        double xq = (g.hi - g.lo) * g.inv_s * 0.5 * (1.0 + 1e-12);
        g.qmin_lo = f32_down(erfc(xq) * (1.0 - 1e-13));
    }
    D.n_max = nmax;

    // inputs
    for (int j = 0; j < n_inputs; ++j)
        for (int k = 0; k < m; ++k) P.inputs.push_back(inputs->points[(int64_t)j * m + k]);

    // per-dimension window width bound -> nnz bound and staging need
    std::vector<double> width(n, 0.0);
    if (sys->kind == IMPACT_AFFINE) {
        const double *A = sys->A;
        // image terms: per (d, k, cell i of dim k) the range of A_dk * x_k
        P.term_rn.assign((size_t)n * n * nmax * 2, 0.0);
        P.term_dn.assign((size_t)n * n * nmax, 0.0);
        P.term_up.assign((size_t)n * n * nmax, 0.0);
        for (int d = 0; d < n; ++d) {
            for (int k = 0; k < n; ++k) {
                const double a = A[d * n + k];
                if (!isfinite(a)) return fail(IMPACT_ERR_ARG, "A must be finite");
                const ImpactDim &gk = D.dim[k];
                for (int i = 0; i < gk.N; ++i) {
                    double x0 = P.edges[gk.edge_off + i], x1 = P.edges[gk.edge_off + i + 1];
                    double p0 = a * x0, p1 = a * x1;
                    size_t t = ((size_t)(d * n + k) * nmax + i);
                    P.term_rn[2 * t] = p0 < p1 ? p0 : p1;
                    P.term_rn[2 * t + 1] = p0 < p1 ? p1 : p0;
                    // the rounded products are within half an ulp of the exact ones
                    P.term_dn[t] = std::min(next_down(p0), next_down(p1));
                    P.term_up[t] = std::max(next_up(p0), next_up(p1));
                }
                width[d] += fabs(a) * gk.h;
            }
        }
        // input offsets c_d + sum_k B_dk u_k, in the definition's order, and a bracket
        P.off_rn.assign((size_t)n_inputs * n, 0.0);
        P.off_dn.assign((size_t)n_inputs * n, 0.0);
        P.off_up.assign((size_t)n_inputs * n, 0.0);
        for (int j = 0; j < n_inputs; ++j) {
            const double *u = inputs->points ? inputs->points + (int64_t)j * m : nullptr;
            for (int d = 0; d < n; ++d) {
                double off = sys->c ? sys->c[d] : 0.0;
                double mag = fabs(off);
                for (int k = 0; k < m; ++k) {
                    double t = sys->B[d * m + k] * u[k];
                    off += t;
                    mag += fabs(t);
                }
                if (!isfinite(off)) return fail(IMPACT_ERR_ARG, "B, c and inputs must be finite");
                double err = ldexp(mag, -50) * (double)(m + 2) + 1e-300;
                P.off_rn[(size_t)j * n + d] = off;
                P.off_dn[(size_t)j * n + d] = next_down(off - err);
                P.off_up[(size_t)j * n + d] = next_up(off + err);
            }
        }
    } else if (sys->kind == IMPACT_UNICYCLE) {
        const ImpactDim &gt = D.dim[2];
        P.uni_rn.assign((size_t)gt.N * n_inputs * 4, 0.0);
        P.uni_sd.assign((size_t)gt.N * n_inputs * 4, 0.0);
        double vmax = 0.0;
        for (int i = 0; i < gt.N; ++i) {
            double a = P.edges[gt.edge_off + i], b = P.edges[gt.edge_off + i + 1];
            double cl, ch, sl, sh, cls, chs, sls, shs;
            trig_range(true, a, b, 0.0, cl, ch);
            trig_range(false, a, b, 0.0, sl, sh);
            trig_range(true, a, b, 1e-12, cls, chs);
            trig_range(false, a, b, 1e-12, sls, shs);
            for (int j = 0; j < n_inputs; ++j) {
                double v = inputs->points[(int64_t)j * m + 0];
                vmax = std::max(vmax, fabs(v));
                double *r = &P.uni_rn[((size_t)i * n_inputs + j) * 4];
                double *s = &P.uni_sd[((size_t)i * n_inputs + j) * 4];
                double c1 = v * cl, c2 = v * ch, s1 = v * sl, s2 = v * sh;
                r[0] = c1 < c2 ? c1 : c2;
                r[1] = c1 < c2 ? c2 : c1;
                r[2] = s1 < s2 ? s1 : s2;
                r[3] = s1 < s2 ? s2 : s1;
                double c3 = v * cls, c4 = v * chs, s3 = v * sls, s4 = v * shs;
                s[0] = next_down(std::min(c3, c4));
                s[1] = next_up(std::max(c3, c4));
                s[2] = next_down(std::min(s3, s4));
                s[3] = next_up(std::max(s3, s4));
            }
        }
        width[0] = D.dim[0].h + 2.0 * vmax;
        width[1] = D.dim[1].h + 2.0 * vmax;
        width[2] = D.dim[2].h;
    }
    // window widths: image width + 2 delta, plus the 2-cell slack and rounding
    // (caller images: the image width is unknown here, so rows whose window
    // is wider than 128 cells are refused at run time)
    int64_t box = 1;
    int64_t need = 0;
    int64_t tsum = 0;
    for (int d = 0; d < n; ++d) {
        ImpactDim &g = D.dim[d];
        int64_t w = g.N;
        if (sys->kind != IMPACT_IMAGES && isfinite(g.delta)) {
            double cw = ceil((width[d] + 2.0 * g.delta) * g.inv_h) + 4.0;
            if (cw < (double)g.N) w = (int64_t)cw;
        }
        box = std::min<int64_t>(box * w, cells);
        need += w;
        g.wcap = (int)(sys->kind == IMPACT_IMAGES ? std::min<int64_t>(w, 128) : w);
        g.delta_cells = isfinite(g.delta) ? (float)(g.delta * g.inv_h) : INFINITY;
        div_magic((uint32_t)g.N, g.div_m, g.div_s);
        tsum += g.wcap;
    }
    div_magic((uint32_t)n_inputs, D.inp_div_m, D.inp_div_s);
    P.table_need = (sys->kind == IMPACT_IMAGES) ? -1 : (int)std::min<int64_t>(need, INT32_MAX);
    if (box > cells) box = cells;
    P.nnz_bound = box * rows;
    if (precision == IMPACT_FP32_SOUND) {
        // a row record holds the window tables of every dimension (8 bytes
        // per target), which the walk copies into one warp's shared memory
        // beside its node lists and the leaf table of the last two
        // dimensions (staged up to IMPACT_LEAF_STAGE entries); wide windows
        // (cutoff 0 on a fine grid, wide noise) need more of it and fewer
        // warps per SM. The walk divides candidate and leaf indices by window
        // widths as umulhi(e, ceil(2^32 / tw)), exact while e tw < 2^32: the
        // leaf table needs wcap_m wcap_l^2 < 2^31, the node lists 64 tw^2
        // < 2^31.
        const int64_t wl = D.dim[n - 1].wcap, wm = n >= 2 ? D.dim[n - 2].wcap : 1;
        int64_t wmax = 0;
        for (int d = 0; d < n; ++d) wmax = std::max<int64_t>(wmax, D.dim[d].wcap);
        const int leaf_cap = (int)std::min<int64_t>(wm * wl, IMPACT_LEAF_STAGE);
        if (tsum > 4096 || wm * wl * wl >= ((int64_t)1 << 31) ||
            IMPACT_WALK_CAP * wmax * wmax >= ((int64_t)1 << 31) ||
            impact::walk_core_bytes(n, (int)tsum, leaf_cap) > IMPACT_WALK_SMEM_MAX)
            return fail(IMPACT_ERR_ARG,
                        "the per-row windows need " + std::to_string(tsum) +
                            " factor entries, more than one warp's shared memory holds: "
                            "raise the cutoff or use fewer cells");
        D.tsum_cap = (int)tsum;
        D.leaf_cap = leaf_cap;
        D.walk_core = impact::walk_core_bytes(n, D.tsum_cap, D.leaf_cap);
        D.rec_stride = (int)impact::record_stride(n, D.tsum_cap);
        int ro = 0;
        for (int d = 0; d < n; ++d) {
            D.dim[d].rec_off = ro;
            ro += D.dim[d].wcap;
        }
        // tables in erf units (x / (sigma sqrt2)) as FP32 pairs, and in cells
        for (int d = 0; d < n; ++d) {
            const ImpactDim &g = D.dim[d];
            for (int i = 0; i <= g.N; ++i) P.ea.push_back(pair_of(P.edges[g.edge_off + i] * g.inv_s));
        }
        if (sys->kind == IMPACT_AFFINE) {
            P.ta_lo.resize((size_t)n * n * nmax);
            P.ta_hi.resize((size_t)n * n * nmax);
            P.mu_lo.resize((size_t)n * n * nmax);
            P.mu_hi.resize((size_t)n * n * nmax);
            for (int d = 0; d < n; ++d) {
                const ImpactDim &g = D.dim[d];
                for (int k = 0; k < n; ++k)
                    for (int i = 0; i < D.dim[k].N; ++i) {
                        size_t t = (size_t)(d * n + k) * nmax + i;
                        P.ta_lo[t] = pair_of(P.term_rn[2 * t] * g.inv_s);
                        P.ta_hi[t] = pair_of(P.term_rn[2 * t + 1] * g.inv_s);
                        P.mu_lo[t] = (float)(P.term_rn[2 * t] * g.inv_h);
                        P.mu_hi[t] = (float)(P.term_rn[2 * t + 1] * g.inv_h);
                    }
            }
            P.oa.resize((size_t)n_inputs * n);
            P.mo.resize((size_t)n_inputs * n);
            for (int j = 0; j < n_inputs; ++j)
                for (int d = 0; d < n; ++d) {
                    const ImpactDim &g = D.dim[d];
                    double off = P.off_rn[(size_t)j * n + d];
                    P.oa[(size_t)j * n + d] = pair_of(off * g.inv_s);
                    P.mo[(size_t)j * n + d] = (float)((off - g.lo) * g.inv_h);
                }
        } else if (sys->kind == IMPACT_UNICYCLE) {
            const ImpactDim &gx = D.dim[0], &gy = D.dim[1], &gt = D.dim[2];
            size_t cnt = (size_t)gt.N * n_inputs * 4;
            P.ua.resize(cnt);
            P.um.resize(cnt);
            for (size_t t = 0; t < cnt; ++t) {
                const ImpactDim &g = (t % 4) < 2 ? gx : gy;
                P.ua[t] = pair_of(P.uni_sd[t] * g.inv_s);
                P.um[t] = (float)(P.uni_sd[t] * g.inv_h);
            }
            for (int j = 0; j < n_inputs; ++j) {
                double om = inputs->points[(int64_t)j * m + 1];
                P.oma.push_back(pair_of(om * gt.inv_s));
                P.omm.push_back((float)(om * gt.inv_h));
            }
        }
    }
    // identity of the arguments, for reusing a caller's workspace
    uint64_t h = 1469598103934665603ull;
    int hdr[5] = {sys->kind, n, m, (int)precision, n_inputs};
    h = fnv(h, hdr, sizeof(hdr));
    h = fnv(h, &cutoff, 8);
    h = fnv(h, grid->lo, 8 * n);
    h = fnv(h, grid->hi, 8 * n);
    h = fnv(h, grid->cells, 4 * n);
    h = fnv(h, sigma, 8 * n);
    if (sys->kind == IMPACT_AFFINE) {
        h = fnv(h, sys->A, 8 * n * n);
        if (m > 0) h = fnv(h, sys->B, 8 * n * m);
        if (sys->c) h = fnv(h, sys->c, 8 * n);
    }
    if (m > 0) h = fnv(h, inputs->points, 8 * (size_t)n_inputs * m);
    h = fnv(h, &sys->dev_images, sizeof(void *));
    P.hash = h;
    return IMPACT_OK;
}

void pack_tables(const Plan &P, unsigned char *host, unsigned char *dev_base,
                 const double *dev_images)
{
    const TableLayout L = table_layout(P);
    memset(host, 0, L.total);
    ImpactDesc D = P.desc;
    auto dp = [&](size_t off, size_t count) -> const void * {
        return count == 0 ? nullptr : (const void *)(dev_base + off);
    };
    D.edges = (const double *)dp(L.edges, P.edges.size());
    D.term_rn = (const double *)dp(L.term_rn, P.term_rn.size());
    D.term_dn = (const double *)dp(L.term_dn, P.term_dn.size());
    D.term_up = (const double *)dp(L.term_up, P.term_up.size());
    D.off_rn = (const double *)dp(L.off_rn, P.off_rn.size());
    D.off_dn = (const double *)dp(L.off_dn, P.off_dn.size());
    D.off_up = (const double *)dp(L.off_up, P.off_up.size());
    D.uni_rn = (const double *)dp(L.uni_rn, P.uni_rn.size());
    D.uni_sd = (const double *)dp(L.uni_sd, P.uni_sd.size());
    D.inputs = (const double *)dp(L.inputs, P.inputs.size());
    D.ea = (const float2 *)dp(L.ea, P.ea.size());
    D.ta_lo = (const float2 *)dp(L.ta_lo, P.ta_lo.size());
    D.ta_hi = (const float2 *)dp(L.ta_hi, P.ta_hi.size());
    D.oa = (const float2 *)dp(L.oa, P.oa.size());
    D.ua = (const float2 *)dp(L.ua, P.ua.size());
    D.oma = (const float2 *)dp(L.oma, P.oma.size());
    D.mu_lo = (const float *)dp(L.mu_lo, P.mu_lo.size());
    D.mu_hi = (const float *)dp(L.mu_hi, P.mu_hi.size());
    D.mo = (const float *)dp(L.mo, P.mo.size());
    D.um = (const float *)dp(L.um, P.um.size());
    D.omm = (const float *)dp(L.omm, P.omm.size());
    D.images = dev_images;
    memcpy(host + L.desc, &D, sizeof(D));
    auto put = [&](size_t off, const void *src, size_t bytes) {
        if (bytes) memcpy(host + off, src, bytes);
    };
    put(L.edges, P.edges.data(), P.edges.size() * 8);
    put(L.term_rn, P.term_rn.data(), P.term_rn.size() * 8);
    put(L.term_dn, P.term_dn.data(), P.term_dn.size() * 8);
    put(L.term_up, P.term_up.data(), P.term_up.size() * 8);
    put(L.off_rn, P.off_rn.data(), P.off_rn.size() * 8);
    put(L.off_dn, P.off_dn.data(), P.off_dn.size() * 8);
    put(L.off_up, P.off_up.data(), P.off_up.size() * 8);
    put(L.uni_rn, P.uni_rn.data(), P.uni_rn.size() * 8);
    put(L.uni_sd, P.uni_sd.data(), P.uni_sd.size() * 8);
    put(L.inputs, P.inputs.data(), P.inputs.size() * 8);
    put(L.ea, P.ea.data(), P.ea.size() * 8);
    put(L.ta_lo, P.ta_lo.data(), P.ta_lo.size() * 8);
    put(L.ta_hi, P.ta_hi.data(), P.ta_hi.size() * 8);
    put(L.oa, P.oa.data(), P.oa.size() * 8);
    put(L.ua, P.ua.data(), P.ua.size() * 8);
    put(L.oma, P.oma.data(), P.oma.size() * 8);
    put(L.mu_lo, P.mu_lo.data(), P.mu_lo.size() * 4);
    put(L.mu_hi, P.mu_hi.data(), P.mu_hi.size() * 4);
    put(L.mo, P.mo.data(), P.mo.size() * 4);
    put(L.um, P.um.data(), P.um.size() * 4);
    put(L.omm, P.omm.data(), P.omm.size() * 4);
}

}  // namespace impact
