/*
 * sslic_oracle.c -- plain single-threaded CPU oracle for Scalable SLIC
 * (arXiv 1806.08741).  TEST INFRASTRUCTURE ONLY: never linked into, or
 * called by, the product library.  See sslic_oracle.h for the layout and the
 * two arithmetic modes.
 *
 * Build: cc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no -ffast-math).
 * -ffp-contract=off keeps every product and sum a separately rounded IEEE
 * operation, which is what "FP32 canonical" means below.
 *
 * Readings of the paper used here (the paper leaves these open):
 *  R1  seeding lattice: n_d = ceil(N_d/S_d) seeds per axis at
 *      o_d + j*S_d with o_d = floor((N_d - 1 - (n_d - 1)*S_d)/2); cluster
 *      index k is the raster index of (j_0..j_{n-1}), j_0 fastest.
 *  R2  gradient magnitude^2 = sum_c sum_d (I_c(x+e_d) - I_c(x-e_d))^2,
 *      central differences in index space, neighbours outside the image
 *      clamped to the border; the 1/2 factor and the square root are dropped
 *      (neither changes the ordering).
 *  R3  perturbation: best = the seed itself, then the 3^n offsets in raster
 *      order (dim 0 fastest) replace it only on a strictly smaller gradient.
 *  R4  l and d are reset at the start of every iteration.
 *  R5  window of centre c along axis d: c - S_d <= x_d < c + S_d, evaluated
 *      as (x_d - S_d) < c && c <= (x_d + S_d) in the mode's precision.
 *  R6  D^2 evaluation order (FP32 canonical, one rounding per op, no FMA):
 *      e_c = I_c - C_c; dc = ((e_0^2 + e_1^2) + ...) ; t_d = w_d*(delta_d^2)
 *      with delta_d = x_d - c_d and w_d = float(m^2/S_d^2 in double);
 *      ds = ((t_0 + t_1) + ...); D^2 = dc + ds.
 *  R7  ties go to the lowest k (centres visited in ascending k, strict <).
 *  R8  voxels covered by no window keep label -1 and are not accumulated.
 *  R9  integer images: exact int64 sums, centre = float(double(sum)/double(n));
 *      float images: double sums; empty clusters keep their previous centre.
 *  R10 residual = mean over non-empty clusters of sqrt(D^2(C_prev, C_new))
 *      in double with w_d = m^2/S_d^2; stop after the iteration in which it
 *      falls below a positive threshold.
 *  R11 connectivity uses face adjacency (2n neighbours).
 *  R12 phase 1 seed: p = round-half-up(c_k) clamped; if l(p) == k use p,
 *      else the raster-first voxel of label k in the box of offsets
 *      -floor(S_d/2) .. ceil(S_d/2)-1 around p; final iff 4*size > prod S_d.
 *  R13 flood fills run on the pre-relabel labels; new labels count up from K
 *      in scan order.
 *  R14 "last encountered label" = output label of x - e_d for the smallest d
 *      with x_d > 0 (x is the raster-first voxel of its component); the
 *      component at the origin gets a new label.
 *  R15 labels are not compacted; centres are not recomputed afterwards.
 *  R16 colour input: the paper clusters colour in CIE-Lab (Sec. 2, 2.1) and
 *      converts its 8-bit RGB volume to CIE-Lab float first (Sec. 4.1) but
 *      names neither the RGB space nor the white point.  Read as sRGB
 *      (IEC 61966-2-1: its piecewise transfer function and its 4-decimal
 *      RGB->XYZ matrix), the D65 white (0.95047, 1, 1.08883) and CIE 1976
 *      L*a*b*: the one combination whose extremes over the 8-bit cube give
 *      the L, a and b ranges Sec. 2.1 prints, to its three decimals.
 */
#include "sslic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

/* images of 1 to ND dimensions (the paper's filter is n-dimensional, Sec. 3) */
#define ND 4

typedef struct {
    int n;              /* spatial dims actually used */
    int64_t N[ND];      /* sizes, padded with 1 */
    int64_t stride[ND]; /* raster strides */
    int64_t V;          /* voxel count */
    int C;              /* channels */
    int dt;             /* dtype */
    int S[ND];          /* grid, padded with 1 */
    int64_t ns[ND];     /* seeds per axis, padded with 1 */
    int64_t K;          /* clusters */
    int fp64;           /* arithmetic mode */
    float w32[ND];      /* fl32(m^2 / S_d^2) */
    double w64[ND];     /* m^2 / S_d^2 */
} geom;

static int make_geom(const oracle_params* p, geom* g)
{
    if (!p) return ORACLE_EINVAL;
    if (p->ndim < 1 || p->ndim > ND) return ORACLE_EINVAL;
    if (p->channels < 1) return ORACLE_EINVAL;
    if (p->dtype != ORACLE_U8 && p->dtype != ORACLE_U16 && p->dtype != ORACLE_F32) return ORACLE_EINVAL;
    if (p->mode != ORACLE_FP32 && p->mode != ORACLE_FP64) return ORACLE_EINVAL;
    if (!(p->m > 0.0) || !isfinite(p->m)) return ORACLE_EINVAL;
    if (p->max_iter < 1) return ORACLE_EINVAL;
    memset(g, 0, sizeof(*g));
    g->n = p->ndim;
    g->C = p->channels;
    g->dt = p->dtype;
    g->fp64 = (p->mode == ORACLE_FP64);
    g->V = 1;
    g->K = 1;
    for (int d = 0; d < ND; ++d) {
        if (d < g->n) {
            /* positions must be exact in float: N_d <= 2^24 */
            if (p->size[d] < 1 || p->size[d] > (1 << 24)) return ORACLE_EINVAL;
            if (p->grid[d] < 1) return ORACLE_EINVAL;
            g->N[d] = p->size[d];
            g->S[d] = p->grid[d];
        } else {
            g->N[d] = 1;
            g->S[d] = 1;
        }
        g->ns[d] = (g->N[d] + g->S[d] - 1) / g->S[d];
        g->stride[d] = g->V;
        g->V *= g->N[d];
        g->K *= g->ns[d];
        double s = (double)g->S[d];
        g->w64[d] = (p->m * p->m) / (s * s);
        g->w32[d] = (float)g->w64[d];
    }
    return ORACLE_OK;
}

int64_t oracle_num_clusters(const oracle_params* p)
{
    geom g;
    if (make_geom(p, &g) != ORACLE_OK) return -1;
    return g.K;
}

/* ---- pixel access ------------------------------------------------------ */

/* channel c of voxel q as a double (exact for every supported dtype) */
static double pix(const geom* g, const void* image, int64_t q, int c)
{
    int64_t i = q * g->C + c;
    switch (g->dt) {
    case ORACLE_U8: return (double)((const uint8_t*)image)[i];
    case ORACLE_U16: return (double)((const uint16_t*)image)[i];
    default: return (double)((const float*)image)[i];
    }
}

static int64_t pix_int(const geom* g, const void* image, int64_t q, int c)
{
    int64_t i = q * g->C + c;
    if (g->dt == ORACLE_U8) return (int64_t)((const uint8_t*)image)[i];
    return (int64_t)((const uint16_t*)image)[i];
}

static void coords(const geom* g, int64_t q, int64_t* x)
{
    for (int d = 0; d < ND; ++d) x[d] = (q / g->stride[d]) % g->N[d];
}

static int64_t index_of(const geom* g, const int64_t* x)
{
    int64_t q = 0;
    for (int d = 0; d < ND; ++d) q += x[d] * g->stride[d];
    return q;
}

/* The points of the box lo..hi (inclusive on every axis) in raster order,
 * dimension 0 fastest: box_first sets x to the first point (0: the box is
 * empty), box_next moves x to the next one (0: x was the last). */
static int box_first(int64_t* x, const int64_t* lo, const int64_t* hi)
{
    int ok = 1;
    for (int d = 0; d < ND; ++d) {
        x[d] = lo[d];
        ok = ok && lo[d] <= hi[d];
    }
    return ok;
}

static int box_next(int64_t* x, const int64_t* lo, const int64_t* hi)
{
    for (int d = 0; d < ND; ++d) {
        if (x[d] < hi[d]) {
            ++x[d];
            return 1;
        }
        x[d] = lo[d];
    }
    return 0;
}

/* ---- gradient (R2) ------------------------------------------------------ */

static double gradient(const geom* g, const void* image, int64_t q)
{
    int64_t x[ND];
    coords(g, q, x);
    if (g->dt != ORACLE_F32) {
        /* integer images: exact in int64 */
        int64_t acc = 0;
        for (int c = 0; c < g->C; ++c) {
            for (int d = 0; d < g->n; ++d) {
                int64_t hi = x[d] + 1 < g->N[d] ? q + g->stride[d] : q;
                int64_t lo = x[d] > 0 ? q - g->stride[d] : q;
                int64_t diff = pix_int(g, image, hi, c) - pix_int(g, image, lo, c);
                acc += diff * diff;
            }
        }
        return (double)acc;
    }
    if (!g->fp64) {
        /* float images, FP32 canonical: channel outer, axis inner, left to right */
        float acc = 0.0f;
        int first = 1;
        for (int c = 0; c < g->C; ++c) {
            for (int d = 0; d < g->n; ++d) {
                int64_t hi = x[d] + 1 < g->N[d] ? q + g->stride[d] : q;
                int64_t lo = x[d] > 0 ? q - g->stride[d] : q;
                float diff = (float)pix(g, image, hi, c) - (float)pix(g, image, lo, c);
                float sq = diff * diff;
                acc = first ? sq : acc + sq;
                first = 0;
            }
        }
        return (double)acc;
    }
    double acc = 0.0;
    for (int c = 0; c < g->C; ++c) {
        for (int d = 0; d < g->n; ++d) {
            int64_t hi = x[d] + 1 < g->N[d] ? q + g->stride[d] : q;
            int64_t lo = x[d] > 0 ? q - g->stride[d] : q;
            double diff = pix(g, image, hi, c) - pix(g, image, lo, c);
            acc += diff * diff;
        }
    }
    return acc;
}

double oracle_gradient(const oracle_params* p, const void* image, int64_t q)
{
    geom g;
    if (make_geom(p, &g) != ORACLE_OK || q < 0) return -1.0;
    if (q >= g.V) return -1.0;
    return gradient(&g, image, q);
}

/* ---- seeding and perturbation (R1, R3) ---------------------------------- */

static void store_centre(const geom* g, const void* image, int64_t q, double* row)
{
    int64_t x[ND];
    coords(g, q, x);
    for (int c = 0; c < g->C; ++c) {
        double v = pix(g, image, q, c);
        row[c] = g->fp64 ? v : (double)(float)v;
    }
    for (int d = 0; d < g->n; ++d) row[g->C + d] = (double)x[d];
}

static int seed(const geom* g, int perturb, const void* image, double* centres)
{
    const int width = g->C + g->n;
    for (int64_t k = 0; k < g->K; ++k) {
        int64_t x[ND];
        int64_t rem = k;
        for (int d = 0; d < ND; ++d) {
            int64_t j = rem % g->ns[d];
            rem /= g->ns[d];
            int64_t o = (g->N[d] - 1 - (g->ns[d] - 1) * g->S[d]) / 2;
            x[d] = o + j * g->S[d];
        }
        int64_t best = index_of(g, x);
        if (perturb) {
            double best_g = gradient(g, image, best);
            /* 3^n offsets in raster order, dimension 0 fastest */
            int64_t lo[ND], hi[ND], y[ND];
            for (int d = 0; d < ND; ++d) {
                lo[d] = d < g->n ? x[d] - 1 : 0;
                hi[d] = d < g->n ? x[d] + 1 : 0;
            }
            for (int more = box_first(y, lo, hi); more; more = box_next(y, lo, hi)) {
                int inside = 1;
                for (int d = 0; d < ND; ++d)
                    if (y[d] < 0 || y[d] >= g->N[d]) inside = 0;
                if (!inside) continue;
                int64_t q = index_of(g, y);
                double gq = gradient(g, image, q);
                if (gq < best_g) {
                    best_g = gq;
                    best = q;
                }
            }
        }
        store_centre(g, image, best, centres + k * width);
    }
    return ORACLE_OK;
}

int oracle_seed(const oracle_params* p, const void* image, double* centres)
{
    geom g;
    int rc = make_geom(p, &g);
    if (rc != ORACLE_OK) return rc;
    if (!image || !centres) return ORACLE_EINVAL;
    return seed(&g, p->perturb, image, centres);
}

/* ---- distance (R6) ------------------------------------------------------ */

static float dist32(const geom* g, const float* f, const int64_t* x, const double* ctr)
{
    float dc = 0.0f;
    for (int c = 0; c < g->C; ++c) {
        float e = f[c] - (float)ctr[c];
        float sq = e * e;
        dc = (c == 0) ? sq : dc + sq;
    }
    float ds = 0.0f;
    for (int d = 0; d < g->n; ++d) {
        float delta = (float)x[d] - (float)ctr[g->C + d];
        float dd = delta * delta;
        float t = g->w32[d] * dd;
        ds = (d == 0) ? t : ds + t;
    }
    return dc + ds;
}

static double dist64(const geom* g, const double* f, const int64_t* x, const double* ctr)
{
    double dc = 0.0;
    for (int c = 0; c < g->C; ++c) {
        double e = f[c] - ctr[c];
        dc = (c == 0) ? e * e : dc + e * e;
    }
    double ds = 0.0;
    for (int d = 0; d < g->n; ++d) {
        double delta = (double)x[d] - ctr[g->C + d];
        double t = g->w64[d] * (delta * delta);
        ds = (d == 0) ? t : ds + t;
    }
    return dc + ds;
}

double oracle_distance(const oracle_params* p, const double* feature,
                       const int64_t* pos, const double* centre)
{
    geom g;
    if (make_geom(p, &g) != ORACLE_OK) return -1.0;
    int64_t x[ND] = {0};
    for (int d = 0; d < g.n; ++d) x[d] = pos[d];
    if (g.fp64) return dist64(&g, feature, x, centre);
    float f[4096];
    if (g.C > 4096) return -1.0;
    for (int c = 0; c < g.C; ++c) f[c] = (float)feature[c];
    return (double)dist32(&g, f, x, centre);
}

/* ---- assignment (Sec. 2.2 / 3.1 step 2; R4, R5, R7, R8) ------------------ */

/* window test along one axis (R5) */
static int in_window(const geom* g, int d, int64_t xd, double c)
{
    if (g->fp64) return (double)(xd - g->S[d]) < c && c <= (double)(xd + g->S[d]);
    float cf = (float)c;
    return (float)(xd - g->S[d]) < cf && cf <= (float)(xd + g->S[d]);
}

/* The assignment of the voxels in planes plo .. phi-1 of the last axis
 * (all of them: plo = 0, phi = N_{n-1}).  A voxel sees the same centres in
 * the same order whatever range it is assigned in, so splitting the image
 * into such ranges leaves every label unchanged (the paper's non-overlapping
 * regions, Sec. 3.1). */
static int assign_planes(const geom* g, const void* image, const double* centres, int64_t K,
                         int32_t* labels, int64_t plo, int64_t phi)
{
    const int width = g->C + g->n;
    const int last = g->n - 1;
    const int64_t qlo = plo * g->stride[last], qhi = phi * g->stride[last];
    const int64_t nq = qhi - qlo;
    float* d32 = NULL;
    double* d64 = NULL;
    if (g->fp64) d64 = (double*)malloc((size_t)(nq > 0 ? nq : 1) * sizeof(double));
    else d32 = (float*)malloc((size_t)(nq > 0 ? nq : 1) * sizeof(float));
    float* f32 = (float*)malloc((size_t)g->C * sizeof(float));
    double* f64 = (double*)malloc((size_t)g->C * sizeof(double));
    int64_t* xs[ND] = {NULL};
    int64_t len[ND];
    int ok = (d32 || d64) && f32 && f64;
    for (int d = 0; d < ND && ok; ++d) {
        xs[d] = (int64_t*)malloc((size_t)(2 * g->S[d] + 3) * sizeof(int64_t));
        if (!xs[d]) ok = 0;
    }
    if (!ok) {
        free(d32); free(d64); free(f32); free(f64);
        for (int d = 0; d < ND; ++d) free(xs[d]);
        return ORACLE_ENOMEM;
    }
    /* R4: reset l = undefined (-1), d = +inf */
    for (int64_t q = qlo; q < qhi; ++q) {
        labels[q] = -1;
        if (g->fp64) d64[q - qlo] = INFINITY;
        else d32[q - qlo] = INFINITY;
    }
    for (int64_t k = 0; k < K; ++k) {
        const double* ctr = centres + k * width;
        /* the window of centre k, axis by axis (R5) */
        for (int d = 0; d < ND; ++d) {
            len[d] = 0;
            if (d >= g->n) {
                xs[d][len[d]++] = 0;
                continue;
            }
            double c = ctr[g->C + d];
            int64_t fl = (int64_t)floor(c);
            for (int64_t xd = fl - g->S[d] - 1; xd <= fl + g->S[d] + 1; ++xd) {
                if (xd < 0 || xd >= g->N[d]) continue;
                if (d == last && (xd < plo || xd >= phi)) continue;
                if (in_window(g, d, xd, c)) xs[d][len[d]++] = xd;
            }
        }
        /* the window's voxels in raster order */
        int64_t ilo[ND], ihi[ND], ii[ND];
        for (int d = 0; d < ND; ++d) {
            ilo[d] = 0;
            ihi[d] = len[d] - 1;
        }
        for (int more = box_first(ii, ilo, ihi); more; more = box_next(ii, ilo, ihi)) {
            int64_t x[ND];
            for (int d = 0; d < ND; ++d) x[d] = xs[d][ii[d]];
            int64_t q = index_of(g, x);
            if (g->fp64) {
                for (int c = 0; c < g->C; ++c) f64[c] = pix(g, image, q, c);
                double D = dist64(g, f64, x, ctr);
                if (D < d64[q - qlo]) { d64[q - qlo] = D; labels[q] = (int32_t)k; }
            } else {
                for (int c = 0; c < g->C; ++c) f32[c] = (float)pix(g, image, q, c);
                float D = dist32(g, f32, x, ctr);
                if (D < d32[q - qlo]) { d32[q - qlo] = D; labels[q] = (int32_t)k; }
            }
        }
    }
    free(d32); free(d64); free(f32); free(f64);
    for (int d = 0; d < ND; ++d) free(xs[d]);
    return ORACLE_OK;
}

static int assign(const geom* g, const void* image, const double* centres, int64_t K,
                  int32_t* labels)
{
    return assign_planes(g, image, centres, K, labels, 0, g->N[g->n - 1]);
}

int oracle_assign(const oracle_params* p, const void* image, const double* centres,
                  int64_t K, int32_t* labels)
{
    geom g;
    int rc = make_geom(p, &g);
    if (rc != ORACLE_OK) return rc;
    if (!image || !centres || !labels || K < 0 || K > 0x7fffffffLL) return ORACLE_EINVAL;
    return assign(&g, image, centres, K, labels);
}

/* The assignment at chosen voxels only, for images too large for
 * oracle_assign: the same rule as assign() above, evaluated for one voxel at
 * a time.  The centre loop of assign() visits every centre in ascending k
 * and keeps a strictly smaller D^2; at one voxel that is the lexicographic
 * minimum of (D^2, k) over the centres whose window covers it, which does
 * not depend on the order the candidates are listed in. */
int oracle_assign_voxels(const oracle_params* p, const void* image, const double* centres, int64_t K,
                         const int64_t* q, int64_t nq, const int64_t* cand_start, const int64_t* cand,
                         int32_t* labels_out)
{
    geom g;
    int rc = make_geom(p, &g);
    if (rc != ORACLE_OK) return rc;
    if (nq < 0 || (nq > 0 && (!image || !centres || !q || !cand_start || !cand || !labels_out)))
        return ORACLE_EINVAL;
    const int width = g.C + g.n;
    float* f32 = (float*)malloc((size_t)g.C * sizeof(float));
    double* f64 = (double*)malloc((size_t)g.C * sizeof(double));
    if (!f32 || !f64) { free(f32); free(f64); return ORACLE_ENOMEM; }
    for (int64_t i = 0; i < nq; ++i) {
        if (q[i] < 0 || q[i] >= g.V) { free(f32); free(f64); return ORACLE_EINVAL; }
        int64_t x[ND];
        coords(&g, q[i], x);
        for (int c = 0; c < g.C; ++c) {
            f64[c] = pix(&g, image, q[i], c);
            f32[c] = (float)f64[c];
        }
        int32_t best = -1;
        double bd64 = INFINITY;
        float bd32 = INFINITY;
        for (int64_t j = cand_start[i]; j < cand_start[i + 1]; ++j) {
            const int64_t k = cand[j];
            if (k < 0 || k >= K) { free(f32); free(f64); return ORACLE_EINVAL; }
            const double* ctr = centres + k * width;
            int inside = 1;
            for (int d = 0; d < g.n; ++d) inside = inside && in_window(&g, d, x[d], ctr[g.C + d]);
            if (!inside) continue;
            if (g.fp64) {
                double D = dist64(&g, f64, x, ctr);
                if (D < bd64 || (D == bd64 && k < best)) { bd64 = D; best = (int32_t)k; }
            } else {
                float D = dist32(&g, f32, x, ctr);
                if (D < bd32 || (D == bd32 && k < best)) { bd32 = D; best = (int32_t)k; }
            }
        }
        labels_out[i] = best;
    }
    free(f32); free(f64);
    return ORACLE_OK;
}

/* ---- update (Sec. 2.2 "Update clusters", Sec. 3.1 map-reduce; R9, R10) --- */

/* map: accumulate [I(x), x] of the voxels qlo .. qhi-1 per label */
static int update_map(const geom* g, const void* image, const int32_t* labels, int64_t K, int64_t qlo,
                      int64_t qhi, int64_t* cnt, int64_t* isum, double* fsum)
{
    const int width = g->C + g->n;
    for (int64_t q = qlo; q < qhi; ++q) {
        int32_t k = labels[q];
        if (k < 0) continue; /* R8 */
        if (k >= K) return ORACLE_EINVAL;
        int64_t x[ND];
        coords(g, q, x);
        cnt[k] += 1;
        for (int c = 0; c < g->C; ++c) {
            if (g->dt == ORACLE_F32) fsum[k * g->C + c] += pix(g, image, q, c);
            else isum[k * width + c] += pix_int(g, image, q, c);
        }
        for (int d = 0; d < g->n; ++d) isum[k * width + g->C + d] += x[d];
    }
    return ORACLE_OK;
}

/* reduce, one cluster: its new centre as the member mean (an empty cluster
 * keeps its centre); returns the cluster's residual term sqrt(D^2(C_prev,
 * C_new)), or -1 when it is empty */
static double update_divide(const geom* g, int64_t k, const int64_t* cnt, const int64_t* isum,
                            const double* fsum, double* centres)
{
    const int width = g->C + g->n;
    double* row = centres + k * width;
    if (cnt[k] == 0) return -1.0;
    double n = (double)cnt[k];
    double D2 = 0.0;
    for (int j = 0; j < width; ++j) {
        double s = (j < g->C && g->dt == ORACLE_F32) ? fsum[k * g->C + j]
                                                      : (double)isum[k * width + j];
        double mean = s / n;
        double v = g->fp64 ? mean : (double)(float)mean;
        double diff = v - row[j];
        D2 += (j < g->C) ? diff * diff : g->w64[j - g->C] * (diff * diff);
        row[j] = v;
    }
    return sqrt(D2);
}

static int update(const geom* g, const void* image, const int32_t* labels, int64_t K,
                  double* centres, int64_t* counts_out, double* residual)
{
    const int width = g->C + g->n;
    int64_t* cnt = (int64_t*)calloc((size_t)K, sizeof(int64_t));
    int64_t* isum = (int64_t*)calloc((size_t)K * width, sizeof(int64_t));
    double* fsum = (double*)calloc((size_t)K * g->C, sizeof(double));
    if (!cnt || !isum || !fsum) {
        free(cnt); free(isum); free(fsum);
        return ORACLE_ENOMEM;
    }
    int rc = update_map(g, image, labels, K, 0, g->V, cnt, isum, fsum);
    if (rc != ORACLE_OK) { free(cnt); free(isum); free(fsum); return rc; }
    /* reduce: divide, keep empty clusters unchanged */
    double rsum = 0.0;
    int64_t nonempty = 0;
    for (int64_t k = 0; k < K; ++k) {
        if (counts_out) counts_out[k] = cnt[k];
        double t = update_divide(g, k, cnt, isum, fsum, centres);
        if (t < 0.0) continue;
        rsum += t;
        nonempty += 1;
    }
    if (residual) *residual = nonempty ? rsum / (double)nonempty : 0.0;
    free(cnt); free(isum); free(fsum);
    return ORACLE_OK;
}

int oracle_update(const oracle_params* p, const void* image, const int32_t* labels,
                  int64_t K, double* centres, int64_t* counts, double* residual)
{
    geom g;
    int rc = make_geom(p, &g);
    if (rc != ORACLE_OK) return rc;
    if (!image || !labels || !centres || K < 0) return ORACLE_EINVAL;
    return update(&g, image, labels, K, centres, counts, residual);
}

/* ---- connectivity enforcement (Sec. 3.1 stage 3; R11-R15) --------------- */

/* Flood fill of the face-connected component of label lab containing s, on
 * the pre-relabel image.  Visited voxels are marked in vis; the component's
 * voxels are left in queue[0..return). */
static int64_t flood(const geom* g, const int32_t* lab_in, int64_t s, int32_t lab,
                     uint8_t* vis, int64_t* queue)
{
    int64_t head = 0, tail = 0;
    queue[tail++] = s;
    vis[s] = 1;
    while (head < tail) {
        int64_t q = queue[head++];
        int64_t x[ND];
        coords(g, q, x);
        for (int d = 0; d < g->n; ++d) {
            if (x[d] > 0) {
                int64_t r = q - g->stride[d];
                if (!vis[r] && lab_in[r] == lab) { vis[r] = 1; queue[tail++] = r; }
            }
            if (x[d] + 1 < g->N[d]) {
                int64_t r = q + g->stride[d];
                if (!vis[r] && lab_in[r] == lab) { vis[r] = 1; queue[tail++] = r; }
            }
        }
    }
    return tail;
}

static int connectivity(const geom* g, const double* centres, int64_t K,
                        const int32_t* lab_in, int32_t* out, int64_t* num_labels)
{
    const int width = g->C + g->n;
    int64_t sprod = 1;
    for (int d = 0; d < g->n; ++d) sprod *= g->S[d];
    uint8_t* fin = (uint8_t*)calloc((size_t)g->V, 1);   /* marker image m */
    uint8_t* vis = (uint8_t*)calloc((size_t)g->V, 1);
    int64_t* queue = (int64_t*)malloc((size_t)g->V * sizeof(int64_t));
    if (!fin || !vis || !queue) {
        free(fin); free(vis); free(queue);
        return ORACLE_ENOMEM;
    }
    memcpy(out, lab_in, (size_t)g->V * sizeof(int32_t));

    /* phase 1: one component per centre, final if large enough (R12) */
    for (int64_t k = 0; k < K; ++k) {
        const double* ctr = centres + k * width;
        int64_t p[ND] = {0};
        for (int d = 0; d < g->n; ++d) {
            int64_t v = (int64_t)floor(ctr[g->C + d] + 0.5);
            if (v < 0) v = 0;
            if (v > g->N[d] - 1) v = g->N[d] - 1;
            p[d] = v;
        }
        int64_t s = -1;
        int64_t pq = index_of(g, p);
        if (lab_in[pq] == (int32_t)k) {
            s = pq;
        } else {
            int64_t lo[ND], hi[ND], xx[ND];
            for (int d = 0; d < ND; ++d) {
                lo[d] = p[d] - g->S[d] / 2;
                hi[d] = p[d] + (g->S[d] + 1) / 2 - 1;
                if (lo[d] < 0) lo[d] = 0;
                if (hi[d] > g->N[d] - 1) hi[d] = g->N[d] - 1;
            }
            for (int more = box_first(xx, lo, hi); more && s < 0; more = box_next(xx, lo, hi)) {
                int64_t q = index_of(g, xx);
                if (lab_in[q] == (int32_t)k) s = q;
            }
        }
        if (s < 0) continue;
        int64_t size = flood(g, lab_in, s, (int32_t)k, vis, queue);
        int final = 4 * size > sprod;
        for (int64_t i = 0; i < size; ++i) {
            vis[queue[i]] = 0;
            if (final) fin[queue[i]] = 1;
        }
    }

    /* phase 2: raster scan over non-final voxels (R13, R14) */
    int64_t next = K;
    for (int64_t q = 0; q < g->V; ++q) {
        if (fin[q]) continue;
        int64_t size = flood(g, lab_in, q, lab_in[q], vis, queue);
        int32_t newlab;
        if (4 * size > sprod || q == 0) {
            newlab = (int32_t)next++;
        } else {
            int64_t x[ND];
            coords(g, q, x);
            int d = 0;
            while (x[d] == 0) ++d;
            newlab = out[q - g->stride[d]];
        }
        for (int64_t i = 0; i < size; ++i) {
            out[queue[i]] = newlab;
            fin[queue[i]] = 1;
            vis[queue[i]] = 0;
        }
    }
    if (num_labels) *num_labels = next;
    free(fin); free(vis); free(queue);
    return ORACLE_OK;
}

int oracle_connectivity(const oracle_params* p, const double* centres, int64_t K,
                        const int32_t* labels_in, int32_t* labels_out, int64_t* num_labels)
{
    geom g;
    int rc = make_geom(p, &g);
    if (rc != ORACLE_OK) return rc;
    if (!centres || !labels_in || !labels_out || K < 0 || K > 0x7fffffffLL) return ORACLE_EINVAL;
    return connectivity(&g, centres, K, labels_in, labels_out, num_labels);
}

/* ---- region decomposition (Sec. 3.1, "Create non-overlapping regions") --
 * The paper's multi-threaded form: the image is split into non-overlapping
 * regions, here ranges of planes along the last axis; each thread assigns
 * the voxels of its region, visiting every centre whose window meets the
 * region in ascending k (so every voxel sees the centres in the same order
 * as in assign() and keeps the same label), then maps its region's voxels
 * into per-region sums that a reduce merges per label.  Integer sums are
 * exact, so the merged sums -- and the centres -- equal the sequential
 * ones; float images keep the sequential map (their double sums are then
 * added in the same raster order).  Connectivity stays sequential: its
 * raster pass is the paper's largest single-threaded part (Sec. 4).
 * Compiled with -fopenmp the regions run on `threads` threads; without it
 * the pragmas are ignored and the regions run one after another. */
static void region_planes(const geom* g, int nreg, int r, int64_t* plo, int64_t* phi)
{
    const int64_t NL = g->N[g->n - 1];
    *plo = NL * r / nreg;
    *phi = NL * (r + 1) / nreg;
}

static int assign_regions(const geom* g, const void* image, const double* centres, int64_t K,
                          int32_t* labels, int nreg, int threads)
{
    int rc_all = ORACLE_OK;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
    for (int r = 0; r < nreg; ++r) {
        int64_t plo, phi;
        region_planes(g, nreg, r, &plo, &phi);
        int rc = assign_planes(g, image, centres, K, labels, plo, phi);
        if (rc != ORACLE_OK) {
#pragma omp critical
            rc_all = rc;
        }
    }
    return rc_all;
}

static int update_regions(const geom* g, const void* image, const int32_t* labels, int64_t K,
                          double* centres, double* residual, int nreg, int threads)
{
    if (g->dt == ORACLE_F32) return update(g, image, labels, K, centres, NULL, residual);
    const int width = g->C + g->n;
    const int last = g->n - 1;
    int64_t* cnt = (int64_t*)calloc((size_t)(nreg * K), sizeof(int64_t));
    int64_t* isum = (int64_t*)calloc((size_t)(nreg * K * width), sizeof(int64_t));
    double* term = (double*)malloc((size_t)(K > 0 ? K : 1) * sizeof(double));
    if (!cnt || !isum || !term) {
        free(cnt); free(isum); free(term);
        return ORACLE_ENOMEM;
    }
    int rc_all = ORACLE_OK;
    /* map, per region */
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
    for (int r = 0; r < nreg; ++r) {
        int64_t plo, phi;
        region_planes(g, nreg, r, &plo, &phi);
        int rc = update_map(g, image, labels, K, plo * g->stride[last], phi * g->stride[last], cnt + r * K,
                            isum + r * K * width, NULL);
        if (rc != ORACLE_OK) {
#pragma omp critical
            rc_all = rc;
        }
    }
    if (rc_all == ORACLE_OK) {
        /* reduce per label, then divide */
#pragma omp parallel for schedule(static) num_threads(threads)
        for (int64_t k = 0; k < K; ++k) {
            for (int r = 1; r < nreg; ++r) {
                cnt[k] += cnt[r * K + k];
                for (int j = 0; j < width; ++j) isum[k * width + j] += isum[(r * K + k) * width + j];
            }
            term[k] = update_divide(g, k, cnt, isum, NULL, centres);
        }
        /* the residual's sum in ascending k, as in update() */
        double rsum = 0.0;
        int64_t nonempty = 0;
        for (int64_t k = 0; k < K; ++k) {
            if (term[k] < 0.0) continue;
            rsum += term[k];
            nonempty += 1;
        }
        if (residual) *residual = nonempty ? rsum / (double)nonempty : 0.0;
    }
    free(cnt); free(isum); free(term);
    return rc_all;
}

int oracle_threads_available(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int oracle_slic_regions(const oracle_params* p, const void* image, int32_t* labels, double* centres_out,
                        int32_t* iters_done, double* residual, int64_t* num_labels, int threads)
{
    geom g;
    int rc = make_geom(p, &g);
    if (rc != ORACLE_OK) return rc;
    if (!image || !labels || threads < 1) return ORACLE_EINVAL;
    const int width = g.C + g.n;
    /* several regions per thread, so that uneven regions balance */
    int64_t nreg64 = 4 * (int64_t)threads;
    if (nreg64 > g.N[g.n - 1]) nreg64 = g.N[g.n - 1];
    const int nreg = (int)nreg64;
    double* ctr = (double*)malloc((size_t)(g.K * width) * sizeof(double));
    if (!ctr) return ORACLE_ENOMEM;
    rc = seed(&g, p->perturb, image, ctr);
    int32_t it = 0;
    double res = 0.0;
    for (it = 0; rc == ORACLE_OK && it < p->max_iter; ++it) {
        rc = assign_regions(&g, image, ctr, g.K, labels, nreg, threads);
        if (rc == ORACLE_OK) rc = update_regions(&g, image, labels, g.K, ctr, &res, nreg, threads);
        if (rc == ORACLE_OK && p->conv_threshold > 0.0 && res < p->conv_threshold) { ++it; break; }
    }
    if (rc == ORACLE_OK) {
        if (iters_done) *iters_done = it;
        if (residual) *residual = res;
        if (centres_out) memcpy(centres_out, ctr, (size_t)(g.K * width) * sizeof(double));
        if (p->enforce_connectivity) {
            int32_t* tmp = (int32_t*)malloc((size_t)g.V * sizeof(int32_t));
            if (!tmp) rc = ORACLE_ENOMEM;
            else {
                memcpy(tmp, labels, (size_t)g.V * sizeof(int32_t));
                rc = connectivity(&g, ctr, g.K, tmp, labels, num_labels);
                free(tmp);
            }
        } else if (num_labels) {
            *num_labels = g.K;
        }
    }
    free(ctr);
    return rc;
}

/* ---- CIE-Lab conversion (R16) -------------------------------------------- */

/* sRGB code value (0..255) -> linear light */
static double srgb_linear(int code)
{
    const double v = code / 255.0;
    return v <= 0.04045 ? v / 12.92 : pow((v + 0.055) / 1.055, 2.4);
}

/* CIE 1976 companding: cube root above (6/29)^3, the tangent line below */
static double lab_f(double t)
{
    const double d = 6.0 / 29.0;
    return t > d * d * d ? cbrt(t) : t / (3.0 * d * d) + 4.0 / 29.0;
}

int oracle_srgb_to_lab(const uint8_t* rgb, int64_t n, double* lab)
{
    static const double M[3][3] = {{0.4124, 0.3576, 0.1805},
                                   {0.2126, 0.7152, 0.0722},
                                   {0.0193, 0.1192, 0.9505}};
    static const double W[3] = {0.95047, 1.0, 1.08883};
    if (n < 0 || (n > 0 && (!rgb || !lab))) return ORACLE_EINVAL;
    for (int64_t i = 0; i < n; ++i) {
        const double r = srgb_linear(rgb[3 * i]), gr = srgb_linear(rgb[3 * i + 1]),
                     b = srgb_linear(rgb[3 * i + 2]);
        double f[3];
        for (int j = 0; j < 3; ++j) f[j] = lab_f((M[j][0] * r + M[j][1] * gr + M[j][2] * b) / W[j]);
        lab[3 * i] = 116.0 * f[1] - 16.0;
        lab[3 * i + 1] = 500.0 * (f[0] - f[1]);
        lab[3 * i + 2] = 200.0 * (f[1] - f[2]);
    }
    return ORACLE_OK;
}

/* ---- whole method -------------------------------------------------------- */

static int run(const geom* g, const oracle_params* p, const void* image, double* ctr,
               int32_t* labels, double* centres_out, int32_t* iters_done,
               double* residual, int64_t* num_labels)
{
    const int width = g->C + g->n;
    int32_t it = 0;
    double res = 0.0;
    int rc = ORACLE_OK;
    for (it = 0; it < p->max_iter; ++it) {
        rc = assign(g, image, ctr, g->K, labels);
        if (rc != ORACLE_OK) return rc;
        rc = update(g, image, labels, g->K, ctr, NULL, &res);
        if (rc != ORACLE_OK) return rc;
        if (p->conv_threshold > 0.0 && res < p->conv_threshold) { ++it; break; }
    }
    if (iters_done) *iters_done = it;
    if (residual) *residual = res;
    if (centres_out) memcpy(centres_out, ctr, (size_t)(g->K * width) * sizeof(double));
    if (p->enforce_connectivity) {
        int32_t* tmp = (int32_t*)malloc((size_t)g->V * sizeof(int32_t));
        if (!tmp) return ORACLE_ENOMEM;
        memcpy(tmp, labels, (size_t)g->V * sizeof(int32_t));
        rc = connectivity(g, ctr, g->K, tmp, labels, num_labels);
        free(tmp);
    } else if (num_labels) {
        *num_labels = g->K;
    }
    return rc;
}

int oracle_slic(const oracle_params* p, const void* image, int32_t* labels,
                double* centres_out, int32_t* iters_done, double* residual,
                int64_t* num_labels)
{
    geom g;
    int rc = make_geom(p, &g);
    if (rc != ORACLE_OK) return rc;
    if (!image || !labels) return ORACLE_EINVAL;
    double* ctr = (double*)malloc((size_t)(g.K * (g.C + g.n)) * sizeof(double));
    if (!ctr) return ORACLE_ENOMEM;
    rc = seed(&g, p->perturb, image, ctr);
    if (rc == ORACLE_OK)
        rc = run(&g, p, image, ctr, labels, centres_out, iters_done, residual, num_labels);
    free(ctr);
    return rc;
}

int oracle_slic_from(const oracle_params* p, const void* image, const double* init_centres,
                     int32_t* labels, double* centres_out, int32_t* iters_done,
                     double* residual, int64_t* num_labels)
{
    geom g;
    int rc = make_geom(p, &g);
    if (rc != ORACLE_OK) return rc;
    if (!image || !labels || !init_centres) return ORACLE_EINVAL;
    size_t n = (size_t)(g.K * (g.C + g.n));
    double* ctr = (double*)malloc(n * sizeof(double));
    if (!ctr) return ORACLE_ENOMEM;
    memcpy(ctr, init_centres, n * sizeof(double));
    if (!g.fp64)
        for (size_t i = 0; i < n; ++i) ctr[i] = (double)(float)ctr[i];
    rc = run(&g, p, image, ctr, labels, centres_out, iters_done, residual, num_labels);
    free(ctr);
    return rc;
}
