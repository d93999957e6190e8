/*
 * gamma_oracle.c -- plain, slow, FP64 CPU oracle for the gamma index.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (paper Section 2.1, Eq. 1): for every reference voxel r_r
 * that passes the low-dose cutoff,
 *     gamma(r_r) = min over points r_e of the evaluation surface of
 *                  | (r_r/dta, D_r(r_r)/dD) - (r_e/dta, D_e(r_e)/dD) |,
 * where the evaluation surface is the continuous surface spanned by the
 * evaluation dose points (the geometric method the paper adopts from Ju et
 * al.): the graph of the piecewise-linear interpolant of D_e over the
 * Freudenthal (Kuhn) triangulation of the grid, i.e. each grid cube with
 * lower corner p is split into n! simplices p -> p+e_s1 -> p+e_s1+e_s2 -> ...
 * for every permutation s of the axes.
 *
 * How (Algorithm A1, in its order):
 *   1. the maximum over reference voxels of DD/dD, with DD = |D_e - D_r| at the
 *      same voxel (step 1; the sign is lost in the printed text, the absolute
 *      value is needed for the initial bound of step 4a to be a distance);
 *   2. the set of geometric distances L_n of grid cubes around a reference
 *      voxel within that maximum radius (step 2);
 *   3. that set sorted ascending (step 3);
 *   4. per reference voxel: gamma = DD/dD (step 4a); walk the sorted cubes;
 *      stop once L_n reaches the running gamma (step 4b-ii); otherwise take
 *      the distance to each of the cube's closed simplices (step 4b-i) and
 *      keep the minimum (step 4b-iii).
 * The distance to a closed simplex follows the paper's normal equations,
 * omega = (V^T V)^-1 V^T P with omega_{k+1} = 1 - sum(omega), recursing into
 * the sub-simplices opposite the vertices whose weight is negative (Ju et al.
 * recursion, Section 2.1).
 *
 * Readings taken where the paper is silent or garbled:
 *   - L_n of a cube is the distance from the reference voxel to the closed
 *     cube box, divided by dta.  Every simplex of the cube lies in the box, so
 *     its distance is >= L_n and "stop when L_n >= gamma" is exact.  (The
 *     printed break test compares Gamma with L_n, which is not a valid stop.)
 *   - The table is truncated at a cap on its length; a voxel whose walk runs
 *     past the end with gamma still above the truncation radius finishes with
 *     a plain scan of every cube in its search box.  Exact either way.
 *   - Global mode: dD = dd_frac * D_norm, D_norm = dose_norm if > 0 else
 *     max(D_r).  Local mode: dD(v) = dd_frac * D_r(v).
 *   - A reference voxel is evaluated iff D_r(v) >= cutoff_frac * D_norm (and,
 *     in local mode, D_r(v) > 0), compared in float32.  Others get NaN.
 *   - Simplices with a vertex outside the grid do not exist (no
 *     extrapolation).  Every axis of the problem needs >= 2 voxels.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXD 4            /* ambient dimension n + 1 <= 4; a simplex has <= 5 vertices */

typedef struct {
    int i, j, k;             /* lower-corner offset of the cube, voxel units */
    double key;              /* L_n: distance to the cube box / dta */
} or_cell;

typedef struct {
    int ndim;
    int64_t nz, ny, nx;
    double hz, hy, hx;
    double dta, dd_frac, cutoff_frac, dose_norm;
    int local;
    const float *ref, *ev;
    double d_norm;           /* resolved */
    double r_max;            /* max gamma0 over evaluated voxels */
    or_cell *table;
    int64_t ntable;
    double r_cover;          /* every cube with key < r_cover is in the table */
    int perms[6][3];
    int nperm;
} or_ctx;

/* ------------------------------------------------------------------------ */
/* Distance from P to the closed simplex with vertices W[0..nv-1] in R^K.   */
/* ------------------------------------------------------------------------ */

static int or_cholesky_solve(int k, double G[OR_MAXD][OR_MAXD], const double *rhs, double *x)
{
    double L[OR_MAXD][OR_MAXD] = {{0}};
    for (int r = 0; r < k; ++r) {
        for (int c = 0; c <= r; ++c) {
            double s = G[r][c];
            for (int t = 0; t < c; ++t) s -= L[r][t] * L[c][t];
            if (r == c) {
                if (!(s > 1e-300)) return 0;
                L[r][r] = sqrt(s);
            } else {
                L[r][c] = s / L[c][c];
            }
        }
    }
    double y[OR_MAXD];
    for (int r = 0; r < k; ++r) {
        double s = rhs[r];
        for (int t = 0; t < r; ++t) s -= L[r][t] * y[t];
        y[r] = s / L[r][r];
    }
    for (int r = k - 1; r >= 0; --r) {
        double s = y[r];
        for (int t = r + 1; t < k; ++t) s -= L[t][r] * x[t];
        x[r] = s / L[r][r];
    }
    return 1;
}

double oracle_simplex_distance(int K, int nv, const double *W, const double *P)
{
    if (nv == 1) {
        double s = 0;
        for (int r = 0; r < K; ++r) { double d = P[r] - W[r]; s += d * d; }
        return sqrt(s);
    }
    const int k = nv - 1;                 /* base vertex: the last one */
    const double *base = W + (size_t)k * K;
    double V[OR_MAXD][OR_MAXD], b[OR_MAXD];
    for (int r = 0; r < K; ++r) {
        b[r] = P[r] - base[r];
        for (int c = 0; c < k; ++c) V[r][c] = W[(size_t)c * K + r] - base[r];
    }
    double G[OR_MAXD][OR_MAXD], rhs[OR_MAXD], w[OR_MAXD + 1];
    for (int a = 0; a < k; ++a) {
        rhs[a] = 0;
        for (int r = 0; r < K; ++r) rhs[a] += V[r][a] * b[r];
        for (int c = 0; c < k; ++c) {
            double s = 0;
            for (int r = 0; r < K; ++r) s += V[r][a] * V[r][c];
            G[a][c] = s;
        }
    }
    int ok = or_cholesky_solve(k, G, rhs, w);
    if (ok) {
        double sum = 0;
        int inside = 1;
        for (int a = 0; a < k; ++a) { sum += w[a]; if (w[a] < 0) inside = 0; }
        w[k] = 1.0 - sum;
        if (w[k] < 0) inside = 0;
        if (inside) {
            double s = 0;
            for (int r = 0; r < K; ++r) {
                double res = b[r];
                for (int c = 0; c < k; ++c) res -= V[r][c] * w[c];
                s += res * res;
            }
            return sqrt(s);
        }
    }
    /* Recurse into the facets opposite the negative weights (all facets if
     * the simplex is degenerate). */
    double best = INFINITY;
    double F[(OR_MAXD + 1) * OR_MAXD];
    for (int drop = 0; drop <= k; ++drop) {
        if (ok && !(w[drop] < 0)) continue;
        int t = 0;
        for (int v = 0; v <= k; ++v) {
            if (v == drop) continue;
            memcpy(F + (size_t)t * K, W + (size_t)v * K, sizeof(double) * K);
            ++t;
        }
        double d = oracle_simplex_distance(K, k, F, P);
        if (d < best) best = d;
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* Cell table (Algorithm A1, steps 2-3).                                     */
/* ------------------------------------------------------------------------ */

static double or_axis_gap(int i) { return i >= 0 ? (double)i : (double)(-i - 1); }

static double or_key(const or_ctx *c, int i, int j, int k)
{
    double ax = or_axis_gap(i) * c->hx, ay = or_axis_gap(j) * c->hy;
    double az = c->ndim == 3 ? or_axis_gap(k) * c->hz : 0.0;
    return sqrt(ax * ax + ay * ay + az * az) / c->dta;
}

static int or_cmp_cell(const void *pa, const void *pb)
{
    const or_cell *a = (const or_cell *)pa, *b = (const or_cell *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    if (a->k != b->k) return a->k < b->k ? -1 : 1;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    if (a->i != b->i) return a->i < b->i ? -1 : 1;
    return 0;
}

/* Offsets along one axis whose cube can hold a grid cube for some voxel:
 * corner p = v + off with 0 <= p <= n - 2, so -(n - 1) <= off <= n - 2. */
static void or_axis_range(double radius, double dta, double h, int64_t n,
                          int64_t *lo, int64_t *hi)
{
    int64_t lim = (int64_t)ceil(radius * dta / h) + 1;
    *lo = -(n - 1) > -lim - 1 ? -(n - 1) : -lim - 1;
    *hi = n - 2 < lim ? n - 2 : lim;
}

/* Build every cube offset with key < radius (restricted to offsets that can
 * fall inside the grid), sorted.  With cap > 0 the enumeration radius is
 * first lowered until a ball-volume estimate holds about 4 * cap cubes, and
 * the sorted list is cut to cap entries; r_cover records the radius below
 * which the table is complete (the key of the first entry cut). */
static int or_build_table(or_ctx *c, double radius, int64_t cap)
{
    c->table = NULL;
    c->ntable = 0;
    c->r_cover = radius;
    if (!(radius > 0)) return 0;
    if (cap > 0) {
        double cell_vol = (c->hx / c->dta) * (c->hy / c->dta) *
                          (c->ndim == 3 ? c->hz / c->dta : 1.0);
        for (;;) {
            double r = radius;
            double ball = c->ndim == 3 ? 4.18879020478639 * r * r * r : 3.14159265358979 * r * r;
            if (ball / cell_vol < 4.0 * (double)cap + 64.0) break;
            radius *= 0.8;
        }
        c->r_cover = radius;
    }
    int64_t x0, x1, y0, y1, z0 = 0, z1 = 0;
    or_axis_range(radius, c->dta, c->hx, c->nx, &x0, &x1);
    or_axis_range(radius, c->dta, c->hy, c->ny, &y0, &y1);
    if (c->ndim == 3) or_axis_range(radius, c->dta, c->hz, c->nz, &z0, &z1);
    if (x1 < x0 || y1 < y0 || z1 < z0) return 0;
    int64_t cnt = 0, alloc = 1024;
    or_cell *t = (or_cell *)malloc(sizeof(or_cell) * alloc);
    if (!t) return -1;
    for (int64_t k = z0; k <= z1; ++k)
        for (int64_t j = y0; j <= y1; ++j)
            for (int64_t i = x0; i <= x1; ++i) {
                double key = or_key(c, (int)i, (int)j, (int)k);
                if (!(key < radius)) continue;
                if (cnt == alloc) {
                    alloc *= 2;
                    or_cell *nt = (or_cell *)realloc(t, sizeof(or_cell) * alloc);
                    if (!nt) { free(t); return -1; }
                    t = nt;
                }
                t[cnt].i = (int)i; t[cnt].j = (int)j; t[cnt].k = (int)k; t[cnt].key = key;
                ++cnt;
            }
    qsort(t, (size_t)cnt, sizeof(or_cell), or_cmp_cell);
    if (cap > 0 && cnt > cap) {
        c->r_cover = t[cap].key;
        cnt = cap;
    }
    c->table = t;
    c->ntable = cnt;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Per-voxel search (Algorithm A1, step 4).                                  */
/* ------------------------------------------------------------------------ */

static double or_delta_dose(const or_ctx *c, double dr)
{
    return c->local ? c->dd_frac * dr : c->dd_frac * c->d_norm;
}

/* The evaluated / not-evaluated decision is an integer outcome of floating
 * point; it is taken in single precision, threshold = float(cutoff_frac) *
 * float(D_norm) rounded to float, so that every implementation fed the same
 * float32 doses and criteria decides it identically. */
static int or_evaluated(const or_ctx *c, double dr)
{
    const float thr = (float)c->cutoff_frac * (float)c->d_norm;
    if (!((float)dr >= thr)) return 0;
    if (c->local && !(dr > 0)) return 0;
    return 1;
}

static void or_make_perms(or_ctx *c)
{
    if (c->ndim == 2) {
        int p[2][3] = {{0, 1, -1}, {1, 0, -1}};
        memcpy(c->perms, p, sizeof(p));
        c->nperm = 2;
    } else {
        int p[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
        memcpy(c->perms, p, sizeof(p));
        c->nperm = 6;
    }
}

/* Distance from point P (normalised) to the closed simplices of the cube with
 * lower corner (px,py,pz); the caller guarantees the whole cube is inside. */
static double or_cube_distance(const or_ctx *c, int64_t px, int64_t py, int64_t pz,
                               double inv_dd, const double *P, double best)
{
    const int n = c->ndim, K = n + 1;
    for (int s = 0; s < c->nperm; ++s) {
        double W[4 * OR_MAXD];
        int64_t q[3] = {px, py, pz};
        for (int v = 0; v <= n; ++v) {
            if (v > 0) q[c->perms[s][v - 1]] += 1;   /* axis 0 = x, 1 = y, 2 = z */
            int64_t lin = (q[2] * c->ny + q[1]) * c->nx + q[0];
            double *w = W + (size_t)v * K;
            w[0] = (double)q[0] * c->hx / c->dta;
            w[1] = (double)q[1] * c->hy / c->dta;
            if (n == 3) w[2] = (double)q[2] * c->hz / c->dta;
            w[n] = (double)c->ev[lin] * inv_dd;
        }
        double d = oracle_simplex_distance(K, n + 1, W, P);
        if (d < best) best = d;
    }
    return best;
}

static int or_cube_inside(const or_ctx *c, int64_t px, int64_t py, int64_t pz)
{
    if (px < 0 || py < 0 || px > c->nx - 2 || py > c->ny - 2) return 0;
    if (c->ndim == 3 && (pz < 0 || pz > c->nz - 2)) return 0;
    return 1;
}

static double or_gamma_voxel(const or_ctx *c, int64_t v, int64_t *cells_out)
{
    const int64_t x = v % c->nx, y = (v / c->nx) % c->ny, z = v / (c->nx * c->ny);
    const double dr = (double)c->ref[v];
    int64_t cells = 0;
    if (!or_evaluated(c, dr)) { if (cells_out) *cells_out = 0; return NAN; }
    const double ddose = or_delta_dose(c, dr), inv_dd = 1.0 / ddose;
    double P[OR_MAXD];
    P[0] = (double)x * c->hx / c->dta;
    P[1] = (double)y * c->hy / c->dta;
    if (c->ndim == 3) P[2] = (double)z * c->hz / c->dta;
    P[c->ndim] = dr * inv_dd;
    double g = fabs((double)c->ev[v] - dr) * inv_dd;           /* step 4a */
    int64_t t;
    for (t = 0; t < c->ntable; ++t) {                           /* step 4b */
        const or_cell *e = &c->table[t];
        if (e->key >= g) break;                                 /* 4b-ii */
        int64_t px = x + e->i, py = y + e->j, pz = z + e->k;
        if (!or_cube_inside(c, px, py, pz)) continue;
        ++cells;
        g = or_cube_distance(c, px, py, pz, inv_dd, P, g);      /* 4b-i, 4b-iii */
    }
    if (t == c->ntable && g > c->r_cover) {
        /* Walk ran past a truncated table: scan the rest of the search box. */
        int64_t ax = (int64_t)ceil(g * c->dta / c->hx) + 1;
        int64_t ay = (int64_t)ceil(g * c->dta / c->hy) + 1;
        int64_t az = c->ndim == 3 ? (int64_t)ceil(g * c->dta / c->hz) + 1 : 0;
        for (int64_t k = -az - 1; k <= az; ++k) {
            if (c->ndim == 2 && k != 0) continue;
            for (int64_t j = -ay - 1; j <= ay; ++j)
                for (int64_t i = -ax - 1; i <= ax; ++i) {
                    double key = or_key(c, (int)i, (int)j, (int)k);
                    if (key < c->r_cover || !(key < g)) continue;
                    int64_t px = x + i, py = y + j, pz = z + k;
                    if (!or_cube_inside(c, px, py, pz)) continue;
                    ++cells;
                    g = or_cube_distance(c, px, py, pz, inv_dd, P, g);
                }
        }
    }
    if (cells_out) *cells_out = cells;
    return g;
}

static int or_setup(or_ctx *c, const float *ref, const float *ev, int ndim,
                    const int64_t shape[3], const double spacing[3], double dd_frac,
                    double dta_mm, int local, double cutoff_frac, double dose_norm)
{
    memset(c, 0, sizeof(*c));
    if (ndim != 2 && ndim != 3) return -1;
    c->ndim = ndim;
    c->nz = ndim == 3 ? shape[0] : 1;
    c->ny = shape[1];
    c->nx = shape[2];
    c->hz = spacing[0]; c->hy = spacing[1]; c->hx = spacing[2];
    if (c->nx < 2 || c->ny < 2 || (ndim == 3 && c->nz < 2)) return -2;
    if (!(dta_mm > 0) || !(dd_frac > 0) || !(c->hx > 0) || !(c->hy > 0) ||
        (ndim == 3 && !(c->hz > 0)))
        return -1;
    c->dta = dta_mm; c->dd_frac = dd_frac; c->local = local;
    c->cutoff_frac = cutoff_frac; c->dose_norm = dose_norm;
    c->ref = ref; c->ev = ev;
    const int64_t N = c->nz * c->ny * c->nx;
    double m = -INFINITY;
    for (int64_t v = 0; v < N; ++v) {
        if (!isfinite(ref[v]) || !isfinite(ev[v])) return -3;
        if (ref[v] > m) m = ref[v];
    }
    c->d_norm = dose_norm > 0 ? dose_norm : m;
    if (!local && !(c->d_norm > 0)) return -1;
    double rmax = 0;                                            /* step 1 */
    for (int64_t v = 0; v < N; ++v) {
        double dr = ref[v];
        if (!or_evaluated(c, dr)) continue;
        double g0 = fabs((double)ev[v] - dr) / or_delta_dose(c, dr);
        if (g0 > rmax) rmax = g0;
    }
    c->r_max = rmax;
    or_make_perms(c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points                                                     */
/* ------------------------------------------------------------------------ */

/* Gamma for the voxels listed in idx (all voxels when idx == NULL).
 * ref/ev: float32 C-order (z, y, x) grids (2D: shape[0] is ignored, 1 slice).
 * spacing: mm in (z, y, x) order.  gamma_out[t] is gamma of voxel idx[t],
 * NaN when not evaluated.  cells_out (optional): cubes processed per voxel.
 * table_cap: maximum table length (<= 0: unlimited).  threads <= 0: OpenMP
 * default.  Returns 0, or a negative code for bad arguments (-1), a bad
 * shape (-2), non-finite input (-3), out of memory (-4). */
int oracle_gamma(const float *ref, const float *ev, int ndim, const int64_t shape[3],
                 const double spacing[3], double dd_frac, double dta_mm, int local,
                 double cutoff_frac, double dose_norm, const int64_t *idx, int64_t nidx,
                 double *gamma_out, int64_t *cells_out, int64_t table_cap, int threads,
                 double *r_max_out)
{
    or_ctx c;
    int rc = or_setup(&c, ref, ev, ndim, shape, spacing, dd_frac, dta_mm, local,
                      cutoff_frac, dose_norm);
    if (rc) return rc;
    if (or_build_table(&c, c.r_max, table_cap)) return -4;   /* steps 2-3 */
    const int64_t N = c.nz * c.ny * c.nx;
    const int64_t n = idx ? nidx : N;
    if (r_max_out) *r_max_out = c.r_max;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
    for (int64_t t = 0; t < n; ++t) {
        int64_t v = idx ? idx[t] : t;
        if (v < 0 || v >= N) { bad |= 1; gamma_out[t] = NAN; continue; }
        int64_t cells = 0;
        gamma_out[t] = or_gamma_voxel(&c, v, &cells);
        if (cells_out) cells_out[t] = cells;
    }
    free(c.table);
    return bad ? -1 : 0;
}

/* The sorted cube table for the given geometry and radius: offsets (x, y, z
 * per entry, voxel units) and keys.  Returns the number of entries, or the
 * count needed when it exceeds max_entries (nothing written then). */
int64_t oracle_cell_table(int ndim, const int64_t shape[3], const double spacing[3],
                          double dta_mm, double radius, int32_t *offsets, double *keys,
                          int64_t max_entries)
{
    or_ctx c;
    memset(&c, 0, sizeof(c));
    c.ndim = ndim;
    c.nz = ndim == 3 ? shape[0] : 1; c.ny = shape[1]; c.nx = shape[2];
    c.hz = spacing[0]; c.hy = spacing[1]; c.hx = spacing[2];
    c.dta = dta_mm;
    if (or_build_table(&c, radius, 0)) return -4;
    int64_t n = c.ntable;
    if (n <= max_entries) {
        for (int64_t t = 0; t < n; ++t) {
            offsets[3 * t + 0] = c.table[t].i;
            offsets[3 * t + 1] = c.table[t].j;
            offsets[3 * t + 2] = c.table[t].k;
            keys[t] = c.table[t].key;
        }
    }
    free(c.table);
    return n;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Reference and evaluation on different grids.                              */
/* ------------------------------------------------------------------------ */
/* Each grid has its own shape, spacing and origin (mm, same axes).  Eq. 1 is
 * taken literally: for a reference voxel at position x_r with dose D_r,
 *     gamma = min over the evaluation surface (the Freudenthal interpolant of
 *             the evaluation grid, cubes wholly inside it) of
 *             |(x - x_r)/dta, (D_e(x) - D_r)/dD|.
 * The nearest evaluation node is a point of the surface, so its distance
 * g_ub bounds gamma; every cube whose box lies within the running minimum of
 * x_r (in dta units) is searched, by the same simplex distance as above, and
 * no other cube can hold a closer point.  D_norm (global mode) and the
 * cutoff use the reference grid's doses, as for coincident grids. */

typedef struct {
    int ndim;
    int64_t n[3];            /* evaluation grid (x, y, z) */
    double h[3], o[3];       /* evaluation spacing and origin (x, y, z) */
    const float *ev;
    double dta;
} or_egrid;

static double or_grid_cube(const or_egrid *e, const int perms[6][3], int nperm, const int64_t p[3],
                           double inv_dd, const double *P, double best)
{
    const int n = e->ndim, K = n + 1;
    for (int s = 0; s < nperm; ++s) {
        double W[4 * OR_MAXD];
        int64_t q[3] = {p[0], p[1], p[2]};
        for (int v = 0; v <= n; ++v) {
            if (v > 0) q[perms[s][v - 1]] += 1;
            const int64_t lin = (q[2] * e->n[1] + q[1]) * e->n[0] + q[0];
            double *w = W + (size_t)v * K;
            for (int a = 0; a < n; ++a) w[a] = (e->o[a] + (double)q[a] * e->h[a]) / e->dta;
            w[n] = (double)e->ev[lin] * inv_dd;
        }
        double d = oracle_simplex_distance(K, n + 1, W, P);
        if (d < best) best = d;
    }
    return best;
}

/* gamma for the reference voxels listed in idx (all when idx == NULL).
 * ref: float32 (z, y, x) with ref_shape, ref_spacing, ref_origin in (z, y, x)
 * order; likewise ev.  2D: the z entries are ignored.  Returns 0 or a
 * negative code as oracle_gamma. */
int oracle_gamma_grids(const float *ref, const int64_t ref_shape[3], const double ref_spacing[3],
                       const double ref_origin[3], const float *ev, const int64_t ev_shape[3],
                       const double ev_spacing[3], const double ev_origin[3], int ndim,
                       double dd_frac, double dta_mm, int local, double cutoff_frac,
                       double dose_norm, const int64_t *idx, int64_t nidx, double *gamma_out,
                       int threads)
{
    if (ndim != 2 && ndim != 3) return -1;
    if (!(dta_mm > 0) || !(dd_frac > 0)) return -1;
    int64_t rn[3] = {ref_shape[2], ref_shape[1], ndim == 3 ? ref_shape[0] : 1};
    or_egrid e;
    memset(&e, 0, sizeof(e));
    e.ndim = ndim;
    e.ev = ev;
    e.dta = dta_mm;
    e.n[0] = ev_shape[2]; e.n[1] = ev_shape[1]; e.n[2] = ndim == 3 ? ev_shape[0] : 1;
    double rh[3], ro[3];
    for (int a = 0; a < 3; ++a) {
        const int src = 2 - a;                 /* (z, y, x) -> (x, y, z) */
        rh[a] = ref_spacing[src];
        ro[a] = ref_origin[src];
        e.h[a] = ev_spacing[src];
        e.o[a] = ev_origin[src];
    }
    for (int a = 0; a < ndim; ++a) {
        if (rn[a] < 1 || e.n[a] < 2) return -2;
        if (!(rh[a] > 0) || !(e.h[a] > 0)) return -1;
    }
    const int64_t NR = rn[0] * rn[1] * rn[2], NE = e.n[0] * e.n[1] * e.n[2];
    double m = -INFINITY;
    for (int64_t v = 0; v < NR; ++v) {
        if (!isfinite(ref[v])) return -3;
        if (ref[v] > m) m = ref[v];
    }
    for (int64_t v = 0; v < NE; ++v)
        if (!isfinite(ev[v])) return -3;
    or_ctx c;                                  /* criteria helpers only */
    memset(&c, 0, sizeof(c));
    c.ndim = ndim;
    c.dd_frac = dd_frac;
    c.local = local;
    c.cutoff_frac = cutoff_frac;
    c.d_norm = dose_norm > 0 ? dose_norm : m;
    if (!local && !(c.d_norm > 0)) return -1;
    or_make_perms(&c);
    const int64_t n = idx ? nidx : NR;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int64_t t = 0; t < n; ++t) {
        const int64_t v = idx ? idx[t] : t;
        if (v < 0 || v >= NR) { bad |= 1; gamma_out[t] = NAN; continue; }
        const double dr = (double)ref[v];
        if (!or_evaluated(&c, dr)) { gamma_out[t] = NAN; continue; }
        const double inv_dd = 1.0 / or_delta_dose(&c, dr);
        const int64_t ix[3] = {v % rn[0], (v / rn[0]) % rn[1], v / (rn[0] * rn[1])};
        double x[3] = {0, 0, 0}, P[OR_MAXD];
        for (int a = 0; a < ndim; ++a) {
            x[a] = ro[a] + (double)ix[a] * rh[a];
            P[a] = x[a] / dta_mm;
        }
        P[ndim] = dr * inv_dd;
        /* upper bound: the nearest evaluation node */
        int64_t nn[3] = {0, 0, 0};
        for (int a = 0; a < ndim; ++a) {
            double u = floor((x[a] - e.o[a]) / e.h[a] + 0.5);
            if (u < 0) u = 0;
            if (u > (double)(e.n[a] - 1)) u = (double)(e.n[a] - 1);
            nn[a] = (int64_t)u;
        }
        double g2 = 0;
        for (int a = 0; a < ndim; ++a) {
            const double d = (e.o[a] + (double)nn[a] * e.h[a] - x[a]) / dta_mm;
            g2 += d * d;
        }
        {
            const double dd = ((double)ev[(nn[2] * e.n[1] + nn[1]) * e.n[0] + nn[0]] - dr) * inv_dd;
            g2 += dd * dd;
        }
        double g = sqrt(g2);
        /* every cube whose box is within g of x_r */
        int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < ndim; ++a) {
            const double r = g * dta_mm;
            int64_t l = (int64_t)floor((x[a] - r - e.o[a]) / e.h[a]) - 1;
            int64_t u = (int64_t)ceil((x[a] + r - e.o[a]) / e.h[a]) + 1;
            lo[a] = l < 0 ? 0 : l;
            hi[a] = u > e.n[a] - 2 ? e.n[a] - 2 : u;
        }
        for (int64_t pz = lo[2]; pz <= hi[2]; ++pz)
            for (int64_t py = lo[1]; py <= hi[1]; ++py)
                for (int64_t px = lo[0]; px <= hi[0]; ++px) {
                    const int64_t p[3] = {px, py, pz};
                    double key2 = 0;
                    for (int a = 0; a < ndim; ++a) {
                        const double b0 = e.o[a] + (double)p[a] * e.h[a], b1 = b0 + e.h[a];
                        const double d = x[a] < b0 ? b0 - x[a] : (x[a] > b1 ? x[a] - b1 : 0.0);
                        key2 += (d / dta_mm) * (d / dta_mm);
                    }
                    if (!(sqrt(key2) < g)) continue;
                    g = or_grid_cube(&e, c.perms, c.nperm, p, inv_dd, P, g);
                }
        gamma_out[t] = g;
    }
    return bad ? -1 : 0;
}
