/*
 * binning_oracle.c -- plain, slow, single-threaded CPU oracle for particle
 * data binning. TEST INFRASTRUCTURE ONLY: nothing on the product path links,
 * loads or calls this file. It shares no source with the CUDA library.
 *
 * What it computes (Sec. 4.2, "In Situ Data Binning"): two columns of a
 * particle table are the axes of a uniform 2D mesh; each particle's
 * coordinates locate one mesh cell (bin); a per-bin counter gives a
 * histogram, and the other columns are reduced per bin by sum, minimum,
 * maximum and average. The mesh bounds are either given or taken as the
 * minimum and maximum of the coordinate columns.
 *
 * The paper fixes the meaning but not the floating-point details. This
 * oracle takes these readings (each is repeated where it is used):
 *   R1 bin index in the coordinate's own type T:
 *        lo_T = (T)lo, hi_T = (T)hi, s_T = (T)res / (hi_T - lo_T),
 *        t = (x - lo_T) * s_T, i = min((int)t, res - 1),
 *      every operation IEEE round-to-nearest in T, no contraction
 *      (compile with -ffp-contract=off).
 *   R2 explicit bounds are half-open [lo, hi); automatic bounds are the
 *      min/max over finite coordinates and the interval is closed [lo, hi].
 *   R3 particles outside the mesh (or with a NaN coordinate) are dropped
 *      from every reduction.
 *   R4 sums are FP64 with Neumaier compensation (the oracle's job is to be
 *      close to the exact sum, not to mimic any GPU order).
 *   R5 min/max compare in IEEE totalOrder (-0 < +0); NaN attributes are
 *      skipped by min/max and propagate into sum/avg.
 *   R6 empty bins: count 0, sum +0.0, min +inf, max -inf, avg quiet NaN
 *      (bit pattern 0x7ff8000000000000).
 *   R7 count is u64; sum and avg are f64; min and max are in T.
 *
 * Output layout: bin b = iy * res_x + ix (row-major [res_y][res_x]); per-
 * attribute arrays are stacked [n_attrs][B].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "binning_oracle.h"

/* ------------------------------------------------------------------ */
/* grid set-up (R1, R2)                                                */
/* ------------------------------------------------------------------ */

/* Axis parameters for double coordinates. */
typedef struct {
    double lo, hi, s;
    int32_t res;
    int closed;
} axis_d;

typedef struct {
    float lo, hi, s;
    int32_t res;
    int closed;
} axis_f;

static int check_res(const bno_grid* g)
{
    for (int a = 0; a < 2; ++a) {
        if (g->res[a] < 1 || g->res[a] > BNO_MAX_RES) return BNO_ERR_INVALID_ARG;
    }
    if ((int64_t)g->res[0] * (int64_t)g->res[1] > BNO_MAX_BINS) return BNO_ERR_INVALID_ARG;
    return BNO_OK;
}

/* lo_T, hi_T given; fill the rest of the axis. R1: s_T = (T)res / (hi_T - lo_T). */
static int make_axis_d(double lo, double hi, int32_t res, int closed, axis_d* ax)
{
    if (!isfinite(lo) || !isfinite(hi)) return BNO_ERR_INVALID_ARG;
    double width = hi - lo;
    if (!(width > 0.0) || !isfinite(width)) return BNO_ERR_INVALID_ARG;
    double s = (double)res / width;
    if (!isfinite(s) || !(s > 0.0)) return BNO_ERR_INVALID_ARG;
    ax->lo = lo; ax->hi = hi; ax->s = s; ax->res = res; ax->closed = closed;
    return BNO_OK;
}

static int make_axis_f(float lo, float hi, int32_t res, int closed, axis_f* ax)
{
    if (!isfinite(lo) || !isfinite(hi)) return BNO_ERR_INVALID_ARG;
    float width = hi - lo;
    if (!(width > 0.0f) || !isfinite(width)) return BNO_ERR_INVALID_ARG;
    float s = (float)res / width;
    if (!isfinite(s) || !(s > 0.0f)) return BNO_ERR_INVALID_ARG;
    ax->lo = lo; ax->hi = hi; ax->s = s; ax->res = res; ax->closed = closed;
    return BNO_OK;
}

/* R1 + R2 + R3: is x inside the axis, and if so which bin. */
static int axis_bin_d(const axis_d* ax, double x, int32_t* i)
{
    int inside = ax->closed ? (ax->lo <= x && x <= ax->hi) : (ax->lo <= x && x < ax->hi);
    if (!inside) return 0;             /* NaN fails both comparisons */
    double t = (x - ax->lo) * ax->s;   /* two roundings, never fused */
    int32_t k = (int32_t)t;            /* t >= 0, so truncation is floor */
    if (k > ax->res - 1) k = ax->res - 1;
    *i = k;
    return 1;
}

static int axis_bin_f(const axis_f* ax, float x, int32_t* i)
{
    int inside = ax->closed ? (ax->lo <= x && x <= ax->hi) : (ax->lo <= x && x < ax->hi);
    if (!inside) return 0;
    float t = (x - ax->lo) * ax->s;
    int32_t k = (int32_t)t;
    if (k > ax->res - 1) k = ax->res - 1;
    *i = k;
    return 1;
}

/* R2 automatic bounds: min and max over the finite values of a column. */
static int finite_range_d(const double* c, int64_t n, double* lo, double* hi)
{
    int any = 0;
    for (int64_t k = 0; k < n; ++k) {
        double v = c[k];
        if (!isfinite(v)) continue;
        if (!any || v < *lo) *lo = v;
        if (!any || v > *hi) *hi = v;
        any = 1;
    }
    return any;
}

static int finite_range_f(const float* c, int64_t n, float* lo, float* hi)
{
    int any = 0;
    for (int64_t k = 0; k < n; ++k) {
        float v = c[k];
        if (!isfinite(v)) continue;
        if (!any || v < *lo) *lo = v;
        if (!any || v > *hi) *hi = v;
        any = 1;
    }
    return any;
}

int bno_setup_axes_f64(bno_grid* g, const double* x, const double* y, int64_t n,
                       double* lo_out, double* hi_out, double* s_out)
{
    int st = check_res(g);
    if (st) return st;
    axis_d ax[2];
    const double* col[2] = {x, y};
    for (int a = 0; a < 2; ++a) {
        double lo, hi;
        if (g->auto_bounds) {
            if (!finite_range_d(col[a], n, &lo, &hi)) return BNO_ERR_DEGENERATE;
            st = make_axis_d(lo, hi, g->res[a], 1, &ax[a]);
            if (st) return BNO_ERR_DEGENERATE;
        } else {
            st = make_axis_d(g->lo[a], g->hi[a], g->res[a], 0, &ax[a]);
            if (st) return st;
        }
        lo_out[a] = ax[a].lo; hi_out[a] = ax[a].hi; s_out[a] = ax[a].s;
    }
    return BNO_OK;
}

int bno_setup_axes_f32(bno_grid* g, const float* x, const float* y, int64_t n,
                       double* lo_out, double* hi_out, double* s_out)
{
    int st = check_res(g);
    if (st) return st;
    axis_f ax[2];
    const float* col[2] = {x, y};
    for (int a = 0; a < 2; ++a) {
        float lo, hi;
        if (g->auto_bounds) {
            if (!finite_range_f(col[a], n, &lo, &hi)) return BNO_ERR_DEGENERATE;
            st = make_axis_f(lo, hi, g->res[a], 1, &ax[a]);
            if (st) return BNO_ERR_DEGENERATE;
        } else {
            st = make_axis_f((float)g->lo[a], (float)g->hi[a], g->res[a], 0, &ax[a]);
            if (st) return st;
        }
        lo_out[a] = ax[a].lo; hi_out[a] = ax[a].hi; s_out[a] = ax[a].s;
    }
    return BNO_OK;
}

/* ------------------------------------------------------------------ */
/* per-bin state                                                       */
/* ------------------------------------------------------------------ */

/* R5: a < b in IEEE totalOrder, for non-NaN a and b. */
static int total_less_d(double a, double b)
{
    if (a < b) return 1;
    if (a == 0.0 && b == 0.0) return signbit(a) && !signbit(b);
    return 0;
}

static int total_less_f(float a, float b)
{
    if (a < b) return 1;
    if (a == 0.0f && b == 0.0f) return signbit(a) && !signbit(b);
    return 0;
}

/* R4: one Neumaier step on (s, c). */
static void neumaier_add(double* s, double* c, double a)
{
    double t = *s + a;
    if (fabs(*s) >= fabs(a))
        *c += (*s - t) + a;
    else
        *c += (a - t) + *s;
    *s = t;
}

void bno_state_init_f64(int64_t B, int n_attrs, uint64_t* count, double* sum_s, double* sum_c,
                        double* mn, double* mx)
{
    for (int64_t b = 0; b < B; ++b) count[b] = 0;
    for (int64_t k = 0; k < B * n_attrs; ++k) {
        sum_s[k] = 0.0; sum_c[k] = 0.0; mn[k] = INFINITY; mx[k] = -INFINITY;
    }
}

void bno_state_init_f32(int64_t B, int n_attrs, uint64_t* count, double* sum_s, double* sum_c,
                        float* mn, float* mx)
{
    for (int64_t b = 0; b < B; ++b) count[b] = 0;
    for (int64_t k = 0; k < B * n_attrs; ++k) {
        sum_s[k] = 0.0; sum_c[k] = 0.0; mn[k] = INFINITY; mx[k] = -INFINITY;
    }
}

/*
 * Accumulate particles [0, n) in input order into the state. The axes come
 * from bno_setup_axes_*: lo, hi and s already in T, closed = auto bounds.
 */
int bno_accumulate_f64(int64_t n, const double* x, const double* y, int n_attrs,
                       const double* const* attrs, const bno_grid* g,
                       const double* lo, const double* hi, const double* s,
                       uint64_t* count, double* sum_s, double* sum_c, double* mn, double* mx)
{
    axis_d ax[2];
    for (int a = 0; a < 2; ++a) {
        ax[a].lo = lo[a]; ax[a].hi = hi[a]; ax[a].s = s[a];
        ax[a].res = g->res[a]; ax[a].closed = g->auto_bounds != 0;
    }
    const int64_t B = (int64_t)g->res[0] * g->res[1];
    for (int64_t k = 0; k < n; ++k) {
        int32_t ix, iy;
        if (!axis_bin_d(&ax[0], x[k], &ix)) continue;
        if (!axis_bin_d(&ax[1], y[k], &iy)) continue;
        int64_t b = (int64_t)iy * g->res[0] + ix;
        count[b] += 1;
        for (int a = 0; a < n_attrs; ++a) {
            double v = attrs[a][k];
            int64_t j = (int64_t)a * B + b;
            neumaier_add(&sum_s[j], &sum_c[j], v);
            if (isnan(v)) continue;
            if (total_less_d(v, mn[j])) mn[j] = v;
            if (total_less_d(mx[j], v)) mx[j] = v;
        }
    }
    return BNO_OK;
}

int bno_accumulate_f32(int64_t n, const float* x, const float* y, int n_attrs,
                       const float* const* attrs, const bno_grid* g,
                       const double* lo, const double* hi, const double* s,
                       uint64_t* count, double* sum_s, double* sum_c, float* mn, float* mx)
{
    axis_f ax[2];
    for (int a = 0; a < 2; ++a) {
        /* lo, hi, s were produced in float and widened exactly; narrow back. */
        ax[a].lo = (float)lo[a]; ax[a].hi = (float)hi[a]; ax[a].s = (float)s[a];
        ax[a].res = g->res[a]; ax[a].closed = g->auto_bounds != 0;
    }
    const int64_t B = (int64_t)g->res[0] * g->res[1];
    for (int64_t k = 0; k < n; ++k) {
        int32_t ix, iy;
        if (!axis_bin_f(&ax[0], x[k], &ix)) continue;
        if (!axis_bin_f(&ax[1], y[k], &iy)) continue;
        int64_t b = (int64_t)iy * g->res[0] + ix;
        count[b] += 1;
        for (int a = 0; a < n_attrs; ++a) {
            float v = attrs[a][k];
            int64_t j = (int64_t)a * B + b;
            neumaier_add(&sum_s[j], &sum_c[j], (double)v);   /* widening is exact */
            if (isnan(v)) continue;
            if (total_less_f(v, mn[j])) mn[j] = v;
            if (total_less_f(mx[j], v)) mx[j] = v;
        }
    }
    return BNO_OK;
}

/* Combine state b into state a (shard merge; Sec. 4.2 bins with MPI, so the
 * per-rank partial meshes must combine associatively). */
void bno_state_merge_f64(int64_t B, int n_attrs, uint64_t* count, double* sum_s, double* sum_c,
                         double* mn, double* mx, const uint64_t* count_b, const double* sum_s_b,
                         const double* sum_c_b, const double* mn_b, const double* mx_b)
{
    for (int64_t b = 0; b < B; ++b) count[b] += count_b[b];
    for (int64_t k = 0; k < B * n_attrs; ++k) {
        neumaier_add(&sum_s[k], &sum_c[k], sum_s_b[k]);
        sum_c[k] += sum_c_b[k];
        if (total_less_d(mn_b[k], mn[k])) mn[k] = mn_b[k];
        if (total_less_d(mx[k], mx_b[k])) mx[k] = mx_b[k];
    }
}

void bno_state_merge_f32(int64_t B, int n_attrs, uint64_t* count, double* sum_s, double* sum_c,
                         float* mn, float* mx, const uint64_t* count_b, const double* sum_s_b,
                         const double* sum_c_b, const float* mn_b, const float* mx_b)
{
    for (int64_t b = 0; b < B; ++b) count[b] += count_b[b];
    for (int64_t k = 0; k < B * n_attrs; ++k) {
        neumaier_add(&sum_s[k], &sum_c[k], sum_s_b[k]);
        sum_c[k] += sum_c_b[k];
        if (total_less_f(mn_b[k], mn[k])) mn[k] = mn_b[k];
        if (total_less_f(mx[k], mx_b[k])) mx[k] = mx_b[k];
    }
}

/* R4 + R6: sum = s + c (or s alone once it is not finite), avg = sum / count. */
void bno_finalize(int64_t B, int n_attrs, const uint64_t* count, const double* sum_s,
                  const double* sum_c, double* sum, double* avg)
{
    uint64_t qnan_bits = 0x7ff8000000000000ull;
    double qnan;
    memcpy(&qnan, &qnan_bits, sizeof qnan);
    for (int a = 0; a < n_attrs; ++a) {
        for (int64_t b = 0; b < B; ++b) {
            int64_t j = (int64_t)a * B + b;
            double v = isfinite(sum_s[j]) ? sum_s[j] + sum_c[j] : sum_s[j];
            sum[j] = v;
            avg[j] = count[b] ? v / (double)count[b] : qnan;
        }
    }
}

/* ------------------------------------------------------------------ */
/* one-call drivers                                                    */
/* ------------------------------------------------------------------ */

int bno_bin_f64(int64_t n, const double* x, const double* y, int n_attrs,
                const double* const* attrs, bno_grid* g, uint64_t* count, double* sum,
                double* mn, double* mx, double* avg, double* bounds_out)
{
    if (n < 0 || n_attrs < 0 || n_attrs > BNO_MAX_ATTR) return BNO_ERR_INVALID_ARG;
    double lo[2], hi[2], s[2];
    int st = bno_setup_axes_f64(g, x, y, n, lo, hi, s);
    if (st) return st;
    const int64_t B = (int64_t)g->res[0] * g->res[1];
    double* sum_c = (double*)malloc(sizeof(double) * (size_t)(B * n_attrs + 1));
    double* sum_s = (double*)malloc(sizeof(double) * (size_t)(B * n_attrs + 1));
    if (!sum_c || !sum_s) { free(sum_c); free(sum_s); return BNO_ERR_NO_MEMORY; }
    bno_state_init_f64(B, n_attrs, count, sum_s, sum_c, mn, mx);
    bno_accumulate_f64(n, x, y, n_attrs, attrs, g, lo, hi, s, count, sum_s, sum_c, mn, mx);
    bno_finalize(B, n_attrs, count, sum_s, sum_c, sum, avg);
    free(sum_c); free(sum_s);
    if (bounds_out) { bounds_out[0] = lo[0]; bounds_out[1] = hi[0]; bounds_out[2] = lo[1]; bounds_out[3] = hi[1]; }
    return BNO_OK;
}

int bno_bin_f32(int64_t n, const float* x, const float* y, int n_attrs,
                const float* const* attrs, bno_grid* g, uint64_t* count, double* sum,
                float* mn, float* mx, double* avg, double* bounds_out)
{
    if (n < 0 || n_attrs < 0 || n_attrs > BNO_MAX_ATTR) return BNO_ERR_INVALID_ARG;
    double lo[2], hi[2], s[2];
    int st = bno_setup_axes_f32(g, x, y, n, lo, hi, s);
    if (st) return st;
    const int64_t B = (int64_t)g->res[0] * g->res[1];
    double* sum_c = (double*)malloc(sizeof(double) * (size_t)(B * n_attrs + 1));
    double* sum_s = (double*)malloc(sizeof(double) * (size_t)(B * n_attrs + 1));
    if (!sum_c || !sum_s) { free(sum_c); free(sum_s); return BNO_ERR_NO_MEMORY; }
    bno_state_init_f32(B, n_attrs, count, sum_s, sum_c, mn, mx);
    bno_accumulate_f32(n, x, y, n_attrs, attrs, g, lo, hi, s, count, sum_s, sum_c, mn, mx);
    bno_finalize(B, n_attrs, count, sum_s, sum_c, sum, avg);
    free(sum_c); free(sum_s);
    if (bounds_out) { bounds_out[0] = lo[0]; bounds_out[1] = hi[0]; bounds_out[2] = lo[1]; bounds_out[3] = hi[1]; }
    return BNO_OK;
}

/* Single-particle bin index, exposed so tests can pin R1/R2 point by point.
 * Returns 1 and writes (ix, iy) when the particle is inside, else 0. */
int bno_particle_bin_f64(double x, double y, const double* lo, const double* hi,
                         const double* s, const int32_t* res, int closed, int32_t* ixy)
{
    axis_d ax[2];
    for (int a = 0; a < 2; ++a) {
        ax[a].lo = lo[a]; ax[a].hi = hi[a]; ax[a].s = s[a]; ax[a].res = res[a]; ax[a].closed = closed;
    }
    return axis_bin_d(&ax[0], x, &ixy[0]) && axis_bin_d(&ax[1], y, &ixy[1]);
}

int bno_particle_bin_f32(float x, float y, const double* lo, const double* hi,
                         const double* s, const int32_t* res, int closed, int32_t* ixy)
{
    axis_f ax[2];
    for (int a = 0; a < 2; ++a) {
        ax[a].lo = (float)lo[a]; ax[a].hi = (float)hi[a]; ax[a].s = (float)s[a];
        ax[a].res = res[a]; ax[a].closed = closed;
    }
    return axis_bin_f(&ax[0], x, &ixy[0]) && axis_bin_f(&ax[1], y, &ixy[1]);
}
