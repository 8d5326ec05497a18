/*
 * binning_threaded.c -- the all-core CPU baseline for particle data binning.
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY: it is timed beside the GPU path as
 * a reported baseline and checked against the single-threaded oracle; the
 * CUDA library never links, loads or calls it.
 *
 * The plain FP64 binning of Sec. 4.2 spread over host threads the way the
 * paper spreads it over MPI ranks (each rank bins its own particles, then
 * the partial meshes combine): the particles are cut into one contiguous
 * shard per thread, every thread bins its shard into a private mesh with
 * the oracle's own accumulate step (binning_oracle.c: same bin index, same
 * Neumaier sums, same totalOrder min/max), then the threads merge the
 * private meshes bin range by bin range with the oracle's merge step and
 * the oracle's finalise step computes sum and avg. No new arithmetic is
 * introduced here; only the order in which partial sums combine differs
 * from the single-threaded oracle.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "binning_oracle.h"

typedef struct shard_s {
    int dt;                  /* 8: f64, 4: f32 */
    int64_t n0, n1;          /* particle shard */
    int64_t b0, b1;          /* bin range of the merge phase */
    int n_attrs;
    const void* x;
    const void* y;
    const void* const* attrs;
    const bno_grid* g;
    const double* lo;
    const double* hi;
    const double* s;
    int64_t B;
    uint64_t* count;
    double* sum_s;
    double* sum_c;
    void* mn;
    void* mx;
    int rc;
    struct shard_s* all;     /* every shard of the call (merge phase) */
    int nall;
} shard_t;

static void* accumulate_shard(void* p)
{
    shard_t* t = (shard_t*)p;
    const int64_t n = t->n1 - t->n0;
    const void* ap[BNO_MAX_ATTR];
    if (t->dt == 8) {
        for (int a = 0; a < t->n_attrs; ++a) ap[a] = (const double*)t->attrs[a] + t->n0;
        bno_state_init_f64(t->B, t->n_attrs, t->count, t->sum_s, t->sum_c, (double*)t->mn, (double*)t->mx);
        t->rc = bno_accumulate_f64(n, (const double*)t->x + t->n0, (const double*)t->y + t->n0, t->n_attrs,
                                   (const double* const*)ap, t->g, t->lo, t->hi, t->s, t->count,
                                   t->sum_s, t->sum_c, (double*)t->mn, (double*)t->mx);
    } else {
        for (int a = 0; a < t->n_attrs; ++a) ap[a] = (const float*)t->attrs[a] + t->n0;
        bno_state_init_f32(t->B, t->n_attrs, t->count, t->sum_s, t->sum_c, (float*)t->mn, (float*)t->mx);
        t->rc = bno_accumulate_f32(n, (const float*)t->x + t->n0, (const float*)t->y + t->n0, t->n_attrs,
                                   (const float* const*)ap, t->g, t->lo, t->hi, t->s, t->count,
                                   t->sum_s, t->sum_c, (float*)t->mn, (float*)t->mx);
    }
    return NULL;
}

/* Merge bins [b0, b1) of shards 1.. into shard 0, in shard order. */
static void* merge_range(void* p)
{
    shard_t* t = (shard_t*)p;
    const int64_t len = t->b1 - t->b0;
    if (len <= 0) return NULL;
    shard_t* d = &t->all[0];
    uint64_t* scratch = (uint64_t*)calloc((size_t)len, sizeof(uint64_t));
    if (!scratch) { t->rc = BNO_ERR_NO_MEMORY; return NULL; }
    for (int k = 1; k < t->nall; ++k) {
        shard_t* s = &t->all[k];
        const int64_t b0 = t->b0;
        if (t->dt == 8) {
            bno_state_merge_f64(len, 0, d->count + b0, NULL, NULL, NULL, NULL, s->count + b0, NULL, NULL,
                                NULL, NULL);
            for (int a = 0; a < t->n_attrs; ++a) {
                const int64_t o = (int64_t)a * t->B + b0;
                bno_state_merge_f64(len, 1, scratch, d->sum_s + o, d->sum_c + o, (double*)d->mn + o,
                                    (double*)d->mx + o, s->count + b0, s->sum_s + o, s->sum_c + o,
                                    (const double*)s->mn + o, (const double*)s->mx + o);
            }
        } else {
            bno_state_merge_f32(len, 0, d->count + b0, NULL, NULL, NULL, NULL, s->count + b0, NULL, NULL,
                                NULL, NULL);
            for (int a = 0; a < t->n_attrs; ++a) {
                const int64_t o = (int64_t)a * t->B + b0;
                bno_state_merge_f32(len, 1, scratch, d->sum_s + o, d->sum_c + o, (float*)d->mn + o,
                                    (float*)d->mx + o, s->count + b0, s->sum_s + o, s->sum_c + o,
                                    (const float*)s->mn + o, (const float*)s->mx + o);
            }
        }
    }
    free(scratch);
    return NULL;
}

static int run_threads(shard_t* sh, int T, void* (*fn)(void*))
{
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)T);
    if (!th) return BNO_ERR_NO_MEMORY;
    int started = 0, rc = BNO_OK;
    for (int k = 1; k < T; ++k) {
        if (pthread_create(&th[k], NULL, fn, &sh[k]) != 0) { rc = BNO_ERR_NO_MEMORY; break; }
        started = k;
    }
    fn(&sh[0]);
    for (int k = 1; k <= started; ++k) pthread_join(th[k], NULL);
    free(th);
    for (int k = 0; k < T && rc == BNO_OK; ++k) rc = sh[k].rc;
    return rc;
}

/*
 * Bin with nthreads host threads (dt = 8: f64 columns and min/max, dt = 4:
 * f32). Outputs as bno_bin_f64 / bno_bin_f32. Every thread holds a private
 * mesh of B * (8 + n_attrs * (16 + 2 * dt)) bytes.
 */
static int bin_threaded(int dt, int64_t n, const void* x, const void* y, int n_attrs,
                        const void* const* attrs, bno_grid* g, int nthreads, uint64_t* count,
                        double* sum, void* mn, void* mx, double* avg)
{
    if (n < 0 || n_attrs < 0 || n_attrs > BNO_MAX_ATTR || nthreads < 1) return BNO_ERR_INVALID_ARG;
    double lo[2], hi[2], s[2];
    int st = dt == 8 ? bno_setup_axes_f64(g, (const double*)x, (const double*)y, n, lo, hi, s)
                     : bno_setup_axes_f32(g, (const float*)x, (const float*)y, n, lo, hi, s);
    if (st) return st;
    const int64_t B = (int64_t)g->res[0] * g->res[1];
    const int T = (int64_t)nthreads > n + 1 ? (int)(n + 1) : nthreads;
    shard_t* sh = (shard_t*)calloc((size_t)T, sizeof(shard_t));
    if (!sh) return BNO_ERR_NO_MEMORY;
    const size_t AB = (size_t)(B * n_attrs + 1);
    int rc = BNO_OK;
    for (int k = 0; k < T && rc == BNO_OK; ++k) {
        shard_t* t = &sh[k];
        t->dt = dt;
        t->n0 = n * k / T;
        t->n1 = n * (k + 1) / T;
        t->b0 = B * k / T;
        t->b1 = B * (k + 1) / T;
        t->n_attrs = n_attrs;
        t->x = x; t->y = y; t->attrs = attrs; t->g = g;
        t->lo = lo; t->hi = hi; t->s = s;
        t->B = B;
        t->all = sh;
        t->nall = T;
        t->sum_s = (double*)malloc(sizeof(double) * AB);
        t->sum_c = (double*)malloc(sizeof(double) * AB);
        if (k == 0) {  /* shard 0 accumulates into the caller's outputs */
            t->count = count; t->mn = mn; t->mx = mx;
        } else {
            t->count = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(B + 1));
            t->mn = malloc((size_t)dt * AB);
            t->mx = malloc((size_t)dt * AB);
        }
        if (!t->sum_s || !t->sum_c || !t->count || (n_attrs > 0 && (!t->mn || !t->mx))) rc = BNO_ERR_NO_MEMORY;
    }
    if (rc == BNO_OK) rc = run_threads(sh, T, accumulate_shard);
    if (rc == BNO_OK) rc = run_threads(sh, T, merge_range);
    if (rc == BNO_OK) bno_finalize(B, n_attrs, count, sh[0].sum_s, sh[0].sum_c, sum, avg);
    for (int k = 0; k < T; ++k) {
        free(sh[k].sum_s);
        free(sh[k].sum_c);
        if (k > 0) { free(sh[k].count); free(sh[k].mn); free(sh[k].mx); }
    }
    free(sh);
    return rc;
}

int bno_bin_threaded_f64(int64_t n, const double* x, const double* y, int n_attrs,
                         const double* const* attrs, bno_grid* g, int nthreads, uint64_t* count,
                         double* sum, double* mn, double* mx, double* avg)
{
    return bin_threaded(8, n, x, y, n_attrs, (const void* const*)attrs, g, nthreads, count, sum, mn, mx, avg);
}

int bno_bin_threaded_f32(int64_t n, const float* x, const float* y, int n_attrs,
                         const float* const* attrs, bno_grid* g, int nthreads, uint64_t* count,
                         double* sum, float* mn, float* mx, double* avg)
{
    return bin_threaded(4, n, x, y, n_attrs, (const void* const*)attrs, g, nthreads, count, sum, mn, mx, avg);
}
