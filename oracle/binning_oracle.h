/*
 * binning_oracle.h -- CPU oracle for particle data binning (Sec. 4.2).
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * CPU-baseline timing; the CUDA library never includes or links it.
 */
#ifndef BINNING_ORACLE_H
#define BINNING_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BNO_OK 0
#define BNO_ERR_INVALID_ARG (-1)
#define BNO_ERR_NO_MEMORY (-3)
#define BNO_ERR_DEGENERATE (-7)

#define BNO_MAX_ATTR 16
#define BNO_MAX_RES 65536
#define BNO_MAX_BINS (1LL << 30)

/* lo/hi per axis (ignored when auto_bounds != 0), res per axis. */
typedef struct {
    double lo[2];
    double hi[2];
    int32_t res[2];
    int32_t auto_bounds;
} bno_grid;

int bno_setup_axes_f64(bno_grid* g, const double* x, const double* y, int64_t n,
                       double* lo, double* hi, double* s);
int bno_setup_axes_f32(bno_grid* g, const float* x, const float* y, int64_t n,
                       double* lo, double* hi, double* s);

void bno_state_init_f64(int64_t B, int n_attrs, uint64_t* count, double* sum_s, double* sum_c,
                        double* mn, double* mx);
void bno_state_init_f32(int64_t B, int n_attrs, uint64_t* count, double* sum_s, double* sum_c,
                        float* mn, float* mx);

int bno_accumulate_f64(int64_t n, const double* x, const double* y, int n_attrs,
                       const double* const* attrs, const bno_grid* g,
                       const double* lo, const double* hi, const double* s,
                       uint64_t* count, double* sum_s, double* sum_c, double* mn, double* mx);
int bno_accumulate_f32(int64_t n, const float* x, const float* y, int n_attrs,
                       const float* const* attrs, const bno_grid* g,
                       const double* lo, const double* hi, const double* s,
                       uint64_t* count, double* sum_s, double* sum_c, float* mn, float* mx);

void bno_state_merge_f64(int64_t B, int n_attrs, uint64_t* count, double* sum_s, double* sum_c,
                         double* mn, double* mx, const uint64_t* count_b, const double* sum_s_b,
                         const double* sum_c_b, const double* mn_b, const double* mx_b);
void bno_state_merge_f32(int64_t B, int n_attrs, uint64_t* count, double* sum_s, double* sum_c,
                         float* mn, float* mx, const uint64_t* count_b, const double* sum_s_b,
                         const double* sum_c_b, const float* mn_b, const float* mx_b);

void bno_finalize(int64_t B, int n_attrs, const uint64_t* count, const double* sum_s,
                  const double* sum_c, double* sum, double* avg);

int bno_bin_f64(int64_t n, const double* x, const double* y, int n_attrs,
                const double* const* attrs, bno_grid* g, uint64_t* count, double* sum,
                double* mn, double* mx, double* avg, double* bounds_out);
int bno_bin_f32(int64_t n, const float* x, const float* y, int n_attrs,
                const float* const* attrs, bno_grid* g, uint64_t* count, double* sum,
                float* mn, float* mx, double* avg, double* bounds_out);

/* All-core CPU baseline (binning_threaded.c): per-thread private meshes,
 * then a merge; results as bno_bin_*. */
int bno_bin_threaded_f64(int64_t n, const double* x, const double* y, int n_attrs,
                         const double* const* attrs, bno_grid* g, int nthreads, uint64_t* count,
                         double* sum, double* mn, double* mx, double* avg);
int bno_bin_threaded_f32(int64_t n, const float* x, const float* y, int n_attrs,
                         const float* const* attrs, bno_grid* g, int nthreads, uint64_t* count,
                         double* sum, float* mn, float* mx, double* avg);

int bno_particle_bin_f64(double x, double y, const double* lo, const double* hi,
                         const double* s, const int32_t* res, int closed, int32_t* ixy);
int bno_particle_bin_f32(float x, float y, const double* lo, const double* hi,
                         const double* s, const int32_t* res, int closed, int32_t* ixy);

#ifdef __cplusplus
}
#endif
#endif
