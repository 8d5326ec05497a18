/*
 * harness.h -- benchmark harness kernels that ship in libbinning.so but are
 * not part of the binning path.
 *
 * bn_nbody_step: one kick-drift-kick leapfrog step of a direct-sum gravity
 * simulation (the role of the Newton++ solver of Sec. 4.1: a producer that
 * keeps the GPU busy while in situ binning runs beside it). Softened
 * acceleration a_i = sum_j m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^(3/2)
 * (G = 1), all pairs, FP32.
 *   pos, vel  device float4 arrays of n bodies (x, y, z, w); pos.w is the mass
 *   acc       device float4 scratch of n bodies, holding the accelerations of
 *             the current positions (computed on the first call when
 *             *acc_valid == 0, then kept up to date)
 *   stream    cudaStream_t the step is queued on
 * Each force evaluation is queued as launches over chunks of 4096 source
 * bodies, in order, so that no CTA of the producer holds an SM for a whole
 * step: kernels of other streams (the binning server) get SMs between
 * chunks. The j-order of the sums is the same as one launch's.
 * Errors: BN_ERR_INVALID_ARG for NULL pointers or n < 1, BN_ERR_CUDA.
 */
#ifndef BINNING_HARNESS_H
#define BINNING_HARNESS_H

#include "binning.h"

#ifdef __cplusplus
extern "C" {
#endif

BN_API bn_status bn_nbody_step(void* pos, void* vel, void* acc, int* acc_valid, int64_t n,
                               float dt, float eps, void* stream);

#ifdef __cplusplus
}
#endif
#endif
