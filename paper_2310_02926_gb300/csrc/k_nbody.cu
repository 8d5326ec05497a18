// k_nbody.cu -- K6, the producer of the serving benchmark: a direct-sum
// gravity leapfrog step (Sec. 4.1's Newton++ is a direct n-body code with a
// second-order symplectic integrator). Not on the binning path.
#include <cuda_runtime.h>

#include "../../include/harness.h"
#include "bn_runtime.h"

namespace {

constexpr int kTile = 256;
// Bodies j one launch of the force kernel sums over. One launch over all
// bodies keeps every CTA resident for the whole step (about 2.7 ms at
// N = 65,536), and a kernel of another stream that needs a whole SM (a
// binning request of the server) waits for those CTAs to finish; chunks of
// 4096 end every CTA after about 0.2 ms. The chunks run in order on the
// producer's stream, each adding to the previous one's sums, so the result
// does not depend on how the launches interleave with other work.
constexpr int64_t kChunk = 4096;

// Accelerations from bodies [j_begin, j_end): each thread owns one body, the
// block walks those bodies in shared-memory tiles of kTile; the first chunk
// writes acc, later chunks add to it.
__global__ void __launch_bounds__(kTile) k_nbody_acc(const float4* __restrict__ pos,
                                                     float4* __restrict__ acc, int64_t n, float eps2,
                                                     int64_t j_begin, int64_t j_end) {
    __shared__ float4 tile[kTile];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float4 pi = i < n ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float ax = 0.f, ay = 0.f, az = 0.f;
    if (j_begin > 0 && i < n) {
        const float4 a = acc[i];
        ax = a.x;
        ay = a.y;
        az = a.z;
    }
    for (int64_t j0 = j_begin; j0 < j_end; j0 += kTile) {
        const int64_t j = j0 + threadIdx.x;
        tile[threadIdx.x] = j < j_end ? pos[j] : make_float4(0.f, 0.f, 0.f, 0.f);  // w = 0: no pull
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kTile; ++k) {
            const float4 pj = tile[k];
            const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
            const float inv = rsqrtf(r2);
            const float s = pj.w * inv * inv * inv;
            ax = fmaf(dx, s, ax);
            ay = fmaf(dy, s, ay);
            az = fmaf(dz, s, az);
        }
        __syncthreads();
    }
    if (i < n) acc[i] = make_float4(ax, ay, az, 0.f);
}

// half kick with the current accelerations, then drift
__global__ void k_nbody_kick_drift(float4* __restrict__ pos, float4* __restrict__ vel,
                                   const float4* __restrict__ acc, int64_t n, float dt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 v = vel[i];
    const float4 a = acc[i];
    v.x = fmaf(0.5f * dt, a.x, v.x);
    v.y = fmaf(0.5f * dt, a.y, v.y);
    v.z = fmaf(0.5f * dt, a.z, v.z);
    float4 p = pos[i];
    p.x = fmaf(dt, v.x, p.x);
    p.y = fmaf(dt, v.y, p.y);
    p.z = fmaf(dt, v.z, p.z);
    pos[i] = p;
    vel[i] = v;
}

// second half kick with the new accelerations
__global__ void k_nbody_kick(float4* __restrict__ vel, const float4* __restrict__ acc, int64_t n, float dt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 v = vel[i];
    const float4 a = acc[i];
    v.x = fmaf(0.5f * dt, a.x, v.x);
    v.y = fmaf(0.5f * dt, a.y, v.y);
    v.z = fmaf(0.5f * dt, a.z, v.z);
    vel[i] = v;
}

}  // namespace

extern "C" bn_status bn_nbody_step(void* pos, void* vel, void* acc, int* acc_valid, int64_t n,
                                   float dt, float eps, void* stream) {
    if (!pos || !vel || !acc || !acc_valid || n < 1)
        return bn::fail(BN_ERR_INVALID_ARG, "bn_nbody_step: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned grid = (unsigned)((n + kTile - 1) / kTile);
    float4* P = static_cast<float4*>(pos);
    float4* V = static_cast<float4*>(vel);
    float4* A = static_cast<float4*>(acc);
    const float eps2 = eps * eps;
    auto forces = [&]() {
        for (int64_t j = 0; j < n; j += kChunk)
            k_nbody_acc<<<grid, kTile, 0, s>>>(P, A, n, eps2, j, j + kChunk < n ? j + kChunk : n);
    };
    if (!*acc_valid) {
        forces();
        *acc_valid = 1;
    }
    k_nbody_kick_drift<<<grid, kTile, 0, s>>>(P, V, A, n, dt);
    forces();
    k_nbody_kick<<<grid, kTile, 0, s>>>(V, A, n, dt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bn::cuda_fail(e, "bn_nbody_step");
    return BN_OK;
}
