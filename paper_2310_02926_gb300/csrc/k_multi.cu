// k_multi.cu -- fused multi-grid pass: several binnings of the same
// particles in one launch (Sec. 4.3 bins 10 variables in 9 coordinate
// systems every step).
//
// CTAs take tiles of kMultiTile particles and run every spec over a tile
// before moving to the next. A spec reads its coordinate and attribute
// columns for the tile; the first spec to touch a column brings it from
// DRAM, the others find it in L1/L2 (a tile of one f64 column is 8 KB), so
// each column crosses DRAM once however many specs use it. Each spec bins
// exactly as the global strategy does (same bin index, same commit), so its
// result equals a bn_bin_particles call on its columns and grid.
#include <cuda_runtime.h>

#include "bn_device.cuh"
#include "bn_internal.cuh"
#include "bn_kernels.h"

namespace bn {

template <typename T>
__global__ void __launch_bounds__(256) k_bin_multi(const MultiSpec* __restrict__ specs, int n_specs,
                                                   int64_t n) {
    // every spec's binner, built once per CTA
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ MultiSpec cur;
    Binner<T>* binners = reinterpret_cast<Binner<T>*>(smem);
    for (int s = threadIdx.x; s < n_specs; s += blockDim.x) {
        const GridDesc g = *specs[s].grid;
        Binner<T> bnr;
        if (g.valid) bnr.init(g);
        else bnr.rx = -1;  // marks an invalid mesh: the spec is skipped
        binners[s] = bnr;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = threadIdx.x & ~31;
    const int64_t ntiles = (n + kMultiTile - 1) / kMultiTile;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t i0 = t * kMultiTile;
        const int64_t i1 = (n - i0) < kMultiTile ? n : i0 + kMultiTile;
        for (int s = 0; s < n_specs; ++s) {
            const Binner<T>& binner = binners[s];
            if (binner.rx < 0) continue;
            // the spec's descriptor in shared memory: its pointers cannot alias
            // the global atomics, so they are not reloaded around every commit
            __syncthreads();
            {
                const int* src = reinterpret_cast<const int*>(specs + s);
                int* dst = reinterpret_cast<int*>(&cur);
                for (int w = threadIdx.x; w < (int)(sizeof(MultiSpec) / sizeof(int)); w += blockDim.x)
                    dst[w] = src[w];
            }
            __syncthreads();
            const MultiSpec& sp = cur;
            const T* __restrict__ X = static_cast<const T*>(sp.x);
            const T* __restrict__ Y = static_cast<const T*>(sp.y);
            const int A = sp.n_attrs;
            const bool agg = sp.aggregate != 0;
            // whole warps iterate together (warp_commit needs every lane)
            for (int64_t base = i0 + warp0; base < i1; base += blockDim.x) {
                const int64_t i = base + lane;
                int b = -1;
                T v[kMaxAttr];
                if (i < i1) {
                    b = binner.bin(X[i], Y[i]);
                    for (int a = 0; a < A; ++a) v[a] = static_cast<const T*>(sp.a[a])[i];
                }
                warp_commit<T, -1>(sp.st, A, b, v, agg);
            }
        }
    }
}

cudaError_t launch_bin_multi(const KernelCtx& kc, int dtype, const MultiSpec* dev_specs, int n_specs,
                             int64_t n) {
    if (n <= 0 || n_specs <= 0) return cudaSuccess;
    const int block = 256;
    int64_t grid = (n + kMultiTile - 1) / kMultiTile;
    // 4 CTAs per SM: a tile's columns (kMultiTile x columns x 8 B) stay within
    // a CTA's share of L2 between the specs that read them
    const int64_t cap = (int64_t)kc.num_sms * 4;
    if (grid > cap) grid = cap;
    if (dtype == BN_F64)
        k_bin_multi<double><<<(int)grid, block, sizeof(Binner<double>) * n_specs, kc.stream>>>(dev_specs, n_specs, n);
    else
        k_bin_multi<float><<<(int)grid, block, sizeof(Binner<float>) * n_specs, kc.stream>>>(dev_specs, n_specs, n);
    kc.count_launch();
    return cudaGetLastError();
}

}  // namespace bn
