// k_multi.cu -- fused multi-grid pass: several binnings of the same
// particles in one launch (Sec. 4.3 bins 10 variables in 9 coordinate
// systems every step).
//
// CTAs take tiles of kMultiTile particles and run every spec over a tile
// before moving to the next. A spec reads its coordinate and attribute
// columns for the tile; the first spec to touch a column brings it from
// DRAM, the others find it in L1/L2 (a tile of one f64 column is 8 KB), so
// each column crosses DRAM once however many specs use it. Each spec bins
// exactly as the global strategy does (same bin index, same commit, count
// and sums as one bulk reduction of the bin's record), so its result equals
// a bn_bin_particles call on its columns and grid.
#include <cuda_runtime.h>

#include "bn_device.cuh"
#include "bn_internal.cuh"
#include "bn_kernels.h"

namespace bn {

// One spec over one tile. K: the spec's attribute count, so that the
// per-particle values and the commit's partial sums live in registers (-1:
// any count, through local memory). For up to four attributes, when every
// column of the spec is 16-byte aligned, a lane reads VN consecutive
// particles with one vector load per column (read-only cache: the next
// specs of the tile read the same columns); the tile's last partial group
// goes one particle per lane. (With ten f64 attributes the vector values
// raised the kernel from 126 to 194 registers and the 9 x 10 pass from
// 4.48 to 5.08 ms, so larger counts load one particle per lane.)
template <typename T, int K>
__device__ __forceinline__ void multi_tile(const MultiSpec& sp, const Binner<T>& binner, int64_t i0,
                                           int64_t i1, double* slot) {
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::N;
    constexpr int KC = K > 0 ? K : (K == 0 ? 1 : kMaxAttr);
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = threadIdx.x & ~31;
    const T* __restrict__ X = static_cast<const T*>(sp.x);
    const T* __restrict__ Y = static_cast<const T*>(sp.y);
    const int A = K >= 0 ? K : sp.n_attrs;
    const bool agg = sp.aggregate != 0;
    constexpr bool kVec = K >= 0 && K <= 4;
    bool vec = kVec && ((uintptr_t)X & 15) == 0 && ((uintptr_t)Y & 15) == 0 && i0 % VN == 0;
    if constexpr (K > 0) {
#pragma unroll
        for (int a = 0; a < K; ++a) vec = vec && ((uintptr_t)sp.a[a] & 15) == 0;
    }
    int64_t s0 = i0;  // first particle of the scalar part
    if constexpr (kVec) {
        if (vec) {
            const int64_t g0 = i0 / VN, g1 = i1 / VN;
            const V* XV = reinterpret_cast<const V*>(X);
            const V* YV = reinterpret_cast<const V*>(Y);
            for (int64_t base = g0 + warp0; base < g1; base += blockDim.x) {
                const int64_t gi = base + lane;
                const bool live = gi < g1;
                V xv, yv, av[KC];
                if (live) {
                    xv = __ldg(XV + gi);
                    yv = __ldg(YV + gi);
                    if constexpr (K > 0) {
    #pragma unroll
                        for (int a = 0; a < K; ++a) av[a] = __ldg(reinterpret_cast<const V*>(sp.a[a]) + gi);
                    }
                }
    #pragma unroll
                for (int j = 0; j < VN; ++j) {
                    int b = -1;
                    T v[KC];
                    if (live) {
                        b = binner.bin(vget<T>(xv, j), vget<T>(yv, j));
                        if constexpr (K > 0) {
    #pragma unroll
                            for (int a = 0; a < K; ++a) v[a] = vget<T>(av[a], j);
                        }
                    }
                    warp_commit<T, K>(sp.st, A, b, v, agg, slot);
                }
            }
            s0 = g1 * VN;
        }
    }
    // whole warps iterate together (warp_commit needs every lane)
    for (int64_t base = s0 + warp0; base < i1; base += blockDim.x) {
        const int64_t i = base + lane;
        int b = -1;
        T v[KC];
        if (i < i1) {
            b = binner.bin(X[i], Y[i]);
            if constexpr (K > 0) {
#pragma unroll
                for (int a = 0; a < K; ++a) v[a] = static_cast<const T*>(sp.a[a])[i];
            } else if constexpr (K < 0) {
                for (int a = 0; a < A; ++a) v[a] = static_cast<const T*>(sp.a[a])[i];
            }
        }
        warp_commit<T, K>(sp.st, A, b, v, agg, slot);
    }
}

// All specs of one launch have K attributes (the host groups them).
template <typename T, int K>
__global__ void __launch_bounds__(256, 2) k_bin_multi(const MultiSpec* __restrict__ specs, int n_specs,
                                                   int64_t n) {
    // every spec's binner, built once per CTA
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ MultiSpec cur;
    // count-and-sums records (StateDesc::rec): each thread's staging slot
    constexpr int RDS = K >= 1 ? ((K + 2) & ~1) : 2;
    __shared__ __align__(16) double rec_slots[256 * RDS];
    Binner<T>* binners = reinterpret_cast<Binner<T>*>(smem);
    for (int s = threadIdx.x; s < n_specs; s += blockDim.x) {
        const GridDesc g = *specs[s].grid;
        Binner<T> bnr;
        if (g.valid) bnr.init(g);
        else bnr.rx = -1;  // marks an invalid mesh: the spec is skipped
        binners[s] = bnr;
    }
    __syncthreads();
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
            multi_tile<T, K>(cur, binner, i0, i1, (K >= 1 && cur.st.rec) ? rec_slots + threadIdx.x * RDS : nullptr);
        }
    }
    if (K >= 1) record_drain();
}

template <typename T, int K>
static void launch_group(const KernelCtx& kc, const MultiSpec* specs, int n_specs, int64_t n, int grid) {
    k_bin_multi<T, K><<<grid, 256, sizeof(Binner<T>) * n_specs, kc.stream>>>(specs, n_specs, n);
}

template <typename T>
static void launch_group_k(const KernelCtx& kc, int k, const MultiSpec* specs, int n_specs, int64_t n,
                           int grid) {
    switch (k) {
        case 0: launch_group<T, 0>(kc, specs, n_specs, n, grid); break;
        case 1: launch_group<T, 1>(kc, specs, n_specs, n, grid); break;
        case 2: launch_group<T, 2>(kc, specs, n_specs, n, grid); break;
        case 3: launch_group<T, 3>(kc, specs, n_specs, n, grid); break;
        case 4: launch_group<T, 4>(kc, specs, n_specs, n, grid); break;
        case 5: launch_group<T, 5>(kc, specs, n_specs, n, grid); break;
        case 6: launch_group<T, 6>(kc, specs, n_specs, n, grid); break;
        case 7: launch_group<T, 7>(kc, specs, n_specs, n, grid); break;
        case 8: launch_group<T, 8>(kc, specs, n_specs, n, grid); break;
        case 9: launch_group<T, 9>(kc, specs, n_specs, n, grid); break;
        case 10: launch_group<T, 10>(kc, specs, n_specs, n, grid); break;
        default: launch_group<T, -1>(kc, specs, n_specs, n, grid); break;
    }
}

cudaError_t launch_bin_multi(const KernelCtx& kc, int dtype, const MultiSpec* dev_specs,
                             const int* group_attrs, const int* group_size, int n_groups, int64_t n) {
    if (n <= 0 || n_groups <= 0) return cudaSuccess;
    int64_t grid = (n + kMultiTile - 1) / kMultiTile;
    // 2 CTAs per SM: a tile's columns (kMultiTile x columns x 8 B) stay within
    // a CTA's share of L2 between the specs that read them (measured at 2^22
    // f64 particles, 13 columns: 1, 2 and 4 CTAs per SM took 5.14, 4.43 and
    // 4.45 ms for 9 x 10 binnings on 256^2 meshes)
    const int64_t cap = (int64_t)kc.num_sms * 2;
    if (grid > cap) grid = cap;
    const MultiSpec* p = dev_specs;
    for (int g = 0; g < n_groups; ++g) {
        if (dtype == BN_F64) launch_group_k<double>(kc, group_attrs[g], p, group_size[g], n, (int)grid);
        else launch_group_k<float>(kc, group_attrs[g], p, group_size[g], n, (int)grid);
        kc.count_launch();
        p += group_size[g];
    }
    return cudaGetLastError();
}

}  // namespace bn
