// k_batch.cu -- K4: many independent binning problems in one persistent
// launch (Sec. 4.3 runs 90 binning operations, 10 variables x 9 coordinate
// systems, after every simulation step; here each "block" is one such
// operation with its own columns, mesh and outputs).
//
// The host planner (batch.cu) cuts every block into work items of `tile`
// particles and chooses a strategy per block (its autotuner). Persistent
// CTAs pull items from one queue:
//   private items: clear a shared-memory copy of the block's mesh, stream
//     the item's particles into it, merge it into the block's outputs (a
//     mesh larger than shared memory is cut into bands of rows, one item per
//     band and tile, each skipping the particles of other bands);
//   global items: stream the item's particles straight into the block's
//     global mesh with (optionally warp-aggregated) atomics.
// Around it, one launch each initialises all meshes, builds all f64 edge
// tables and finalises all averages, so a batch is four launches whatever
// the number of blocks; the host captures them in a CUDA graph.
#include <cuda_runtime.h>

#include "bn_device.cuh"
#include "bn_internal.cuh"
#include "bn_kernels.h"

namespace bn {

// --------------------------------------------------------------- init / fin
// One thread per (block, bin) pair, blocks laid end to end: bin_start[k]
// is the first flat index of block k (exclusive scan of bins).
__device__ __forceinline__ int find_block(const int64_t* start, int nblk, int64_t i) {
    int lo = 0, hi = nblk;  // start[lo] <= i < start[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

template <typename T>
__global__ void k_batch_init(const BatchBlock* blocks, const int64_t* bin_start, int nblk) {
    const int64_t total = bin_start[nblk];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int k = find_block(bin_start, nblk, i);
        const BatchBlock& bb = blocks[k];
        const int64_t b = i - bin_start[k];
        bb.st.count[b] = 0ull;
        for (int a = 0; a < bb.st.n_attrs; ++a) {
            if (bb.st.do_sum) bb.st.sum[a][b] = 0.0;
            if (bb.st.do_min) static_cast<T*>(bb.st.mn[a])[b] = pos_inf<T>();
            if (bb.st.do_max) static_cast<T*>(bb.st.mx[a])[b] = neg_inf<T>();
        }
    }
}

__global__ void k_batch_finalize(const BatchBlock* blocks, const int64_t* bin_start, int nblk) {
    const int64_t total = bin_start[nblk];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int k = find_block(bin_start, nblk, i);
        const BatchBlock& bb = blocks[k];
        if (!bb.st.do_avg) continue;
        const int64_t b = i - bin_start[k];
        const unsigned long long c = bb.st.count[b];
        for (int a = 0; a < bb.st.n_attrs; ++a)
            bb.st.avg[a][b] = c ? bin_average(bb.st.sum[a][b], c) : qnan;
    }
}

// Edge keys of every f64 block: one thread per (block, edge), flattened
// with edge_start (exclusive scan of res_x + res_y + 2 per block).
__global__ void k_batch_edges(BatchBlock* blocks, const int64_t* edge_start, int nblk) {
    const int64_t total = edge_start[nblk];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int k = find_block(edge_start, nblk, i);
        const BatchBlock& bb = blocks[k];
        const int64_t j = i - edge_start[k];
        const int n0 = bb.g.ax[0].res + 1;
        long long* e = const_cast<long long*>(j < n0 ? bb.g.edges[0] : bb.g.edges[1]);
        const int idx = (int)(j < n0 ? j : j - n0);
        e[idx] = edge_key(bb.g.ax[j < n0 ? 0 : 1], idx);
    }
}

// --------------------------------------------------------------- persistent
template <typename T, int A_CT, int MODE>
__global__ void __launch_bounds__(1024) k_batch_bin(const BatchBlock* blocks, const int4* items,
                                                    int n_items, int* counter, int n_attrs) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    const int A = A_CT >= 0 ? A_CT : n_attrs;
    constexpr int AC = A_CT > 0 ? A_CT : kMaxAttr;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        const int4 it = items[item];  // {block, tile index, band, -}
        const BatchBlock& bb = blocks[it.x];
        const int64_t p0 = (int64_t)it.y * bb.tile;
        const int64_t p1 = min(bb.n, p0 + bb.tile);
        Binner<T> binner;
        binner.init(bb.g);
        const T* __restrict__ X = static_cast<const T*>(bb.x);
        const T* __restrict__ Y = static_cast<const T*>(bb.y);
        const T* acol[A_CT > 0 ? A_CT : kMaxAttr];
        for (int a = 0; a < A; ++a) acol[a] = static_cast<const T*>(bb.a[a]);
        if (bb.strategy == BN_STRATEGY_PRIVATE && bb.bands > 1) {
            // one band of the mesh (rows r0 .. r0 + nrows): every particle
            // of the tile is located, those of other bands are skipped
            // before their attributes are read
            SmemMesh<T, MODE> m;
            const int rx = bb.g.ax[0].res, ry = bb.g.ax[1].res;
            const int r0 = it.z * bb.band_rows;
            const int nrows = min(bb.band_rows, ry - r0);
            const int B = nrows * rx, base = r0 * rx;
            m.carve(smem, B, A, bb.st.do_sum != 0, bb.st.do_min != 0, bb.st.do_max != 0);
            m.clear(A);
            __syncthreads();
            if (MODE == kSumLimbs && bb.st.do_sum) {
                const int64_t i = p0 + threadIdx.x;
                if (i < p1)
                    for (int a = 0; a < A; ++a) m.sample(a, acol[a][i]);
                m.bind_fallback(bb.st.sum, base);
                __syncthreads();
            }
            const int64_t step = blockDim.x;
            for (int64_t i0 = p0 + threadIdx.x; i0 < p1; i0 += 4 * step) {
                T xs[4], ys[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t i = i0 + u * step;
                    xs[u] = i < p1 ? __ldcs(X + i) : T(0);
                    ys[u] = i < p1 ? __ldcs(Y + i) : T(0);
                }
                int l[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int b = i0 + u * step < p1 ? binner.bin(xs[u], ys[u]) : -1;
                    l[u] = (b >= base && b < base + B) ? b - base : -1;
                }
                constexpr int AF = A_CT > 0 ? A_CT : 1;
                T vs[4][AF];
                if (A_CT > 0) {
#pragma unroll
                    for (int a = 0; a < AF; ++a)
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (l[u] >= 0) vs[u][a] = __ldcs(acol[a] + i0 + u * step);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (l[u] < 0) continue;
                    m.add_count(l[u]);
                    if (A_CT > 0) {
#pragma unroll
                        for (int a = 0; a < AF; ++a) m.add(a, l[u], vs[u][a]);
                    } else {
                        for (int a = 0; a < A; ++a) m.add(a, l[u], acol[a][i0 + u * step]);
                    }
                }
            }
            __syncthreads();
            m.merge(bb.st, A, base, B);
            __syncthreads();
        } else if (bb.strategy == BN_STRATEGY_PRIVATE) {
            SmemMesh<T, MODE> m;
            const int B = bb.g.ax[0].res * bb.g.ax[1].res;
            m.carve(smem, B, A, bb.st.do_sum != 0, bb.st.do_min != 0, bb.st.do_max != 0);
            m.clear(A);
            __syncthreads();
            if (MODE == kSumLimbs && bb.st.do_sum) {
                // the window of the limb sums: the item's first particles
                // (an item holds at most kLimbMaxAdds particles)
                const int64_t i = p0 + threadIdx.x;
                if (i < p1)
                    for (int a = 0; a < A; ++a) m.sample(a, acol[a][i]);
                m.bind_fallback(bb.st.sum, 0);
                __syncthreads();
            }
            // coalesced scalar loads, four particles in flight per thread
            const int64_t step = blockDim.x;
            int64_t i = p0 + threadIdx.x;
            for (; i + 3 * step < p1; i += 4 * step) {
                T xs[4], ys[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    xs[u] = __ldcs(X + i + u * step);
                    ys[u] = __ldcs(Y + i + u * step);
                }
                constexpr int AF = A_CT > 0 ? A_CT : 1;
                T vs[4][AF];
                if (A_CT > 0) {
#pragma unroll
                    for (int a = 0; a < AF; ++a)
#pragma unroll
                        for (int u = 0; u < 4; ++u) vs[u][a] = __ldcs(acol[a] + i + u * step);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int b = binner.bin(xs[u], ys[u]);
                    if (b < 0) continue;
                    m.add_count(b);
                    if (A_CT > 0) {
#pragma unroll
                        for (int a = 0; a < AF; ++a) m.add(a, b, vs[u][a]);
                    } else {
                        for (int a = 0; a < A; ++a) m.add(a, b, acol[a][i + u * step]);
                    }
                }
            }
            for (; i < p1; i += step) {
                const int b = binner.bin(X[i], Y[i]);
                if (b < 0) continue;
                m.add_count(b);
                for (int a = 0; a < A; ++a) m.add(a, b, acol[a][i]);
            }
            __syncthreads();
            m.merge(bb.st, A);
            __syncthreads();
        } else {
            // global atomics; warps walk the item together (warp_commit needs
            // every lane)
            const int lane = threadIdx.x & 31;
            for (int64_t base = p0 + (threadIdx.x - lane); base < p1; base += blockDim.x) {
                const int64_t i = base + lane;
                T v[AC];
                int b = -1;
                if (i < p1) {
                    b = binner.bin(__ldcs(X + i), __ldcs(Y + i));
                    for (int a = 0; a < A; ++a) v[a] = __ldcs(acol[a] + i);
                } else {
                    for (int a = 0; a < A; ++a) v[a] = T(0);
                }
                warp_commit<T, A_CT>(bb.st, A, b, v, bb.aggregate != 0);
            }
        }
    }
}

// --------------------------------------------------------------- launchers
static int grid_cap(int64_t work, int block, int cap) {
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

cudaError_t launch_batch_prepare(const KernelCtx& kc, int dtype, BatchBlock* dev_blocks,
                                 const int64_t* dev_bin_start, const int64_t* dev_edge_start,
                                 int nblk, int64_t total_bins, int64_t total_edges) {
    if (dtype == BN_F64)
        k_batch_init<double><<<grid_cap(total_bins, 256, kc.num_sms * 8), 256, 0, kc.stream>>>(
            dev_blocks, dev_bin_start, nblk);
    else
        k_batch_init<float><<<grid_cap(total_bins, 256, kc.num_sms * 8), 256, 0, kc.stream>>>(
            dev_blocks, dev_bin_start, nblk);
    kc.count_launch();
    if (dtype == BN_F64 && total_edges > 0) {
        k_batch_edges<<<grid_cap(total_edges, 128, kc.num_sms * 4), 128, 0, kc.stream>>>(
            dev_blocks, dev_edge_start, nblk);
        kc.count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const KernelCtx& kc, const BatchBlock* dev_blocks,
                                  const int64_t* dev_bin_start, int nblk, int64_t total_bins) {
    k_batch_finalize<<<grid_cap(total_bins, 256, kc.num_sms * 8), 256, 0, kc.stream>>>(
        dev_blocks, dev_bin_start, nblk);
    kc.count_launch();
    return cudaGetLastError();
}

template <typename T, int A_CT, int MODE>
static cudaError_t launch_batch_bin_t(const KernelCtx& kc, const BatchBlock* blocks, const int4* items,
                                      int n_items, int* counter, int n_attrs, size_t smem) {
    auto kern = k_batch_bin<T, A_CT, MODE>;
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(kern), kc.smem_optin);
    if (e != cudaSuccess) return e;
    const int block = 1024;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = kc.num_sms * per_sm;
    if (grid > n_items) grid = n_items > 0 ? n_items : 1;
    kern<<<grid, block, smem, kc.stream>>>(blocks, items, n_items, counter, n_attrs);
    kc.count_launch();
    return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t dispatch_batch(const KernelCtx& kc, const BatchBlock* blocks, const int4* items,
                                  int n_items, int* counter, int n_attrs, size_t smem) {
    switch (n_attrs) {
        case 0: return launch_batch_bin_t<T, 0, MODE>(kc, blocks, items, n_items, counter, n_attrs, smem);
        case 1: return launch_batch_bin_t<T, 1, MODE>(kc, blocks, items, n_items, counter, n_attrs, smem);
        case 2: return launch_batch_bin_t<T, 2, MODE>(kc, blocks, items, n_items, counter, n_attrs, smem);
        case 3: return launch_batch_bin_t<T, 3, MODE>(kc, blocks, items, n_items, counter, n_attrs, smem);
        case 4: return launch_batch_bin_t<T, 4, MODE>(kc, blocks, items, n_items, counter, n_attrs, smem);
        default: return launch_batch_bin_t<T, -1, MODE>(kc, blocks, items, n_items, counter, n_attrs, smem);
    }
}

cudaError_t launch_batch_bin(const KernelCtx& kc, int dtype, int sum_mode, const BatchBlock* blocks,
                             const int4* items, int n_items, int* counter, int n_attrs, size_t smem) {
    if (dtype == BN_F64) return dispatch_batch<double, kSumF64>(kc, blocks, items, n_items, counter, n_attrs, smem);
    if (smem_sum_mode(dtype, sum_mode) == kSumF32)
        return dispatch_batch<float, kSumF32>(kc, blocks, items, n_items, counter, n_attrs, smem);
    return dispatch_batch<float, kSumLimbs>(kc, blocks, items, n_items, counter, n_attrs, smem);
}

}  // namespace bn
