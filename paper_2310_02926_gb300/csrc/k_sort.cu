// k_sort.cu -- K2: sort by bin (bucketed) + privatised reduction, for meshes
// too large for one CTA's shared memory.
//
// Sec. 4.2 reduces every particle into its mesh cell; on a large mesh the
// direct way is one global atomic per particle and reduction (Sec. 4.4 names
// these atomics as binning's GPU cost), which on GB300 runs at the speed of
// L2's atomic units and serialises on dense cells. Instead:
//
//   pass 1 (k_sort_scatter): each CTA takes a tile of TP particles, locates
//     each particle's bin, counting-sorts the tile in shared memory by
//     bucket (a bucket is a run of BK consecutive bins, small enough that
//     its state fits one CTA's shared memory) and writes the tile's records
//     (u16 bin within the bucket + attributes) contiguously, bucket after
//     bucket, plus one row of bucket offsets for the tile;
//   plan (k_sort_plan): per bucket, split its tiles into work items of about
//     `chunk` records (dense buckets get several items);
//   pass 2 (k_sort_reduce): persistent CTAs take items, gather the item's
//     records segment by segment into a shared-memory mesh of the bucket
//     (shared-memory atomics only), then store the bucket's bins (an item
//     that holds a whole bucket) or merge them with global atomics.
//
// Every particle is read once in pass 1 and its record is written once and
// read once; global atomics happen only per (split item, bin).
#include <cuda_runtime.h>

#include <cstring>

#include "bn_device.cuh"
#include "bn_internal.cuh"
#include "bn_kernels.h"

namespace bn {

// Block-wide exclusive scan of one int per thread; returns the thread's
// prefix and writes the block total to *total. `warp_sums` holds 32 ints.
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nwarps ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nwarps) warp_sums[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const int before = warp > 0 ? warp_sums[warp - 1] : 0;
    *total = warp_sums[nwarps - 1];
    __syncthreads();
    return before + x - v;
}

// ------------------------------------------------------------------ pass 1
// One tile of TP = PER * blockDim particles per CTA. Coordinates are loaded
// first (8 per thread, coalesced), each particle's bucket rank is taken with
// a shared-memory atomic, the bucket counts are scanned, and then the
// attributes are loaded and written straight to their sorted slot in shared
// memory, so registers hold only (bucket, local bin, rank) per particle and
// two CTAs fit on an SM.
template <typename T, int A_CT, int PER>
__global__ void __launch_bounds__(512) k_sort_scatter(BinArgs args, SortDesc sd) {
    extern __shared__ __align__(16) unsigned char smem[];
    // PER particles per thread: TP = PER * blockDim
    const GridDesc g = args.dev_grid ? *args.dev_grid : args.grid;
    if (!g.valid) return;
    const int A = A_CT >= 0 ? A_CT : args.n_attrs;
    const int NB = sd.nb;
    const int TP = sd.tp;
    int* hist = reinterpret_cast<int*>(smem);                       // NB + 1
    __shared__ int warp_sums[32];
    __shared__ int s_total;
    T* sattr = reinterpret_cast<T*>(smem + sd.off_sattr);           // [A][TP]
    unsigned short* skey = reinterpret_cast<unsigned short*>(smem + sd.off_skey);  // [TP]

    const int64_t tile = blockIdx.x;
    const int64_t base = tile * TP;
    const int64_t n = args.n;
    for (int k = threadIdx.x; k <= NB; k += blockDim.x) hist[k] = 0;
    Binner<T> binner;
    binner.init(g);
    __syncthreads();

    const T* __restrict__ X = static_cast<const T*>(args.x);
    const T* __restrict__ Y = static_cast<const T*>(args.y);
    int bucket[PER], slot[PER];  // slot = local bin | rank << 16, then the sorted position
    {
        const int lane = threadIdx.x & 31;
        const unsigned lt = (1u << lane) - 1u;
        // coordinates in groups of 8 per thread, so only the bucket and slot
        // of each particle stay in registers
#pragma unroll
        for (int j0 = 0; j0 < PER; j0 += 8) {
            T xv[8], yv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t p = base + (j0 + u) * blockDim.x + threadIdx.x;
                xv[u] = p < n ? __ldcs(X + p) : T(0);
                yv[u] = p < n ? __ldcs(Y + p) : T(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u;
                const int64_t p = base + j * blockDim.x + threadIdx.x;
                const int b = p < n ? binner.bin(xv[u], yv[u]) : -1;
                bucket[j] = b < 0 ? -1 : (b >> sd.log2bk);
                // one shared atomic per distinct bucket in the warp: the lowest
                // lane of each group reserves the group's ranks
                const unsigned peers = __match_any_sync(0xffffffffu, bucket[j]);
                const int leader = __ffs(peers) - 1;
                int r0 = 0;
                if (lane == leader && bucket[j] >= 0) r0 = atomicAdd(&hist[bucket[j]], __popc(peers));
                r0 = __shfl_sync(0xffffffffu, r0, leader);
                const int r = r0 + __popc(peers & lt);
                slot[j] = (b & ((1 << sd.log2bk) - 1)) | (r << 16);
            }
        }
    }
    __syncthreads();
    // exclusive scan of the bucket counts, NB + 1 entries (the last is 0)
    {
        const int per = (NB + 1 + blockDim.x - 1) / blockDim.x;
        const int k0 = threadIdx.x * per;
        int loc = 0;
        for (int k = k0; k < k0 + per && k <= NB; ++k) loc += hist[k];
        int pre = block_exclusive_scan(loc, warp_sums, &s_total);
        for (int k = k0; k < k0 + per && k <= NB; ++k) {
            int c = hist[k];
            hist[k] = pre;
            pre += c;
        }
    }
    __syncthreads();
    const int n_in = hist[NB];
    // this tile's row of bucket offsets, and per-bucket totals for planning
    int* row = sd.table + tile * (int64_t)(NB + 1);
    for (int k = threadIdx.x; k <= NB; k += blockDim.x) {
        const int o = hist[k];
        row[k] = o;
        if (k < NB) {
            const int c = hist[k + 1] - o;
            if (c) atomicAdd(&sd.bucket_total[k], c);
        }
    }
    // sorted position of each particle (reusing slot); keys now, attributes
    // column by column in groups of 8
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int pos = bucket[j] < 0 ? -1 : hist[bucket[j]] + (slot[j] >> 16);
        if (pos >= 0) skey[pos] = (unsigned short)(slot[j] & 0xffff);
        slot[j] = pos;
    }
    for (int a = 0; a < A; ++a) {
        const T* __restrict__ col = static_cast<const T*>(args.a[a]);
#pragma unroll
        for (int j0 = 0; j0 < PER; j0 += 8) {
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t p = base + (j0 + u) * blockDim.x + threadIdx.x;
                v[u] = slot[j0 + u] >= 0 ? __ldcs(col + p) : T(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (slot[j0 + u] >= 0) sattr[a * TP + slot[j0 + u]] = v[u];
        }
    }
    __syncthreads();
    // records out, coalesced
    unsigned short* okey = sd.keys + base;
    for (int i = threadIdx.x; i < n_in; i += blockDim.x) okey[i] = skey[i];
    for (int a = 0; a < A; ++a) {
        T* oa = static_cast<T*>(sd.attrs) + (int64_t)a * sd.slots + base;
        for (int i = threadIdx.x; i < n_in; i += blockDim.x) oa[i] = sattr[a * TP + i];
    }
}

// Transpose the [tiles][nb + 1] offset table to [nb + 1][tiles] so pass 2
// reads each bucket's offsets contiguously. 32 x 32 tiles through shared
// memory, both sides coalesced.
__global__ void k_sort_transpose(SortDesc sd) {
    __shared__ int t[32][33];
    const int64_t rows = sd.tiles, cols = sd.nb + 1;
    // blockIdx.x walks tiles (can be many), blockIdx.y walks buckets
    const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[i][threadIdx.x] = sd.table[r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) sd.table_t[c * rows + r] = t[threadIdx.x][i];
    }
}

// ------------------------------------------------------------------ plan
// One block: bucket totals -> work items {bucket, first tile, end tile, sole}.
__global__ void k_sort_plan(SortDesc sd) {
    __shared__ int warp_sums[32];
    __shared__ int s_total;
    const int NB = sd.nb;
    const int per = (NB + blockDim.x - 1) / blockDim.x;
    const int k0 = threadIdx.x * per;
    int mine = 0;
    for (int k = k0; k < k0 + per && k < NB; ++k) {
        const int c = sd.bucket_total[k];
        mine += (c + sd.chunk - 1) / sd.chunk;
    }
    int off = block_exclusive_scan(mine, warp_sums, &s_total);
    for (int k = k0; k < k0 + per && k < NB; ++k) {
        const int c = sd.bucket_total[k];
        const int parts = (c + sd.chunk - 1) / sd.chunk;
        for (int j = 0; j < parts; ++j) {
            int4 it;
            it.x = k;
            it.y = (int)((int64_t)j * sd.tiles / parts);
            it.z = (int)((int64_t)(j + 1) * sd.tiles / parts);
            it.w = parts == 1 ? 1 : 0;
            sd.items[off + j] = it;
        }
        off += parts;
    }
    if (threadIdx.x == 0) sd.counters[0] = s_total;
}

// ------------------------------------------------------------------ pass 2
// Persistent CTAs take work items. For an item (bucket k, tiles [t0, t1))
// each warp takes 32 consecutive tiles at a time: lane i reads tile i's
// segment of bucket k from the transposed table, the warp scans the 32
// lengths, and the lanes then walk the concatenated records (each finds its
// segment with a 5-step search over the scanned lengths held in registers).
template <typename T, int A_CT, int MODE>
__global__ void __launch_bounds__(1024) k_sort_reduce(BinArgs args, SortDesc sd) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    const int A = A_CT >= 0 ? A_CT : args.n_attrs;
    const int BK = 1 << sd.log2bk;
    const int64_t B = args.st.bins;
    const int64_t T_ = sd.tiles;
    SmemMesh<T, MODE> m;
    m.carve(smem + sd.off_mesh, BK, A, args.st.do_sum != 0, args.st.do_min != 0,
            args.st.do_max != 0);
    const unsigned short* __restrict__ keys = sd.keys;
    const T* __restrict__ attrs = static_cast<const T*>(sd.attrs);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&sd.counters[1], 1);
        __syncthreads();
        const int item = s_item;
        if (item >= sd.counters[0]) break;
        const int4 it = sd.items[item];
        const int k = it.x;
        m.clear(A);
        __syncthreads();
        const int* __restrict__ off0 = sd.table_t + (int64_t)k * T_;
        const int* __restrict__ off1 = off0 + T_;
        for (int tb = it.y + warp * 32; tb < it.z; tb += nwarps * 32) {
            const int t = tb + lane;
            int first = 0, len = 0;
            if (t < it.z) {
                first = off0[t];
                len = off1[t] - first;
            }
            int incl = len;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            const int excl = incl - len;
            const int64_t seg_base = (int64_t)t * sd.tp + first;  // record index of the segment start
            for (int r0 = 0; r0 < total; r0 += 32) {
                const int r = r0 + lane;
                // lane holding the segment of record r: last s with excl_s <= r
                int s = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int e = __shfl_sync(0xffffffffu, excl, s + step);
                    if (e <= r) s += step;
                }
                const int64_t sb = __shfl_sync(0xffffffffu, seg_base, s);
                const int se = __shfl_sync(0xffffffffu, excl, s);
                if (r < total) {
                    const int64_t idx = sb + (r - se);
                    const int l = keys[idx];
                    m.add_count(l);
                    for (int a = 0; a < A; ++a) m.add(a, l, attrs[(int64_t)a * sd.slots + idx]);
                }
            }
        }
        __syncthreads();
        const int64_t bin0 = (int64_t)k * BK;
        const int nbins = (int)((B - bin0) < BK ? (B - bin0) : BK);
        m.merge(args.st, A, bin0, nbins, it.w != 0);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host side
static size_t mesh_bytes(int dtype, int mode, int bins, int A, bool s, bool lo, bool hi) {
    const bool wide = dtype == BN_F64 || mode == kSumF64;
    const size_t tsz = dtype == BN_F64 ? 8 : 4;
    size_t b = ((size_t)bins * 4 + 15) & ~(size_t)15;
    if (s) b += (size_t)A * bins * (wide ? 8 : (mode == kSumF32C ? 8 : 4));
    b = (b + 15) & ~(size_t)15;
    if (lo || hi) b += (size_t)A * bins * 2 * tsz;  // {min key, max key}
    return b;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool sort_plan(const BinArgs& a, int smem_optin_total, SortDesc* sd) {
    const int smem_optin = smem_optin_total - 1024;  // room for the kernels' static shared memory
    const int64_t B = (int64_t)a.grid.ax[0].res * a.grid.ax[1].res;
    const int mode = a.dtype == BN_F64 ? kSumF64 : a.sum_mode;
    const size_t tsz = a.dtype == BN_F64 ? 8 : 4;
    const size_t seg_bytes = 256;
    // largest power-of-two bucket whose shared-memory mesh fits
    int log2bk = 16;
    while (log2bk > 5 && seg_bytes + mesh_bytes(a.dtype, mode, 1 << log2bk, a.n_attrs, a.st.do_sum,
                                                 a.st.do_min, a.st.do_max) > (size_t)smem_optin)
        --log2bk;
    while (log2bk > 5 && ((int64_t)1 << (log2bk - 1)) >= B) --log2bk;
    if (seg_bytes + mesh_bytes(a.dtype, mode, 1 << log2bk, a.n_attrs, a.st.do_sum, a.st.do_min,
                               a.st.do_max) > (size_t)smem_optin)
        return false;
    const int64_t nb = (B + (1 << log2bk) - 1) >> log2bk;
    if (nb > 8192) return false;
    // tile: as large as shared memory allows (up to 16384 particles, 32 per
    // thread of a 512-thread block), so the per-tile bucket table stays
    // small next to the records; at least 4096 when it fits
    auto scatter_bytes = [&](int tp_) {
        return align256((size_t)(nb + 1) * 4) + align256((size_t)tp_ * 2) + (size_t)a.n_attrs * tp_ * tsz;
    };
    // smallest tile from 4096 up whose bucket table stays under a quarter of
    // the tile's record bytes, then shrunk to what shared memory holds
    const double rec = 2.0 + (double)a.n_attrs * tsz;
    int tp = 4096;
    while (tp < 16384 && (double)(nb + 1) * 4.0 > 0.25 * rec * tp) tp <<= 1;
    while (tp > 512 && scatter_bytes(tp) > (size_t)smem_optin) tp >>= 1;
    if (scatter_bytes(tp) > (size_t)smem_optin) return false;
    memset(sd, 0, sizeof *sd);
    sd->log2bk = log2bk;
    sd->nb = (int)nb;
    sd->tp = tp;
    sd->tiles = (a.n + tp - 1) / tp;
    sd->slots = sd->tiles * tp;
    sd->chunk = 1 << 16;
    sd->off_skey = (int)align256((size_t)(nb + 1) * 4);
    sd->off_sattr = sd->off_skey + (int)align256((size_t)tp * 2);
    sd->smem_scatter = (size_t)sd->off_sattr + (size_t)a.n_attrs * tp * tsz;
    sd->per = tp >= 16384 ? 32 : tp >= 8192 ? 16 : 8;
    sd->off_mesh = (int)seg_bytes;
    sd->smem_reduce = seg_bytes + mesh_bytes(a.dtype, mode, 1 << log2bk, a.n_attrs, a.st.do_sum,
                                             a.st.do_min, a.st.do_max);
    sd->max_items = nb + (a.n + sd->chunk - 1) / sd->chunk + 1;
    return true;
}

size_t sort_scratch_bytes(const SortDesc& sd, const BinArgs& a) {
    const size_t tsz = a.dtype == BN_F64 ? 8 : 4;
    size_t b = 0;
    b += align256((size_t)sd.slots * 2);                       // keys
    b += align256((size_t)sd.slots * tsz * (a.n_attrs ? a.n_attrs : 1));  // attributes
    b += 2 * align256((size_t)sd.tiles * (sd.nb + 1) * 4);     // offset table, and transposed
    b += align256((size_t)sd.nb * 4);                          // bucket totals
    b += align256((size_t)sd.max_items * 16);                  // items
    b += 256;                                                  // counters
    return b;
}

template <typename T, int A_CT, int MODE>
static cudaError_t launch_sort_t(const KernelCtx& kc, const BinArgs& a, const SortDesc& sd) {
    auto scat = sd.per == 32 ? k_sort_scatter<T, A_CT, 32>
              : sd.per == 16 ? k_sort_scatter<T, A_CT, 16> : k_sort_scatter<T, A_CT, 8>;
    auto red = k_sort_reduce<T, A_CT, MODE>;
    static bool configured[3] = {false, false, false};
    const int ci = sd.per == 32 ? 2 : sd.per == 16 ? 1 : 0;
    if (!configured[ci]) {
        // the opt-in limit covers static plus dynamic shared memory
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, scat);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(scat, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kc.smem_optin - (int)fa.sharedSizeBytes);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, red);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(red, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kc.smem_optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
        configured[ci] = true;
    }
    scat<<<(unsigned)sd.tiles, sd.tp / sd.per, sd.smem_scatter, kc.stream>>>(a, sd);
    {
        dim3 tb(32, 8);
        dim3 tg((unsigned)((sd.tiles + 31) / 32), (unsigned)((sd.nb + 1 + 31) / 32));
        k_sort_transpose<<<tg, tb, 0, kc.stream>>>(sd);
    }
    k_sort_plan<<<1, 1024, 0, kc.stream>>>(sd);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, red, 1024, sd.smem_reduce);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)kc.num_sms * per_sm;
    if (grid > sd.max_items) grid = sd.max_items;
    red<<<(unsigned)grid, 1024, sd.smem_reduce, kc.stream>>>(a, sd);
    kc.count_launch(4);
    return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t dispatch_sort(const KernelCtx& kc, const BinArgs& a, const SortDesc& sd) {
    switch (a.n_attrs) {
        case 0: return launch_sort_t<T, 0, MODE>(kc, a, sd);
        case 1: return launch_sort_t<T, 1, MODE>(kc, a, sd);
        case 2: return launch_sort_t<T, 2, MODE>(kc, a, sd);
        case 3: return launch_sort_t<T, 3, MODE>(kc, a, sd);
        case 4: return launch_sort_t<T, 4, MODE>(kc, a, sd);
        default: return launch_sort_t<T, -1, MODE>(kc, a, sd);
    }
}

cudaError_t launch_bin_sort(const KernelCtx& kc, const BinArgs& a, SortDesc sd, void* scratch) {
    const size_t tsz = a.dtype == BN_F64 ? 8 : 4;
    unsigned char* p = static_cast<unsigned char*>(scratch);
    sd.keys = reinterpret_cast<unsigned short*>(p);
    p += align256((size_t)sd.slots * 2);
    sd.attrs = p;
    p += align256((size_t)sd.slots * tsz * (a.n_attrs ? a.n_attrs : 1));
    sd.table = reinterpret_cast<int*>(p);
    p += align256((size_t)sd.tiles * (sd.nb + 1) * 4);
    sd.table_t = reinterpret_cast<int*>(p);
    p += align256((size_t)sd.tiles * (sd.nb + 1) * 4);
    sd.bucket_total = reinterpret_cast<int*>(p);
    p += align256((size_t)sd.nb * 4);
    sd.items = reinterpret_cast<int4*>(p);
    p += align256((size_t)sd.max_items * 16);
    sd.counters = reinterpret_cast<int*>(p);
    cudaError_t e = cudaMemsetAsync(sd.bucket_total, 0, (size_t)sd.nb * 4, kc.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sd.counters, 0, 256, kc.stream);
    if (e != cudaSuccess) return e;
    if (a.dtype == BN_F64) return dispatch_sort<double, kSumF64>(kc, a, sd);
    switch (a.sum_mode) {
        case kSumF32: return dispatch_sort<float, kSumF32>(kc, a, sd);
        case kSumF64: return dispatch_sort<float, kSumF64>(kc, a, sd);
        default: return dispatch_sort<float, kSumF32C>(kc, a, sd);
    }
}

}  // namespace bn
