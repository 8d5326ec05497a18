// k_sort.cu -- K2: bucketed counting sort + privatised reduction, for meshes
// too large for one CTA's shared memory.
//
// Sec. 4.2 reduces every particle into its mesh cell; on a large mesh the
// direct way is one global atomic per particle and reduction (Sec. 4.4 names
// these atomics as binning's GPU cost), which on GB300 runs at the speed of
// L2's atomic units, or of DRAM once the mesh state outgrows L2. Instead the
// mesh is cut into buckets of BK consecutive bins, few enough that a
// bucket's state fits one CTA's shared memory, and:
//
//   count (k_sort_count): every particle's bucket; records per bucket;
//   plan (k_sort_plan): each bucket's first record slot (exclusive scan) and
//     work items of at most `chunk` consecutive records of one bucket;
//   pass 1 (k_sort_scatter): each CTA takes a tile of TP particles,
//     counting-sorts it by bucket in shared memory, reserves its run in each
//     bucket it feeds with one global atomic, and writes its records (u16
//     bin within the bucket + attributes) there: every bucket's records end
//     up contiguous;
//   pass 2 (k_sort_reduce): persistent CTAs take items and stream the item's
//     records into a shared-memory mesh of the bucket (shared-memory atomics
//     only), then store the bucket's bins (an item that holds a whole
//     bucket) or merge them with global atomics.
//
// Coordinates are read twice (count and pass 1), attributes once; a record
// is written once and read once; global atomics happen per (tile, bucket)
// and per (split item, bin). Within a bucket the records are in the order
// the tiles reserved their runs, which varies from run to run like the
// order of any atomic accumulation.
#include <cuda_runtime.h>

#include <climits>
#include <cstring>
#include <type_traits>

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

// ------------------------------------------------------------------ count
// Records per bucket: one shared-memory atomic per particle (measured
// faster on GB300 than combining a warp's lanes with __match_any_sync
// first, even on clustered data).
template <typename T>
// The kernels taking BinArgs read them from dargs when it is set (a batch
// plan's device copy, rewritten before every replay of its CUDA graph, so
// that the graph's kernel parameters do not change from call to call).
__global__ void __launch_bounds__(512) k_sort_count(BinArgs args_v, SortDesc sd, const BinArgs* dargs) {
    const BinArgs& args = dargs ? *dargs : args_v;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned* hist = reinterpret_cast<unsigned*>(smem);  // NB
    const GridDesc g = args.dev_grid ? *args.dev_grid : args.grid;
    if (!g.valid) return;
    const int NB = sd.nb;
    for (int k = threadIdx.x; k < NB; k += blockDim.x) hist[k] = 0u;
    Binner<T> binner;
    binner.init(g);
    __syncthreads();
    const T* __restrict__ X = static_cast<const T*>(args.x);
    const T* __restrict__ Y = static_cast<const T*>(args.y);
    const int64_t n = args.n;
    const int lane = threadIdx.x & 31;
    constexpr int U = 4;  // particles per thread per step, loads first
    const int64_t step = (int64_t)gridDim.x * blockDim.x * U;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * U;
    for (int64_t base = warp0; base < n; base += step) {
        T xv[U], yv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = base + u * 32 + lane;
            xv[u] = i < n ? __ldcs(X + i) : T(0);
            yv[u] = i < n ? __ldcs(Y + i) : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = base + u * 32 + lane;
            const int b = i < n ? binner.bin(xv[u], yv[u]) : -1;
            const int bk = b < 0 ? -1 : (b >> sd.log2bk);
            if (bk >= 0) atomicAdd(&hist[bk], 1u);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NB; k += blockDim.x)
        if (hist[k]) atomicAdd(&sd.bucket_total[k], hist[k]);
}

// ------------------------------------------------------------------ plan
// One block: bucket totals -> first record slot of each bucket (into the
// cursors) and work items {bucket, first record, end record, sole}. A sole
// item (the only one of its bucket) stores the bucket's bins outright,
// except when accumulating into existing outputs.
__global__ void k_sort_plan(SortDesc sd) {
    __shared__ int warp_sums[32];
    __shared__ int s_total;
    const int NB = sd.nb;
    const int per = (NB + blockDim.x - 1) / blockDim.x;
    const int k0 = threadIdx.x * per;
    int recs = 0, mine = 0;
    for (int k = k0; k < k0 + per && k < NB; ++k) {
        const int c = (int)sd.bucket_total[k];
        recs += c;
        mine += (c + sd.chunk - 1) / sd.chunk;
    }
    int rec_off = block_exclusive_scan(recs, warp_sums, &s_total);
    int off = block_exclusive_scan(mine, warp_sums, &s_total);
    for (int k = k0; k < k0 + per && k < NB; ++k) {
        const int c = (int)sd.bucket_total[k];
        sd.cursor[k] = (unsigned)rec_off;
        const int parts = (c + sd.chunk - 1) / sd.chunk;
        for (int j = 0; j < parts; ++j) {
            int4 it;
            it.x = k;
            it.y = rec_off + (int)((int64_t)j * c / parts);
            it.z = rec_off + (int)((int64_t)(j + 1) * c / parts);
            it.w = (parts == 1 && !sd.accumulate) ? 1 : 0;
            sd.items[off + j] = it;
        }
        off += parts;
        rec_off += c;
    }
    if (threadIdx.x == 0) sd.counters[0] = s_total;
}

// ------------------------------------------------------------------ pass 1
// One tile of TP = PER * blockDim particles per CTA (up to 1024 threads, at
// most 64 registers: the per-particle bucket and slot of PER particles live
// in registers). Coordinates are loaded
// first (8 per thread, coalesced), each particle's bucket rank is taken with
// a shared-memory atomic, the bucket counts are scanned, the tile's run in
// each bucket is reserved, and then the attributes are loaded and written
// straight to their sorted slot in shared memory, so registers hold only
// (bucket, local bin, rank) per particle. The sorted records then go out to
// their reserved runs. VEC (every column 16-byte aligned): a thread's
// particles come in 16-byte vectors, vector v of the tile holding particles
// v*VN .. v*VN+VN-1; otherwise one coalesced element per load.
template <typename T>
__device__ __forceinline__ void load_group8(const T* __restrict__ col, int64_t base, int j0, int64_t n,
                                            bool vec, T* out) {
    constexpr int VN = VecOf<T>::N;
    using V = typename VecOf<T>::type;
    if (vec) {
#pragma unroll
        for (int q = 0; q < 8 / VN; ++q) {
            const int64_t p0 = base + ((int64_t)(j0 / VN + q) * blockDim.x + threadIdx.x) * VN;
            if (p0 + VN <= n) {
                const V v = __ldcs(reinterpret_cast<const V*>(col + p0));
#pragma unroll
                for (int e = 0; e < VN; ++e) out[q * VN + e] = vget<T>(v, e);
            } else {
#pragma unroll
                for (int e = 0; e < VN; ++e) out[q * VN + e] = p0 + e < n ? __ldcs(col + p0 + e) : T(0);
            }
        }
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t p = base + (int64_t)(j0 + u) * blockDim.x + threadIdx.x;
            out[u] = p < n ? __ldcs(col + p) : T(0);
        }
    }
}

template <typename T, int A_CT, int PER, bool VEC>
__global__ void __launch_bounds__(1024) k_sort_scatter(BinArgs args_v, SortDesc sd, const BinArgs* dargs) {
    const BinArgs& args = dargs ? *dargs : args_v;
    extern __shared__ __align__(16) unsigned char smem[];
    const GridDesc g = args.dev_grid ? *args.dev_grid : args.grid;
    if (!g.valid) return;
    const int A = A_CT >= 0 ? A_CT : args.n_attrs;
    const int NB = sd.nb;
    const int TP = sd.tp;
    int* hist = reinterpret_cast<int*>(smem);                                       // NB + 1
    int* gpos = reinterpret_cast<int*>(smem + sd.off_gpos);                         // NB
    unsigned short* skey = reinterpret_cast<unsigned short*>(smem + sd.off_skey);  // TP
    unsigned short* sbk = reinterpret_cast<unsigned short*>(smem + sd.off_sbk);    // TP
    T* sattr = reinterpret_cast<T*>(smem + sd.off_sattr);                           // [A][TP]
    __shared__ int warp_sums[32];
    __shared__ int s_total;

    const int64_t tile = blockIdx.x;
    const int64_t base = tile * TP;
    const int64_t n = args.n;
    for (int k = threadIdx.x; k <= NB; k += blockDim.x) hist[k] = 0;
    Binner<T> binner;
    binner.init(g);
    __syncthreads();

    const T* __restrict__ X = static_cast<const T*>(args.x);
    const T* __restrict__ Y = static_cast<const T*>(args.y);
    constexpr int VN = VecOf<T>::N;
    // the particle that is this thread's j-th
    auto pidx = [&](int j) -> int64_t {
        return VEC ? base + ((int64_t)(j / VN) * blockDim.x + threadIdx.x) * VN + (j % VN)
                   : base + (int64_t)j * blockDim.x + threadIdx.x;
    };
    int bucket[PER], slot[PER];  // slot = local bin | rank << 16, then the sorted position
    {
        // coordinates in groups of 8 per thread, so only the bucket and slot
        // of each particle stay in registers
#pragma unroll
        for (int j0 = 0; j0 < PER; j0 += 8) {
            T xv[8], yv[8];
            load_group8<T>(X, base, j0, n, VEC, xv);
            load_group8<T>(Y, base, j0, n, VEC, yv);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u;
                const int64_t p = pidx(j);
                const int b = p < n ? binner.bin(xv[u], yv[u]) : -1;
                bucket[j] = b < 0 ? -1 : (b >> sd.log2bk);
                // rank within the tile's bucket: the value the shared atomic
                // returns (the order of a run does not matter)
                const int r = bucket[j] >= 0 ? atomicAdd(&hist[bucket[j]], 1) : 0;
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
    // reserve this tile's run in every bucket it feeds: sorted record i of
    // bucket k goes to slot gpos[k] + i
    // (four reservations in flight per thread: their L2 round trips overlap)
    for (int k0 = threadIdx.x; k0 < NB; k0 += 4 * blockDim.x) {
        int got[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = k0 + u * blockDim.x;
            const int c = k < NB ? hist[k + 1] - hist[k] : 0;
            got[u] = c ? (int)atomicAdd(&sd.cursor[k], (unsigned)c) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = k0 + u * blockDim.x;
            if (k < NB) gpos[k] = got[u] - hist[k];
        }
    }
    // sorted position of each particle (reusing slot); key and bucket now,
    // attributes column by column in groups of 8
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int pos = bucket[j] < 0 ? -1 : hist[bucket[j]] + (slot[j] >> 16);
        if (pos >= 0) {
            skey[pos] = (unsigned short)(slot[j] & 0xffff);
            sbk[pos] = (unsigned short)bucket[j];
        }
        slot[j] = pos;
    }
    for (int a = 0; a < A; ++a) {
        const T* __restrict__ col = static_cast<const T*>(args.a[a]);
#pragma unroll
        for (int j0 = 0; j0 < PER; j0 += 8) {
            T v[8];
            load_group8<T>(col, base, j0, n, VEC, v);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (slot[j0 + u] >= 0) sattr[a * TP + slot[j0 + u]] = v[u];
        }
    }
    __syncthreads();
    // records out to their runs (consecutive records of a run are
    // consecutive slots); a slot outside [0, slots) cannot occur when the
    // count pass saw the same particles, and is skipped
    const int64_t S = sd.slots;
    for (int i = threadIdx.x; i < n_in; i += blockDim.x) {
        const int64_t p = (int64_t)gpos[sbk[i]] + i;
        if (p < 0 || p >= S) continue;
        sd.keys[p] = skey[i];
        for (int a = 0; a < A; ++a) static_cast<T*>(sd.attrs)[(int64_t)a * S + p] = sattr[a * TP + i];
    }
}

// ------------------------------------------------------------------ pass 2
// Persistent CTAs take work items; an item's records are consecutive slots,
// streamed U per thread per step (all loads first).
template <typename T, int A_CT, int MODE>
__global__ void __launch_bounds__(1024) k_sort_reduce(BinArgs args_v, SortDesc sd, const BinArgs* dargs) {
    const BinArgs& args = dargs ? *dargs : args_v;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    const int A = A_CT >= 0 ? A_CT : args.n_attrs;
    constexpr int AC = A_CT > 0 ? A_CT : (A_CT == 0 ? 1 : kMaxAttr);
    constexpr int U = (A_CT >= 0 && A_CT <= 4) ? 4 : 1;
    const int BK = 1 << sd.log2bk;
    const int64_t B = args.st.bins;
    const int64_t S = sd.slots;
    SmemMesh<T, MODE> m;
    m.carve(smem, BK, A, args.st.do_sum != 0, args.st.do_min != 0, args.st.do_max != 0);
    const unsigned short* __restrict__ keys = sd.keys;
    const T* __restrict__ attrs = static_cast<const T*>(sd.attrs);
    constexpr bool kLimbs = MODE == kSumLimbs;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&sd.counters[1], 1);
        __syncthreads();
        const int item = s_item;
        if (item >= sd.counters[0]) break;
        const int4 it = sd.items[item];
        m.clear(A);
        if (kLimbs) m.bind_fallback(args.st.sum, (int64_t)it.x * BK);
        __syncthreads();
        if (kLimbs && args.st.do_sum) {
            // the window of the limb sums: the item's first records
            const int r = it.y + (int)threadIdx.x;
            if (r < it.z)
                for (int a = 0; a < A; ++a) m.sample(a, attrs[(int64_t)a * S + r]);
            __syncthreads();
        }
        if constexpr (A_CT >= 0 && A_CT <= 4) {
            // 16-byte loads: groups of VN records (the record planes start
            // on 16-byte boundaries, S being a multiple of 32); the records
            // before the first and after the last whole group one by one
            constexpr int VN = VecOf<T>::N;
            constexpr int G = 2;  // groups per thread per step, loads first
            using V = typename VecOf<T>::type;
            using KV = typename std::conditional<VN == 4, uint2, unsigned>::type;
            const int y = it.y, z = it.z;
            const int vb = min(z, (y + VN - 1) / VN * VN);
            const int ve = max(vb, z / VN * VN);
            auto one = [&](int r) {
                const int l = (int)__ldcs(keys + r);
                m.add_count(l);
#pragma unroll
                for (int a = 0; a < A_CT; ++a) m.add(a, l, __ldcs(attrs + (int64_t)a * S + r));
            };
            for (int r = y + (int)threadIdx.x; r < vb; r += blockDim.x) one(r);
            for (int r = ve + (int)threadIdx.x; r < z; r += blockDim.x) one(r);
            const int ng = (ve - vb) / VN;
            const KV* KG = reinterpret_cast<const KV*>(keys + vb);
            const V* AG[AC];
#pragma unroll
            for (int a = 0; a < AC; ++a) AG[a] = reinterpret_cast<const V*>(attrs + (int64_t)(a < A_CT ? a : 0) * S + vb);
            for (int g0 = threadIdx.x; g0 < ng; g0 += G * blockDim.x) {
                KV kk[G];
                V av[G][AC];
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    const int g = g0 + k * blockDim.x;
                    if (g < ng) {
                        kk[k] = __ldcs(KG + g);
#pragma unroll
                        for (int a = 0; a < A_CT; ++a) av[k][a] = __ldcs(AG[a] + g);
                    }
                }
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    if (g0 + k * (int)blockDim.x >= ng) break;
#pragma unroll
                    for (int j = 0; j < VN; ++j) {
                        unsigned w;
                        if constexpr (VN == 4) w = (j < 2) ? kk[k].x : kk[k].y;
                        else w = kk[k];
                        const int l = (int)((w >> (16 * (j & 1))) & 0xffffu);
                        m.add_count(l);
#pragma unroll
                        for (int a = 0; a < A_CT; ++a) m.add(a, l, vget<T>(av[k][a], j));
                    }
                }
            }
        } else {
            for (int r0 = it.y + threadIdx.x; r0 < it.z; r0 += U * blockDim.x) {
                int l[U];
                T v[U][AC];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int r = r0 + u * blockDim.x;
                    l[u] = r < it.z ? (int)__ldcs(keys + r) : -1;
                    if (l[u] >= 0)
                        for (int a = 0; a < A; ++a) v[u][a] = __ldcs(attrs + (int64_t)a * S + r);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (l[u] < 0) continue;
                    m.add_count(l[u]);
                    for (int a = 0; a < A; ++a) m.add(a, l[u], v[u][a]);
                }
            }
        }
        __syncthreads();
        const int64_t bin0 = (int64_t)it.x * BK;
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
    if (s) b += (size_t)A * bins * (mode == kSumLimbs ? 12 : wide ? 8 : (mode == kSumF32C ? 8 : 4));
    b = (b + 15) & ~(size_t)15;
    if (lo || hi) b += (size_t)A * bins * 2 * tsz;  // {min key, max key}
    if (mode == kSumLimbs) b = ((b + 15) & ~(size_t)15) + (size_t)(A + 1) * 4;  // exponents, flag
    return b;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool sort_plan(const BinArgs& a, int smem_optin_total, SortDesc* sd) {
    const int smem_optin = smem_optin_total - 1024;  // room for the kernels' static shared memory
    if (a.n > (int64_t)INT_MAX - (1 << 16)) return false;  // 32-bit record slots
    const int64_t B = (int64_t)a.grid.ax[0].res * a.grid.ax[1].res;
    const int mode = smem_sum_mode(a.dtype, a.sum_mode);
    const size_t tsz = a.dtype == BN_F64 ? 8 : 4;
    // largest power-of-two bucket whose shared-memory mesh fits
    int log2bk = 16;
    while (log2bk > 5 && mesh_bytes(a.dtype, mode, 1 << log2bk, a.n_attrs, a.st.do_sum, a.st.do_min,
                                    a.st.do_max) > (size_t)smem_optin)
        --log2bk;
    while (log2bk > 5 && ((int64_t)1 << (log2bk - 1)) >= B) --log2bk;
    if (mesh_bytes(a.dtype, mode, 1 << log2bk, a.n_attrs, a.st.do_sum, a.st.do_min, a.st.do_max) >
        (size_t)smem_optin)
        return false;
    const int64_t nb = (B + (1 << log2bk) - 1) >> log2bk;
    if (nb > 8192) return false;  // u16 bucket index in pass 1; count histogram
    // pass-1 tile: large enough that the run reservations (one global atomic
    // per bucket a tile feeds, at most nb) stay at or below one per four
    // records, then shrunk to what shared memory holds
    auto scatter_bytes = [&](int tp_) {
        return align256((size_t)(nb + 1) * 4) + align256((size_t)nb * 4) + 2 * align256((size_t)tp_ * 2) +
               (size_t)a.n_attrs * tp_ * tsz;
    };
    int tp = 2048;
    while (tp < 16384 && 4 * nb > tp) tp <<= 1;
    while (tp > 2048 && scatter_bytes(tp) > (size_t)smem_optin) tp >>= 1;
    if (scatter_bytes(tp) > (size_t)smem_optin) return false;
    memset(sd, 0, sizeof *sd);
    sd->log2bk = log2bk;
    sd->nb = (int)nb;
    sd->tp = tp;
    sd->per = tp >= 8192 ? 16 : 8;  // 1024, 512, 512, 256 threads
    sd->tiles = (a.n + tp - 1) / tp;
    // record capacity, a multiple of 32 so that every attribute plane starts
    // on a 16-byte boundary (the reduce pass reads records in 16-byte groups)
    sd->slots = ((a.n > 0 ? a.n : 1) + 31) & ~(int64_t)31;
    sd->chunk = kLimbMaxAdds;  // records per work item; also bounds a limb mesh's adds per bin
    sd->off_gpos = (int)align256((size_t)(nb + 1) * 4);
    sd->off_skey = sd->off_gpos + (int)align256((size_t)nb * 4);
    sd->off_sbk = sd->off_skey + (int)align256((size_t)tp * 2);
    sd->off_sattr = sd->off_sbk + (int)align256((size_t)tp * 2);
    sd->smem_scatter = (size_t)sd->off_sattr + (size_t)a.n_attrs * tp * tsz;
    sd->smem_count = (size_t)nb * 4;
    sd->smem_reduce = mesh_bytes(a.dtype, mode, 1 << log2bk, a.n_attrs, a.st.do_sum, a.st.do_min,
                                 a.st.do_max);
    sd->max_items = nb + (a.n + sd->chunk - 1) / sd->chunk + 1;
    return true;
}

size_t sort_scratch_bytes(const SortDesc& sd, const BinArgs& a) {
    const size_t tsz = a.dtype == BN_F64 ? 8 : 4;
    size_t b = 0;
    b += align256((size_t)sd.slots * 2);                                   // keys
    b += align256((size_t)sd.slots * tsz * (a.n_attrs ? a.n_attrs : 1));  // attributes
    b += 2 * align256((size_t)sd.nb * 4);                                  // totals, cursors
    b += align256((size_t)sd.max_items * 16);                              // items
    b += 256;                                                              // counters
    return b;
}

template <typename T, int A_CT, int MODE>
static cudaError_t launch_sort_t(const KernelCtx& kc, const BinArgs& a, const SortDesc& sd,
                                 const BinArgs* dargs) {
    // 16-byte column loads when every column allows them
    bool vec = true;
    for (int k = -2; k < a.n_attrs; ++k) {
        const void* p = k == -2 ? a.x : k == -1 ? a.y : a.a[k];
        vec = vec && ((uintptr_t)p % 16) == 0;
    }
    auto scat = vec ? (sd.per == 16 ? k_sort_scatter<T, A_CT, 16, true> : k_sort_scatter<T, A_CT, 8, true>)
                    : (sd.per == 16 ? k_sort_scatter<T, A_CT, 16, false> : k_sort_scatter<T, A_CT, 8, false>);
    auto red = k_sort_reduce<T, A_CT, MODE>;
    auto cnt = k_sort_count<T>;
    // the opt-in limit covers static plus dynamic shared memory
    cudaError_t e0 = raise_smem_limit(reinterpret_cast<const void*>(scat), kc.smem_optin);
    if (e0 == cudaSuccess) e0 = raise_smem_limit(reinterpret_cast<const void*>(red), kc.smem_optin);
    if (e0 != cudaSuccess) return e0;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cnt, 512, sd.smem_count);
    if (e != cudaSuccess) return e;
    int64_t cgrid = (int64_t)kc.num_sms * (per_sm > 0 ? per_sm : 1);
    const int64_t cwant = (a.n + 512 * 4 - 1) / (512 * 4);
    if (cgrid > cwant) cgrid = cwant;
    if (cgrid < 1) cgrid = 1;
    cnt<<<(unsigned)cgrid, 512, sd.smem_count, kc.stream>>>(a, sd, dargs);
    k_sort_plan<<<1, 1024, 0, kc.stream>>>(sd);
    scat<<<(unsigned)sd.tiles, sd.tp / sd.per, sd.smem_scatter, kc.stream>>>(a, sd, dargs);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, red, 1024, sd.smem_reduce);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)kc.num_sms * per_sm;
    if (grid > sd.max_items) grid = sd.max_items;
    red<<<(unsigned)grid, 1024, sd.smem_reduce, kc.stream>>>(a, sd, dargs);
    kc.count_launch(4);
    return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t dispatch_sort(const KernelCtx& kc, const BinArgs& a, const SortDesc& sd,
                                 const BinArgs* dargs) {
    switch (a.n_attrs) {
        case 0: return launch_sort_t<T, 0, MODE>(kc, a, sd, dargs);
        case 1: return launch_sort_t<T, 1, MODE>(kc, a, sd, dargs);
        case 2: return launch_sort_t<T, 2, MODE>(kc, a, sd, dargs);
        case 3: return launch_sort_t<T, 3, MODE>(kc, a, sd, dargs);
        case 4: return launch_sort_t<T, 4, MODE>(kc, a, sd, dargs);
        default: return launch_sort_t<T, -1, MODE>(kc, a, sd, dargs);
    }
}

cudaError_t launch_bin_sort(const KernelCtx& kc, const BinArgs& a, SortDesc sd, void* scratch,
                            const BinArgs* dargs) {
    const size_t tsz = a.dtype == BN_F64 ? 8 : 4;
    unsigned char* p = static_cast<unsigned char*>(scratch);
    sd.keys = reinterpret_cast<unsigned short*>(p);
    p += align256((size_t)sd.slots * 2);
    sd.attrs = p;
    p += align256((size_t)sd.slots * tsz * (a.n_attrs ? a.n_attrs : 1));
    sd.bucket_total = reinterpret_cast<unsigned*>(p);
    p += align256((size_t)sd.nb * 4);
    sd.cursor = reinterpret_cast<unsigned*>(p);
    p += align256((size_t)sd.nb * 4);
    sd.items = reinterpret_cast<int4*>(p);
    p += align256((size_t)sd.max_items * 16);
    sd.counters = reinterpret_cast<int*>(p);
    cudaError_t e = cudaMemsetAsync(sd.bucket_total, 0, (size_t)sd.nb * 4, kc.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sd.counters, 0, 256, kc.stream);
    if (e != cudaSuccess) return e;
    if (a.dtype == BN_F64) return dispatch_sort<double, kSumF64>(kc, a, sd, dargs);
    if (smem_sum_mode(a.dtype, a.sum_mode) == kSumF32) return dispatch_sort<float, kSumF32>(kc, a, sd, dargs);
    return dispatch_sort<float, kSumLimbs>(kc, a, sd, dargs);
}

}  // namespace bn
