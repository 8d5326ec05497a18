// k_global.cu -- particles straight into the global mesh with L2 atomics,
// for meshes too large to privatise in shared memory (Sec. 4.2 binning; the
// atomic updates whose races Sec. 4.4 names as binning's GPU cost).
//
// Per in-bounds particle: one u64 count add and one FP64 add per attribute
// (executed in L2, not on the SM's FP64 pipe), and min/max atomics only
// when a plain read of the current value shows the particle would change
// it (min only falls and max only rises, so a stale read is safe: it can
// only let through an atomic that turns out to be unnecessary). With
// count-and-sums records (StateDesc::rec) the count and the sums of a
// particle go to L2 as one bulk reduction of the bin's record (measured on
// GB300: 78 G particles/s against 36 G/s for four separate reductions per
// particle into the same 1M bins of a centrally concentrated set). Lanes of a
// warp that hit the same bin are combined first (__match_any_sync) so a
// cluster of particles costs one set of atomics per warp, not per lane.
// With a window (BinArgs::win_*), k_window.cu's kernel runs instead.
#include <cuda_runtime.h>

#include "bn_device.cuh"
#include "bn_internal.cuh"
#include "bn_kernels.h"

namespace bn {

template <typename T> struct GVec;
template <> struct GVec<float> { using type = float4; static constexpr int N = 4; };
template <> struct GVec<double> { using type = double2; static constexpr int N = 2; };

template <typename T>
__device__ __forceinline__ T gget(const typename GVec<T>::type& v, int j);
template <> __device__ __forceinline__ float gget<float>(const float4& v, int j) {
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}
template <> __device__ __forceinline__ double gget<double>(const double2& v, int j) {
    return j == 0 ? v.x : v.y;
}

template <typename T> struct GBinner;
template <> struct GBinner<float> {
    Axis<float> ax, ay;
    int rx;
    __device__ void init(const GridDesc& g) {
        ax = make_axis<float>(g.ax[0]);
        ay = make_axis<float>(g.ax[1]);
        rx = g.ax[0].res;
    }
    __device__ __forceinline__ int bin(float x, float y) const {
        int ix = axis_bin(ax, x);
        int iy = axis_bin(ay, y);
        return (ix < 0 || iy < 0) ? -1 : iy * rx + ix;
    }
};
template <> struct GBinner<double> {
    AxisF64 ax, ay;
    int rx;
    __device__ void init(const GridDesc& g) {
        ax = make_axis_f64(g.ax[0], g.edges[0]);
        ay = make_axis_f64(g.ax[1], g.edges[1]);
        rx = g.ax[0].res;
    }
    __device__ __forceinline__ int bin(double x, double y) const {
        int ix = axis_bin(ax, x);
        int iy = axis_bin(ay, y);
        return (ix < 0 || iy < 0) ? -1 : iy * rx + ix;
    }
};

// 256 threads per CTA. Up to four attributes: at most 64 registers, four
// CTAs per SM (at 5e7 Plummer particles, f64, three attributes: 1.157 ms
// against 1.249 ms for three CTAs per SM at 80 registers; the kernel waits
// on latency, and more warps hide it). The generic kernel (any attribute
// count, values through local memory): three CTAs per SM.
template <int A_CT>
constexpr int global_min_ctas() { return (A_CT >= 0 && A_CT <= 4) ? 4 : 3; }

template <typename T, int A_CT, int NT>
__global__ void __launch_bounds__(NT, global_min_ctas<A_CT>()) k_bin_global(BinArgs args, int64_t head, int64_t groups) {
    using V = typename GVec<T>::type;
    constexpr int VN = GVec<T>::N;
    constexpr int AC = A_CT > 0 ? A_CT : kMaxAttr;
    const GridDesc g = args.dev_grid ? *args.dev_grid : args.grid;
    if (!g.valid) return;
    const int A = A_CT >= 0 ? A_CT : args.n_attrs;
    const StateDesc& st = args.st;
    GBinner<T> binner;
    binner.init(g);
    // count-and-sums records: each thread stages its record in its own slot
    constexpr int RDS = (A_CT >= 1 && A_CT <= kRecMaxAttr) ? ((A_CT + 2) & ~1) : 2;
    __shared__ __align__(16) double rec_slots[NT * RDS];
    double* const slot = (A_CT >= 1 && A_CT <= kRecMaxAttr && st.rec) ? rec_slots + threadIdx.x * RDS : nullptr;

    const T* __restrict__ X = static_cast<const T*>(args.x);
    const T* __restrict__ Y = static_cast<const T*>(args.y);
    const int64_t n = args.n;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;

    // scalar head and tail: whole warps iterate together (warp_commit needs
    // every lane), lanes past the end pass b = -1
    const int64_t tail0 = head + groups * VN;
    const int64_t warp_base = tid - (threadIdx.x & 31);
    // scalar path: strided columns are read in place
    const int64_t sx = args.sx > 1 ? args.sx : 1, sy = args.sy > 1 ? args.sy : 1;
    auto scalar_range = [&](int64_t r0, int64_t r1) {
        for (int64_t base = r0 + warp_base; base < r1; base += nthreads) {
            const int64_t i = base + (threadIdx.x & 31);
            T v[AC];
            int b = -1;
            if (i < r1) {
                b = binner.bin(X[i * sx], Y[i * sy]);
                for (int a = 0; a < A; ++a)
                    v[a] = static_cast<const T*>(args.a[a])[i * (args.sa[a] > 1 ? args.sa[a] : 1)];
            }
            warp_commit<T, A_CT>(st, A, b, v, args.aggregate != 0, slot);
        }
    };
    scalar_range(0, head);
    scalar_range(tail0, n);

    const V* __restrict__ XV = reinterpret_cast<const V*>(X + head);
    const V* __restrict__ YV = reinterpret_cast<const V*>(Y + head);
    // Vector part. Fixed attribute counts: each CTA (one wave of resident
    // CTAs) streams one contiguous range of groups, NT per step. The generic
    // kernel: a grid-stride loop over warps (measured faster for it).
    constexpr bool kContig = A_CT >= 0;
    const int64_t per_cta = ((groups + gridDim.x - 1) / gridDim.x + NT - 1) / NT * NT;
    const int64_t g_begin = kContig ? min(groups, (int64_t)blockIdx.x * per_cta) : warp_base;
    const int64_t g_end = kContig ? min(groups, g_begin + per_cta) : groups;
    const int64_t g_step = kContig ? (int64_t)NT : nthreads;
    for (int64_t gb = g_begin; gb < g_end; gb += g_step) {
        const int64_t gi = gb + (kContig ? (int64_t)threadIdx.x : (int64_t)(threadIdx.x & 31));
        const bool live = gi < g_end;
        V x0, y0;
        V av[A_CT > 0 ? A_CT : 1];
        if (live) {
            x0 = ld_stream(XV + gi);
            y0 = ld_stream(YV + gi);
            if (A_CT > 0) {
#pragma unroll
                for (int a = 0; a < A_CT; ++a)
                    av[a] = ld_stream(reinterpret_cast<const V*>(static_cast<const T*>(args.a[a]) + head) + gi);
            }
        }
#pragma unroll
        for (int j = 0; j < VN; ++j) {
            int b = -1;
            T v[AC];
            if (live) {
                b = binner.bin(gget<T>(x0, j), gget<T>(y0, j));
                if (A_CT > 0) {
#pragma unroll
                    for (int a = 0; a < (A_CT > 0 ? A_CT : 1); ++a) v[a] = gget<T>(av[a], j);
                } else {
                    const int64_t i = head + gi * VN + j;
                    for (int a = 0; a < A; ++a) v[a] = static_cast<const T*>(args.a[a])[i];
                }
            }
            warp_commit<T, A_CT>(st, A, b, v, args.aggregate != 0, slot);
        }
    }
    if (slot) record_drain();
}

template <typename T>
static void gvector_split(const BinArgs& a, int64_t* head, int64_t* groups) {
    constexpr int VN = GVec<T>::N;
    auto phase = [](const void* p) { return (int)(((uintptr_t)p / sizeof(T)) % VN); };
    const bool aligned = ((uintptr_t)a.x % sizeof(T)) == 0;
    int ph = phase(a.x);
    bool same = aligned && phase(a.y) == ph;
    for (int k = 0; k < a.n_attrs; ++k) same = same && phase(a.a[k]) == ph;
    bool strided = a.sx > 1 || a.sy > 1;
    for (int k = 0; k < a.n_attrs; ++k) strided = strided || a.sa[k] > 1;
    if (!same || strided) {
        *head = a.n;
        *groups = 0;
        return;
    }
    int64_t h = (VN - ph) % VN;
    if (h > a.n) h = a.n;
    *head = h;
    *groups = (a.n - h) / VN;
}

template <typename T, int A_CT>
static cudaError_t launch_global_t(const KernelCtx& kc, const BinArgs& a) {
    int64_t head, groups;
    gvector_split<T>(a, &head, &groups);
    const int64_t work = groups > 0 ? groups : a.n;
    const int block = 256;
    auto kern = k_bin_global<T, A_CT, 256>;
    // one wave of resident CTAs, each with a contiguous share of the groups
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0);
    if (e != cudaSuccess) return e;
    int64_t grid = (work + block - 1) / block;
    const int64_t cap = (int64_t)kc.num_sms * (A_CT >= 0 ? (per_sm > 0 ? per_sm : 1) : 8);
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    kern<<<(int)grid, block, 0, kc.stream>>>(a, head, groups);
    kc.count_launch();
    return cudaGetLastError();
}

template <typename T>
static cudaError_t dispatch_global(const KernelCtx& kc, const BinArgs& a) {
    switch (a.n_attrs) {
        case 0: return launch_global_t<T, 0>(kc, a);
        case 1: return launch_global_t<T, 1>(kc, a);
        case 2: return launch_global_t<T, 2>(kc, a);
        case 3: return launch_global_t<T, 3>(kc, a);
        case 4: return launch_global_t<T, 4>(kc, a);
        default: return launch_global_t<T, -1>(kc, a);
    }
}

cudaError_t launch_bin_global(const KernelCtx& kc, const BinArgs& a) {
    if (a.win_nx > 0 && a.win_ny > 0) return launch_bin_window(kc, a);
    return a.dtype == BN_F64 ? dispatch_global<double>(kc, a) : dispatch_global<float>(kc, a);
}

}  // namespace bn
