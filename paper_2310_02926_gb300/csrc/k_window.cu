// k_window.cu -- the global-atomic strategy with a privatised window: each
// CTA keeps the count and the sums of a rectangle of the densest bins in
// shared memory, the rest of the mesh takes global atomics as in
// k_global.cu (Sec. 4.2 binning; Sec. 4.4 names the atomic updates as its
// GPU cost, and a centrally concentrated body set piles most particles
// into few bins).
//
// Window sums are the 96-bit fixed-point integers of bn_device.cuh (Fixed,
// add96): exact integer adds in shared memory, no FP64 pipe. Values the
// CTA's scale cannot hold (and NaN, +-inf, subnormals) go to the FP64
// atomic in global memory like every particle outside the window. At the
// end each CTA converts its window sums to FP64 and merges them, with its
// counts, into the global mesh.
//
// Per-bin error of a window sum: at most 2^-45 * sum|a| from the
// conversions, plus one rounding of the converted partial and the FP64
// merge adds: well inside the 1e-12 * sum|a| contract of the FP64 path.
//
// Min and max are not privatised: every particle goes through
// commit_minmax (key records, with the 32-bit filter for f64 data).
#include <cuda_runtime.h>

#include "bn_device.cuh"
#include "bn_internal.cuh"
#include "bn_kernels.h"

namespace bn {

// ---------------------------------------------------------------- window
size_t window_bytes(int cells, int n_attrs, bool do_sum) {
    if (cells <= 0) return 0;
    return (((size_t)cells * 4 + 15) & ~(size_t)15) + (do_sum ? (size_t)n_attrs * cells * 12 : 0);
}

template <typename T> struct WinAxes;
template <> struct WinAxes<float> {
    Axis<float> ax, ay;
    __device__ void init(const GridDesc& g) {
        ax = make_axis<float>(g.ax[0]);
        ay = make_axis<float>(g.ax[1]);
    }
    __device__ __forceinline__ int bx(float x) const { return axis_bin(ax, x); }
    __device__ __forceinline__ int by(float y) const { return axis_bin(ay, y); }
};
template <> struct WinAxes<double> {
    AxisF64 ax, ay;
    __device__ void init(const GridDesc& g) {
        ax = make_axis_f64(g.ax[0], g.edges[0]);
        ay = make_axis_f64(g.ax[1], g.edges[1]);
    }
    __device__ __forceinline__ int bx(double x) const { return axis_bin(ax, x); }
    __device__ __forceinline__ int by(double y) const { return axis_bin(ay, y); }
};

template <typename T, int A_CT, int NT>
__global__ void __launch_bounds__(NT, 1) k_bin_window(BinArgs args, int64_t head, int64_t groups) {
    extern __shared__ __align__(16) unsigned char wsm[];
    __shared__ int s_emax[kMaxAttr];
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::N;
    constexpr int A = A_CT;
    constexpr int AC = A > 0 ? A : 1;
    const GridDesc g = args.dev_grid ? *args.dev_grid : args.grid;
    if (!g.valid) return;
    const StateDesc& st = args.st;
    const bool do_sum = st.do_sum != 0;
    WinAxes<T> axes;
    axes.init(g);
    const int rx = g.ax[0].res;
    const int x0 = args.win_x0, y0 = args.win_y0, nx = args.win_nx, ny = args.win_ny;
    const int W = nx * ny;
    unsigned int* cnt = reinterpret_cast<unsigned int*>(wsm);
    unsigned long long* lo = reinterpret_cast<unsigned long long*>(wsm + (((size_t)W * 4 + 15) & ~(size_t)15));
    int* hi = reinterpret_cast<int*>(lo + (size_t)A * W);

    for (int k = threadIdx.x; k < W; k += NT) cnt[k] = 0u;
    if (do_sum) {
        for (int k = threadIdx.x; k < A * W; k += NT) {
            lo[k] = 0ull;
            hi[k] = 0;
        }
    }
    if (threadIdx.x < kMaxAttr) s_emax[threadIdx.x] = 0;
    __syncthreads();

    const T* __restrict__ X = static_cast<const T*>(args.x);
    const T* __restrict__ Y = static_cast<const T*>(args.y);
    const T* __restrict__ AT[AC];
#pragma unroll
    for (int a = 0; a < AC; ++a) AT[a] = A > 0 ? static_cast<const T*>(args.a[a]) : nullptr;
    const int64_t n = args.n;
    const int64_t nthreads = (int64_t)gridDim.x * NT;
    const int64_t tid = (int64_t)blockIdx.x * NT + threadIdx.x;
    const V* __restrict__ XV = reinterpret_cast<const V*>(X + head);
    const V* __restrict__ YV = reinterpret_cast<const V*>(Y + head);

    // Scale per attribute: the largest finite exponent among this CTA's
    // first values (each thread's first vector group, or first particle).
    int F[AC];
    if (A > 0 && do_sum) {
        int em[AC];
#pragma unroll
        for (int a = 0; a < AC; ++a) em[a] = 0;
        auto see = [&](int a, T v) {
            const int e = Fixed<T>::expo(v);
            if (e < Fixed<T>::kExpMax) em[a] = max(em[a], e);
        };
        if (groups > 0) {
            if (tid < groups)
#pragma unroll
                for (int a = 0; a < AC; ++a) {
                    const V v = __ldg(reinterpret_cast<const V*>(AT[a] + head) + tid);
#pragma unroll
                    for (int j = 0; j < VN; ++j) see(a, vget<T>(v, j));
                }
        } else if (tid < n) {
#pragma unroll
            for (int a = 0; a < AC; ++a) see(a, AT[a][tid * (args.sa[a] > 1 ? args.sa[a] : 1)]);
        }
#pragma unroll
        for (int a = 0; a < AC; ++a) {
            for (int off = 16; off > 0; off >>= 1) em[a] = max(em[a], __shfl_xor_sync(0xffffffffu, em[a], off));
            if ((threadIdx.x & 31) == 0) atomicMax(&s_emax[a], em[a]);
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < AC; ++a) F[a] = Fixed<T>::scale(s_emax[a]);
    } else {
#pragma unroll
        for (int a = 0; a < AC; ++a) F[a] = 0;
    }

    auto one = [&](T x, T y, const T* v) {
        const int ix = axes.bx(x);
        const int iy = axes.by(y);
        if (ix < 0 || iy < 0) return;
        const int64_t b = (int64_t)iy * rx + ix;
        const unsigned wx = (unsigned)(ix - x0), wy = (unsigned)(iy - y0);
        if (wx < (unsigned)nx && wy < (unsigned)ny) {
            const int k = (int)wy * nx + (int)wx;
            atomicAdd(&cnt[k], 1u);
            if (do_sum) {
#pragma unroll
                for (int a = 0; a < A; ++a) {
                    long long q;
                    if (Fixed<T>::to_fixed(v[a], F[a], &q)) {
                        if (q != 0) add96(&lo[a * W + k], &hi[a * W + k], q);
                    } else {
                        atomicAdd(&st.sum[a][b], (double)v[a]);
                    }
                }
            }
        } else {
            atomicAdd(&st.count[b], 1ull);
            if (do_sum)
#pragma unroll
                for (int a = 0; a < A; ++a) atomicAdd(&st.sum[a][b], (double)v[a]);
        }
        if (A > 0) commit_minmax<T, A>(st, A, b, v, v);
    };

    // scalar head and tail; strided columns are read in place here
    const int64_t sx = args.sx > 1 ? args.sx : 1, sy = args.sy > 1 ? args.sy : 1;
    int64_t sa[AC];
#pragma unroll
    for (int a = 0; a < AC; ++a) sa[a] = args.sa[a] > 1 ? args.sa[a] : 1;
    auto scalar = [&](int64_t i) {
        T v[AC];
#pragma unroll
        for (int a = 0; a < A; ++a) v[a] = AT[a][i * sa[a]];
        one(X[i * sx], Y[i * sy], v);
    };
    for (int64_t i = tid; i < head; i += nthreads) scalar(i);
    for (int64_t i = head + groups * VN + tid; i < n; i += nthreads) scalar(i);
    // vector groups, two per thread and iteration so that more loads are in
    // flight while the atomics of the previous ones drain
    for (int64_t gi = tid; gi < groups; gi += 2 * nthreads) {
        const int64_t g2 = gi + nthreads;
        const bool live2 = g2 < groups;
        V xv[2], yv[2], av[2][AC];
        xv[0] = ld_stream(XV + gi);
        yv[0] = ld_stream(YV + gi);
#pragma unroll
        for (int a = 0; a < A; ++a) av[0][a] = ld_stream(reinterpret_cast<const V*>(AT[a] + head) + gi);
        if (live2) {
            xv[1] = ld_stream(XV + g2);
            yv[1] = ld_stream(YV + g2);
#pragma unroll
            for (int a = 0; a < A; ++a) av[1][a] = ld_stream(reinterpret_cast<const V*>(AT[a] + head) + g2);
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (r == 1 && !live2) break;
#pragma unroll
            for (int j = 0; j < VN; ++j) {
                T v[AC];
#pragma unroll
                for (int a = 0; a < A; ++a) v[a] = vget<T>(av[r][a], j);
                one(vget<T>(xv[r], j), vget<T>(yv[r], j), v);
            }
        }
    }

    // this CTA's window into the global mesh
    __syncthreads();
    for (int k = threadIdx.x; k < W; k += NT) {
        const unsigned int c = cnt[k];
        if (!c) continue;
        const int wy = k / nx, wx = k - wy * nx;
        const int64_t b = (int64_t)(y0 + wy) * rx + (x0 + wx);
        atomicAdd(&st.count[b], (unsigned long long)c);
        if (do_sum)
#pragma unroll
            for (int a = 0; a < A; ++a) {
                const unsigned long long l = lo[a * W + k];
                const int h = hi[a * W + k];
                if (l != 0ull || h != 0) atomicAdd(&st.sum[a][b], fixed_value(l, h, F[a]));
            }
    }
}

template <typename T>
static void window_split(const BinArgs& a, int64_t* head, int64_t* groups) {
    constexpr int VN = VecOf<T>::N;
    auto phase = [](const void* p) { return (int)(((uintptr_t)p / sizeof(T)) % VN); };
    const int ph = phase(a.x);
    bool same = phase(a.y) == ph;
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
static cudaError_t launch_window_t(const KernelCtx& kc, const BinArgs& a) {
    constexpr int NT = 512;
    auto kern = k_bin_window<T, A_CT, NT>;
    const size_t smem = window_bytes(a.win_nx * a.win_ny, a.n_attrs, a.st.do_sum != 0);
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(kern), kc.smem_optin);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t head, groups;
    window_split<T>(a, &head, &groups);
    const int64_t work = groups > 0 ? groups : a.n;
    int64_t grid = (work + NT - 1) / NT;
    const int64_t cap = (int64_t)kc.num_sms * per_sm;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    kern<<<(int)grid, NT, smem, kc.stream>>>(a, head, groups);
    kc.count_launch();
    return cudaGetLastError();
}

template <typename T>
static cudaError_t dispatch_window(const KernelCtx& kc, const BinArgs& a) {
    switch (a.n_attrs) {
        case 0: return launch_window_t<T, 0>(kc, a);
        case 1: return launch_window_t<T, 1>(kc, a);
        case 2: return launch_window_t<T, 2>(kc, a);
        case 3: return launch_window_t<T, 3>(kc, a);
        case 4: return launch_window_t<T, 4>(kc, a);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_bin_window(const KernelCtx& kc, const BinArgs& a) {
    if (a.n_attrs > kWindowMaxAttr || a.win_nx <= 0 || a.win_ny <= 0) return cudaErrorInvalidValue;
    const size_t smem = window_bytes(a.win_nx * a.win_ny, a.n_attrs, a.st.do_sum != 0);
    if (smem > (size_t)kc.smem_optin - 1024) return cudaErrorInvalidValue;
    return a.dtype == BN_F64 ? dispatch_window<double>(kc, a) : dispatch_window<float>(kc, a);
}

}  // namespace bn
