// k_private.cu -- K1: per-CTA shared-memory copy of the whole mesh.
//
// Sec. 4.2 bins each particle into one mesh cell and reduces count, sum,
// min and max per cell; the paper's CUDA version resolves races between
// threads with atomic updates of one global mesh and calls that the reason
// binning suits GPUs poorly (Sec. 4.4). Here each CTA owns a private copy
// of the mesh in shared memory, so the per-particle atomics are shared-
// memory atomics (integer count, FP add, integer min/max on IEEE bits) and
// global atomics happen once per non-empty bin per CTA, in the merge.
//
// Columns are streamed with 16-byte vector loads (two groups per thread
// per iteration, so several loads are in flight); the bin index follows
// the reference rounding sequence exactly (f32: directly; f64: via the
// exact edge keys, no FP64 arithmetic).
#include <cuda_runtime.h>

#include "bn_device.cuh"
#include "bn_internal.cuh"
#include "bn_kernels.h"

namespace bn {

// NT threads per CTA: 512 when two or more CTAs fit on an SM; 1024 (at most
// 64 registers, one vector group per pipeline stage) when the mesh leaves
// room for one CTA only, so that an SM still has 32 warps to hide the
// shared-memory atomic latency with.
template <typename T, int A_CT, int MODE, int NT>
__global__ void __launch_bounds__(NT, 1) k_bin_private(const __grid_constant__ BinArgs args, int64_t head,
                                                       int64_t groups) {
    extern __shared__ __align__(16) unsigned char smem[];
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::N;
    const GridDesc g = args.dev_grid ? *args.dev_grid : args.grid;
    if (!g.valid) return;
    const int A = A_CT >= 0 ? A_CT : args.n_attrs;
    const int B = g.ax[0].res * g.ax[1].res;
    const StateDesc& st = args.st;

    SmemMesh<T, MODE> m;
    m.carve(smem, B, A, st.do_sum != 0, st.do_min != 0, st.do_max != 0);
    if constexpr (MODE == kSumF64Keys) m.bind_keys(st);
    m.clear(A);
    Binner<T> binner;
    binner.init(g);
    __syncthreads();
    if (MODE == kSumLimbs && st.do_sum) {
        // the window of the limb sums: one value per thread and attribute
        const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (i < args.n)
            for (int a = 0; a < A; ++a) {
                const int64_t sa = args.sa[a] > 1 ? args.sa[a] : 1;
                m.sample(a, static_cast<const T*>(args.a[a])[i * sa]);
            }
        m.bind_fallback(st.sum, 0);
        __syncthreads();
    }

    const T* __restrict__ X = static_cast<const T*>(args.x);
    const T* __restrict__ Y = static_cast<const T*>(args.y);
    const int64_t n = args.n;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;

    // scalar path: strided columns are read in place
    const int64_t sx = args.sx > 1 ? args.sx : 1, sy = args.sy > 1 ? args.sy : 1;
    auto one = [&](int64_t i) {
        int b = binner.bin(X[i * sx], Y[i * sy]);
        if (b < 0) return;
        m.add_count(b);
        for (int a = 0; a < A; ++a) {
            const int64_t sa = args.sa[a] > 1 ? args.sa[a] : 1;
            m.add(a, b, static_cast<const T*>(args.a[a])[i * sa]);
        }
    };

    // scalar head (until every column is 16-byte aligned) and tail
    const int64_t tail0 = head + groups * VN;
    for (int64_t i = tid; i < head; i += nthreads) one(i);
    for (int64_t i = tail0 + tid; i < n; i += nthreads) one(i);

    // vector body: groups of VN particles, U groups per thread per step
    constexpr int U = NT >= 1024 ? 1 : 2;
    const V* __restrict__ XV = reinterpret_cast<const V*>(X + head);
    const V* __restrict__ YV = reinterpret_cast<const V*>(Y + head);
    if (A_CT >= 0) {
        constexpr int AC = A_CT > 0 ? A_CT : 1;
        const V* AV[AC];
#pragma unroll
        for (int a = 0; a < AC; ++a)
            AV[a] = reinterpret_cast<const V*>(static_cast<const T*>(args.a[a < A ? a : 0]) + head);
        // software pipeline: the loads of the next U groups are in flight
        // while the current U are binned
        struct Stage {
            V x[U], y[U], a[U][AC];
        };
        auto load = [&](Stage& st, int64_t g) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t gg = g + u * nthreads;
                if (gg < groups) {
                    st.x[u] = ld_stream(XV + gg);
                    st.y[u] = ld_stream(YV + gg);
#pragma unroll
                    for (int a = 0; a < A_CT; ++a) st.a[u][a] = ld_stream(AV[a] + gg);
                }
            }
        };
        auto consume = [&](const Stage& st, int64_t g) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (g + u * nthreads >= groups) break;
#pragma unroll
                for (int j = 0; j < VN; ++j) {
                    const int b = binner.bin(vget<T>(st.x[u], j), vget<T>(st.y[u], j));
                    if (b >= 0) {
                        T v[AC];
#pragma unroll
                        for (int a = 0; a < A_CT; ++a) v[a] = vget<T>(st.a[u][a], j);
                        m.template add_particle<A_CT>(b, v);
                    }
                }
            }
        };
        Stage cur, nxt;
        int64_t gi = tid;
        if (gi < groups) load(cur, gi);
        for (; gi < groups; gi += U * nthreads) {
            const int64_t gn = gi + U * nthreads;
            if (gn < groups) load(nxt, gn);
            consume(cur, gi);
            cur = nxt;
        }
    } else {
        for (int64_t gi = tid; gi < groups; gi += nthreads) {
            V x0 = ld_stream(XV + gi), y0 = ld_stream(YV + gi);
#pragma unroll
            for (int j = 0; j < VN; ++j) {
                int b = binner.bin(vget<T>(x0, j), vget<T>(y0, j));
                if (b < 0) continue;
                m.add_count(b);
                const int64_t i = head + gi * VN + j;
                for (int a = 0; a < A; ++a) m.add(a, b, static_cast<const T*>(args.a[a])[i]);
            }
        }
    }
    __syncthreads();
    m.merge(st, A);
}

// ------------------------------------------------------------------ host side
template <typename T>
static void vector_split(const BinArgs& a, int64_t* head, int64_t* groups) {
    constexpr int VN = VecOf<T>::N;
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

static size_t private_bytes_for(int dtype, int mode, int B, int A, bool s, bool lo, bool hi) {
    const bool wide = dtype == BN_F64 || mode == kSumF64 || mode == kSumF64Keys;
    const size_t tsz = dtype == BN_F64 ? 8 : 4;
    size_t b = ((size_t)B * 4 + 15) & ~(size_t)15;
    if (s) b += (size_t)A * B * (mode == kSumLimbs ? 12 : wide ? 8 : (mode == kSumF32C ? 8 : 4));
    b = (b + 15) & ~(size_t)15;
    // {min key, max key}, or their top 32 bits as a filter (kSumF64Keys)
    if (lo || hi) b += (size_t)A * B * (mode == kSumF64Keys ? 8 : 2 * tsz);
    if (mode == kSumLimbs) b = ((b + 15) & ~(size_t)15) + (size_t)(A + 1) * 4;  // exponents, flag
    return b;
}

// The mesh mode a particle pass uses: f64 min/max go through the global key
// records when the runtime provides them.
static int private_mode(const BinArgs& a) {
    if (a.dtype != BN_F64) return smem_sum_mode(a.dtype, a.sum_mode);
    return (a.st.mmk && (a.st.do_min || a.st.do_max)) ? kSumF64Keys : kSumF64;
}

size_t private_mesh_bytes(int dtype, int sum_mode, int64_t bins, int n_attrs, bool s, bool lo, bool hi) {
    return private_bytes_for(dtype, smem_sum_mode(dtype, sum_mode), (int)bins, n_attrs, s, lo, hi);
}

size_t private_smem_bytes(const BinArgs& a, int smem_optin, int keys) {
    const int64_t B = (int64_t)a.grid.ax[0].res * a.grid.ax[1].res;
    if (B > (1 << 20)) return 0;
    int mode = private_mode(a);
    if (keys >= 0 && a.dtype == BN_F64)
        mode = (keys && (a.st.do_min || a.st.do_max)) ? kSumF64Keys : kSumF64;
    size_t b = private_bytes_for(a.dtype, mode, (int)B, a.n_attrs, a.st.do_sum != 0, a.st.do_min != 0,
                                 a.st.do_max != 0);
    return b <= (size_t)smem_optin ? b : 0;
}

template <typename T, int A_CT, int MODE, int NT>
static cudaError_t configure_private(const KernelCtx& kc, size_t smem, int* per_sm) {
    auto kern = k_bin_private<T, A_CT, MODE, NT>;
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(kern), kc.smem_optin);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, NT, smem);
}

template <typename T, int A_CT, int MODE>
static cudaError_t launch_private_t(const KernelCtx& kc, const BinArgs& a, size_t smem) {
    int per_sm = 0;
    cudaError_t e = configure_private<T, A_CT, MODE, 512>(kc, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // one 512-thread CTA per SM leaves it at 16 warps: use 1024 threads
    // (the generic any-attribute instance keeps 512)
    bool wide = false;
    if constexpr (A_CT >= 0) {
        if (per_sm == 1) {
            int per_sm_w = 0;
            e = configure_private<T, A_CT, MODE, 1024>(kc, smem, &per_sm_w);
            if (e != cudaSuccess) return e;
            wide = per_sm_w >= 1;
        }
    }
    const int block = wide ? 1024 : 512;
    int64_t head, groups;
    vector_split<T>(a, &head, &groups);
    // enough particles per CTA to amortise clearing and merging its mesh
    const int64_t B = (int64_t)a.grid.ax[0].res * a.grid.ax[1].res;
    int64_t want = a.n / (4 * B > 16 * block ? 4 * B : 16 * block);
    if (want < 1) want = 1;
    int64_t grid = (int64_t)kc.num_sms * per_sm;
    if (grid > want) grid = want;
    if (MODE == kSumLimbs) {
        // a limb mesh takes at most kLimbMaxAdds values per bin: enough CTAs
        // that none sees more particles (each thread: at most `per` of the
        // body, one of the head and one of the tail)
        constexpr int VN = VecOf<T>::N;
        const int64_t per = kLimbMaxAdds / block - 2 * VN;
        const int64_t need = (a.n + per * block - 1) / (per * block);
        if (grid < need) grid = need;
    }
    if constexpr (A_CT >= 0) {
        if (wide)
            k_bin_private<T, A_CT, MODE, 1024><<<(int)grid, block, smem, kc.stream>>>(a, head, groups);
    }
    if (!wide) k_bin_private<T, A_CT, MODE, 512><<<(int)grid, block, smem, kc.stream>>>(a, head, groups);
    kc.count_launch();
    return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t dispatch_a(const KernelCtx& kc, const BinArgs& a, size_t smem) {
    switch (a.n_attrs) {
        case 0: return launch_private_t<T, 0, MODE>(kc, a, smem);
        case 1: return launch_private_t<T, 1, MODE>(kc, a, smem);
        case 2: return launch_private_t<T, 2, MODE>(kc, a, smem);
        case 3: return launch_private_t<T, 3, MODE>(kc, a, smem);
        case 4: return launch_private_t<T, 4, MODE>(kc, a, smem);
        default: return launch_private_t<T, -1, MODE>(kc, a, smem);
    }
}

cudaError_t launch_bin_private(const KernelCtx& kc, const BinArgs& a) {
    size_t smem = private_smem_bytes(a, kc.smem_optin);
    if (smem == 0) return cudaErrorInvalidValue;
    if (a.dtype == BN_F64)
        return private_mode(a) == kSumF64Keys ? dispatch_a<double, kSumF64Keys>(kc, a, smem)
                                              : dispatch_a<double, kSumF64>(kc, a, smem);
    if (private_mode(a) == kSumF32) return dispatch_a<float, kSumF32>(kc, a, smem);
    return dispatch_a<float, kSumLimbs>(kc, a, smem);
}

}  // namespace bn
