// k_common.cu -- the small kernels around the binning hot loop:
//   init of the per-bin state, automatic bounds (Sec. 4.2: mesh bounds
//   "obtained on the fly" as the min/max of the coordinates), mesh set-up
//   with exact f64 bin-edge keys, finalisation (avg = sum / count), the
//   merge of partial results of one mesh, and a strided-column gather.
#include <cuda_runtime.h>

#include <climits>
#include <mutex>
#include <set>
#include <type_traits>
#include <utility>

#include "bn_device.cuh"
#include "bn_internal.cuh"
#include "bn_kernels.h"

namespace bn {

// ------------------------------------------------------------------ launch set-up
// cudaFuncSetAttribute acts on the current device's context, so the limit is
// raised once per (kernel, device); the server's worker thread and caller
// threads launch concurrently, hence the lock.
cudaError_t raise_smem_limit(const void* kernel, int smem_optin) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({kernel, dev})) return cudaSuccess;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done.insert({kernel, dev});
    return e;
}

// ------------------------------------------------------------------ init
// Empty-bin state: count 0, sum +0.0, min +inf, max -inf.
template <typename T>
__global__ void k_init_state(StateDesc st, T* bounds_acc) {
    const int64_t B = st.bins;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (bounds_acc && t0 == 0) {
        bounds_acc[0] = pos_inf<T>();
        bounds_acc[1] = neg_inf<T>();
        bounds_acc[2] = pos_inf<T>();
        bounds_acc[3] = neg_inf<T>();
    }
    if (st.rec) {  // count and sums live in the records until k_finalize
        const int64_t nd = B * record_doubles(st.n_attrs);
        for (int64_t q = t0; q < nd; q += stride) st.rec[q] = 0.0;
    } else {
        for (int64_t b = t0; b < B; b += stride) st.count[b] = 0ull;
    }
    if (st.mmk) {
        using KO = KeyOf<T>;
        typename KO::K2 init;
        init.x = KO::kPosInf;
        init.y = KO::kNegInf;
        const int64_t pairs = B * key_record_pairs(st.n_attrs, (int)sizeof(typename KO::K));
        auto* kp = static_cast<typename KO::K2*>(st.mmk);
        for (int64_t q = t0; q < pairs; q += stride) kp[q] = init;
    }
    if (st.mmf) {
        const int64_t pairs = B * filter_record_pairs(st.n_attrs);
        int2* fp = static_cast<int2*>(st.mmf);
        for (int64_t q = t0; q < pairs; q += stride) fp[q] = make_int2(INT_MAX, INT_MIN);
    }
    for (int a = 0; a < st.n_attrs; ++a) {
        if (st.do_sum && !st.rec)
            for (int64_t b = t0; b < B; b += stride) st.sum[a][b] = 0.0;
        if (st.mmk) continue;
        if (st.do_min) {
            T* p = static_cast<T*>(st.mn[a]);
            for (int64_t b = t0; b < B; b += stride) p[b] = pos_inf<T>();
        }
        if (st.do_max) {
            T* p = static_cast<T*>(st.mx[a]);
            for (int64_t b = t0; b < B; b += stride) p[b] = neg_inf<T>();
        }
    }
}

// ------------------------------------------------------------------ bounds
template <typename T> struct KeyT;
template <> struct KeyT<float> { using type = int; };
template <> struct KeyT<double> { using type = long long; };

template <typename T>
__device__ __forceinline__ bool finite_bits(T v);
template <> __device__ __forceinline__ bool finite_bits<float>(float v) {
    return (__float_as_uint(v) & 0x7f800000u) != 0x7f800000u;
}
template <> __device__ __forceinline__ bool finite_bits<double>(double v) {
    return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ull) !=
           0x7ff0000000000000ull;
}

// min/max over the finite values of x and y, reduced with ordered integer
// keys (no FP compares), one atomic per warp into bounds_acc[4] =
// {min x, max x, min y, max y}.
template <typename T>
__global__ void k_bounds_reduce(const T* __restrict__ x, const T* __restrict__ y, int64_t n,
                                T* bounds_acc, int64_t sx, int64_t sy) {
    using K = typename KeyT<T>::type;
    const K kmax = (K)(~(typename std::make_unsigned<K>::type)0 >> 1);
    const K kmin = -kmax - 1;
    K mnx = kmax, mxx = kmin, mny = kmax, mxy = kmin;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        T vx = x[i * sx], vy = y[i * sy];
        if (finite_bits(vx)) {
            K k = ordered_key(vx);
            mnx = min(mnx, k);
            mxx = max(mxx, k);
        }
        if (finite_bits(vy)) {
            K k = ordered_key(vy);
            mny = min(mny, k);
            mxy = max(mxy, k);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        mnx = min(mnx, __shfl_xor_sync(0xffffffffu, mnx, off));
        mxx = max(mxx, __shfl_xor_sync(0xffffffffu, mxx, off));
        mny = min(mny, __shfl_xor_sync(0xffffffffu, mny, off));
        mxy = max(mxy, __shfl_xor_sync(0xffffffffu, mxy, off));
    }
    if ((threadIdx.x & 31) == 0) {
        // keys back to values; a key of kmax/kmin means "no finite value seen"
        auto val = [](K k) -> T {
            if (sizeof(T) == 8) return (T)key_to_double((long long)k);
            int b = (int)k >= 0 ? (int)k : ((int)k ^ 0x7fffffff);
            return (T)__int_as_float(b);
        };
        if (mnx != kmax) atomic_min_total(&bounds_acc[0], val(mnx));
        if (mxx != kmin) atomic_max_total(&bounds_acc[1], val(mxx));
        if (mny != kmax) atomic_min_total(&bounds_acc[2], val(mny));
        if (mxy != kmin) atomic_max_total(&bounds_acc[3], val(mxy));
    }
}

// ------------------------------------------------------------------ set-up
template <typename T>
__device__ bool make_axis_from_bounds(T lo, T hi, int res, AxisDesc* d) {
    // Sec. 4.2 automatic bounds: [min, max] of the finite coordinates, closed.
    if (!finite_bits(lo) || !finite_bits(hi)) return false;
    T width;
    T s;
    if (sizeof(T) == 8) {
        width = (T)__dsub_rn((double)hi, (double)lo);
        s = (T)__ddiv_rn((double)res, (double)width);
    } else {
        width = (T)__fsub_rn((float)hi, (float)lo);
        s = (T)__fdiv_rn((float)res, (float)width);
    }
    if (!(width > (T)0) || !finite_bits(width) || !(s > (T)0) || !finite_bits(s)) return false;
    d->lo = (double)lo;
    d->hi = (double)hi;
    d->s = (double)s;
    d->res = res;
    d->closed = 1;
    return true;
}

// Bound on |t_f - t| in bins for the FP32 estimate of an f64 axis: x and lo
// are truncated to 20 mantissa bits (each off by at most 2^-20 of its
// magnitude m, times s), and the FP32 subtraction, the rounding of s to FP32
// and the FP32 multiplication each add at most 2^-24 * res; the reference t
// itself is within a few 2^-53 * res of the real value. The bound below
// doubles each term. Returns the bound, or a negative value when the
// estimate is not usable (bound >= 1/4, or values outside FP32 range).
__device__ __host__ inline double fast_delta(double lo, double hi, double s, int res) {
    double m = fabs(lo) > fabs(hi) ? fabs(lo) : fabs(hi);
    double err = 2.0 * m * s * (1.0 / 524288.0) + (double)res * (1.0 / 2097152.0);
    return (err < 0.25 && m < 1e37 && s < 1e37) ? err : -1.0;
}

// One block computes the mesh (automatic bounds: from bounds_acc; explicit:
// from the host's descriptor); every block then fills a slice of the f64
// edge tables. Block 0 publishes the descriptor, the bounds actually used
// and, if the automatic bounds collapsed, BN_ERR_DEGENERATE in *status.
template <typename T>
__global__ void k_grid_setup(GridDesc host_desc, const T* bounds_acc, GridDesc* dev_desc,
                             long long* edges0, long long* edges1, double* bounds_out,
                             int* status) {
    __shared__ GridDesc g;
    if (threadIdx.x == 0) {
        g = host_desc;
        if (bounds_acc) {
            bool ok = make_axis_from_bounds<T>(bounds_acc[0], bounds_acc[1], host_desc.ax[0].res,
                                               &g.ax[0]) &&
                      make_axis_from_bounds<T>(bounds_acc[2], bounds_acc[3], host_desc.ax[1].res,
                                               &g.ax[1]);
            g.valid = ok ? 1 : 0;
        }
        for (int a = 0; a < 2; ++a) {
            const double dl = (sizeof(T) == 8 && g.valid)
                                  ? fast_delta(g.ax[a].lo, g.ax[a].hi, g.ax[a].s, g.ax[a].res)
                                  : -1.0;
            g.ax[a].fast = dl >= 0.0 ? 1 : 0;
            // round the margin up so the float comparison stays conservative
            g.ax[a].delta = dl >= 0.0 ? __double2float_ru(dl) : 0.0f;
        }
        g.edges[0] = (sizeof(T) == 8) ? edges0 : nullptr;
        g.edges[1] = (sizeof(T) == 8) ? edges1 : nullptr;
        if (blockIdx.x == 0) {
            *dev_desc = g;
            if (!g.valid && status) *status = BN_ERR_DEGENERATE;
            if (bounds_out && g.valid) {
                bounds_out[0] = g.ax[0].lo;
                bounds_out[1] = g.ax[0].hi;
                bounds_out[2] = g.ax[1].lo;
                bounds_out[3] = g.ax[1].hi;
            } else if (bounds_out) {
                // collapsed automatic bounds: NaN marks the result as failed
                // for callers that do not read the request's status
                const double qnan = __longlong_as_double(0x7ff8000000000000ll);
                for (int k = 0; k < 4; ++k) bounds_out[k] = qnan;
            }
        }
    }
    __syncthreads();
    if (sizeof(T) != 8 || !g.valid) return;
    const int n0 = g.ax[0].res + 1, n1 = g.ax[1].res + 1;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n0 + n1; j += gridDim.x * blockDim.x) {
        if (j < n0) edges0[j] = edge_key(g.ax[0], j);
        else edges1[j - n0] = edge_key(g.ax[1], j - n0);
    }
}

// ------------------------------------------------------------------ finalise
// avg = sum / count in FP64 (round-to-nearest, bin_average); empty bins get
// the quiet NaN 0x7ff8000000000000.
// With key state (st.mmk), also writes min and max from their keys; with
// count-and-sums records (st.rec), count and sum from the records.
template <typename T>
__global__ void k_finalize(StateDesc st) {
    const int64_t B = st.bins;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    using KO = KeyOf<T>;
    const int rd = record_doubles(st.n_attrs);
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += stride) {
        unsigned long long c;
        const double* r = st.rec ? st.rec + b * rd : nullptr;
        if (r) {
            // the record's count is an integer-valued double below 2^53
            c = (unsigned long long)r[0];
            st.count[b] = c;
        } else {
            c = st.do_avg ? st.count[b] : 0ull;
        }
        for (int a = 0; a < st.n_attrs; ++a) {
            if (r) st.sum[a][b] = r[1 + a];
            if (st.do_avg) st.avg[a][b] = c ? bin_average(r ? r[1 + a] : st.sum[a][b], c) : qnan;
            if (st.mmk) {
                const int rp = key_record_pairs(st.n_attrs, (int)sizeof(typename KO::K));
                const auto k = static_cast<const typename KO::K2*>(st.mmk)[b * rp + a];
                if (st.do_min) static_cast<T*>(st.mn[a])[b] = KO::value(k.x);
                if (st.do_max) static_cast<T*>(st.mx[a])[b] = KO::value(k.y);
            }
        }
    }
}

// ------------------------------------------------------------------ merge
// Combine finalized results of one mesh (the cross-rank merge implied by
// MPI-parallel binning, Sec. 4.2): count and sum add, min/max combine in
// totalOrder. avg is recomputed by k_finalize afterwards.
template <typename T>
__global__ void k_merge(StateDesc out, const StateDesc* parts, int n_parts) {
    const int64_t B = out.bins;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += stride) {
        unsigned long long c = 0;
        for (int p = 0; p < n_parts; ++p) c += parts[p].count[b];
        out.count[b] = c;
        for (int a = 0; a < out.n_attrs; ++a) {
            if (out.do_sum) {
                double s = 0.0;
                for (int p = 0; p < n_parts; ++p) s = __dadd_rn(s, parts[p].sum[a][b]);
                out.sum[a][b] = s;
            }
            if (out.do_min) {
                T m = pos_inf<T>();
                for (int p = 0; p < n_parts; ++p) {
                    T v = static_cast<const T*>(parts[p].mn[a])[b];
                    if (total_less(v, m)) m = v;
                }
                static_cast<T*>(out.mn[a])[b] = m;
            }
            if (out.do_max) {
                T m = neg_inf<T>();
                for (int p = 0; p < n_parts; ++p) {
                    T v = static_cast<const T*>(parts[p].mx[a])[b];
                    if (total_less(m, v)) m = v;
                }
                static_cast<T*>(out.mx[a])[b] = m;
            }
        }
    }
}

// ------------------------------------------------------------------ gather
template <typename T>
__global__ void k_gather(T* __restrict__ dst, const T* __restrict__ src, int64_t n, int64_t stride) {
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step)
        dst[i] = src[i * stride];
}

// ------------------------------------------------------------------ launchers
static inline int grid_for(int64_t work, int block, int max_blocks) {
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

cudaError_t launch_init_state(const KernelCtx& kc, int dtype, const StateDesc& st,
                              void* bounds_acc) {
    const int block = 256;
    int grid = grid_for(st.bins, block, kc.num_sms * 8);
    if (dtype == BN_F64)
        k_init_state<double><<<grid, block, 0, kc.stream>>>(st, static_cast<double*>(bounds_acc));
    else
        k_init_state<float><<<grid, block, 0, kc.stream>>>(st, static_cast<float*>(bounds_acc));
    kc.count_launch();
    return cudaGetLastError();
}

cudaError_t launch_bounds_reduce(const KernelCtx& kc, int dtype, const void* x, const void* y,
                                 int64_t n, void* bounds_acc, int64_t sx, int64_t sy) {
    const int block = 256;
    int grid = grid_for(n, block, kc.num_sms * 8);
    sx = sx > 1 ? sx : 1;
    sy = sy > 1 ? sy : 1;
    if (dtype == BN_F64)
        k_bounds_reduce<double><<<grid, block, 0, kc.stream>>>(
            static_cast<const double*>(x), static_cast<const double*>(y), n,
            static_cast<double*>(bounds_acc), sx, sy);
    else
        k_bounds_reduce<float><<<grid, block, 0, kc.stream>>>(
            static_cast<const float*>(x), static_cast<const float*>(y), n,
            static_cast<float*>(bounds_acc), sx, sy);
    kc.count_launch();
    return cudaGetLastError();
}

cudaError_t launch_grid_setup(const KernelCtx& kc, int dtype, const GridDesc& host_desc,
                              const void* bounds_acc, GridDesc* dev_desc, long long* edges0,
                              long long* edges1, double* bounds_out, int* status) {
    const int block = 128;
    int grid = 1;
    if (dtype == BN_F64) {
        int64_t n_edges = (int64_t)host_desc.ax[0].res + host_desc.ax[1].res + 2;
        grid = grid_for(n_edges, block, kc.num_sms * 4);
        k_grid_setup<double><<<grid, block, 0, kc.stream>>>(
            host_desc, static_cast<const double*>(bounds_acc), dev_desc, edges0, edges1,
            bounds_out, status);
    } else {
        k_grid_setup<float><<<grid, block, 0, kc.stream>>>(
            host_desc, static_cast<const float*>(bounds_acc), dev_desc, nullptr, nullptr,
            bounds_out, status);
    }
    kc.count_launch();
    return cudaGetLastError();
}

cudaError_t launch_finalize(const KernelCtx& kc, const StateDesc& st, int dtype) {
    const int block = 256;
    int grid = grid_for(st.bins, block, kc.num_sms * 8);
    if (dtype == BN_F32) k_finalize<float><<<grid, block, 0, kc.stream>>>(st);
    else k_finalize<double><<<grid, block, 0, kc.stream>>>(st);
    kc.count_launch();
    return cudaGetLastError();
}

cudaError_t launch_merge(const KernelCtx& kc, int dtype, const StateDesc& out,
                         const StateDesc* dev_parts, int n_parts) {
    const int block = 256;
    int grid = grid_for(out.bins, block, kc.num_sms * 8);
    if (dtype == BN_F64)
        k_merge<double><<<grid, block, 0, kc.stream>>>(out, dev_parts, n_parts);
    else
        k_merge<float><<<grid, block, 0, kc.stream>>>(out, dev_parts, n_parts);
    kc.count_launch();
    return cudaGetLastError();
}

cudaError_t launch_gather(const KernelCtx& kc, int dtype, void* dst, const void* src, int64_t n,
                          int64_t stride) {
    const int block = 256;
    int grid = grid_for(n, block, kc.num_sms * 8);
    if (dtype == BN_F64)
        k_gather<double><<<grid, block, 0, kc.stream>>>(static_cast<double*>(dst),
                                                        static_cast<const double*>(src), n, stride);
    else
        k_gather<float><<<grid, block, 0, kc.stream>>>(static_cast<float*>(dst),
                                                       static_cast<const float*>(src), n, stride);
    kc.count_launch();
    return cudaGetLastError();
}

double host_fast_delta(double lo, double hi, double s, int res) { return fast_delta(lo, hi, s, res); }

}  // namespace bn
