// exchange.cu -- partial meshes across ranks (Sec. 4.2: the binning is
// parallelised with MPI, each rank binning the bodies of its own subdomain,
// so the per-rank meshes must combine) and automatic device placement
// (Sec. 3, Eq. 1).
//
// A rank's result is packed into one contiguous exchange buffer whose four
// sections each combine across ranks with one plain element-wise collective:
//   count   u64 [B]       sum
//   sum     f64 [A][B]    sum
//   minkey  s64 [A][B]    min
//   maxkey  s64 [A][B]    max
// The keys are the IEEE totalOrder keys of the min / max values (negative
// values with the magnitude bits flipped), widened to 64 bits for f32 data,
// so an integer min / max is the totalOrder min / max: -0 < +0, and the
// empty-bin values +inf / -inf are the identities. Min and max outputs never
// hold NaN (NaN attributes are skipped), so every key is a value's. After
// the collective, unpacking writes count, sum, min and max back and
// recomputes avg = sum / count (FP64, round to nearest; qNaN when empty).
#include <cuda_runtime.h>

#include <cstring>

#include "bn_device.cuh"
#include "bn_runtime.h"

using namespace bn;

namespace {

__device__ __forceinline__ long long key64(double v) { return KeyOf<double>::key(v); }
__device__ __forceinline__ long long key64(float v) { return (long long)KeyOf<float>::key(v); }
template <typename T> __device__ __forceinline__ T from_key64(long long k);
template <> __device__ __forceinline__ double from_key64<double>(long long k) { return KeyOf<double>::value(k); }
template <> __device__ __forceinline__ float from_key64<float>(long long k) { return KeyOf<float>::value((int)k); }

struct ExchangeView {
    unsigned long long* count;
    double* sum;
    long long* minkey;
    long long* maxkey;
};

ExchangeView view_of(void* ex, int64_t B, int A) {
    char* p = static_cast<char*>(ex);
    ExchangeView v;
    v.count = reinterpret_cast<unsigned long long*>(p);
    v.sum = reinterpret_cast<double*>(p + 8 * B);
    v.minkey = reinterpret_cast<long long*>(p + 8 * B + 8 * A * B);
    v.maxkey = reinterpret_cast<long long*>(p + 8 * B + 16 * A * B);
    return v;
}

template <typename T>
__global__ void k_exchange_pack(StateDesc st, ExchangeView ex) {
    const int64_t B = st.bins;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += stride) {
        ex.count[b] = st.count[b];
        for (int a = 0; a < st.n_attrs; ++a) {
            const int64_t k = (int64_t)a * B + b;
            ex.sum[k] = st.sum[a][b];
            ex.minkey[k] = key64(static_cast<const T*>(st.mn[a])[b]);
            ex.maxkey[k] = key64(static_cast<const T*>(st.mx[a])[b]);
        }
    }
}

template <typename T>
__global__ void k_exchange_unpack(ExchangeView ex, StateDesc st) {
    const int64_t B = st.bins;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += stride) {
        const unsigned long long c = ex.count[b];
        st.count[b] = c;
        for (int a = 0; a < st.n_attrs; ++a) {
            const int64_t k = (int64_t)a * B + b;
            const double s = ex.sum[k];
            if (st.do_sum) st.sum[a][b] = s;
            if (st.do_min) static_cast<T*>(st.mn[a])[b] = from_key64<T>(ex.minkey[k]);
            if (st.do_max) static_cast<T*>(st.mx[a])[b] = from_key64<T>(ex.maxkey[k]);
            if (st.do_avg) st.avg[a][b] = c ? bin_average(s, c) : qnan;
        }
    }
}

int grid_for(int64_t B, int sms) {
    int64_t g = (B + 255) / 256;
    if (g > (int64_t)sms * 8) g = (int64_t)sms * 8;
    return g < 1 ? 1 : (int)g;
}

// A device buffer of the context's device holding at least `need` elements.
bn_status dev_buffer(const bn_context* c, const bn_buffer& b, int64_t need, int dtype, const char* what,
                     void** out) {
    if (!b.ptr) return fail(BN_ERR_INVALID_ARG, "%s: missing", what);
    if (b.device != c->device)
        return fail(BN_ERR_DEVICE_MISMATCH, "%s: must be device memory of device %d", what, c->device);
    if (b.stride > 1) return fail(BN_ERR_INVALID_ARG, "%s: must be contiguous", what);
    if (b.dtype != dtype) return fail(BN_ERR_INVALID_ARG, "%s: dtype %d, expected %d", what, b.dtype, dtype);
    if (b.n < need) return fail(BN_ERR_INVALID_ARG, "%s: holds %lld elements, needs %lld", what,
                                (long long)b.n, (long long)need);
    if ((uintptr_t)b.ptr % (dtype == BN_F32 ? 4 : 8))
        return fail(BN_ERR_INVALID_ARG, "%s: misaligned", what);
    *out = b.ptr;
    return BN_OK;
}

bn_status check_shape(int32_t dtype, int n_attrs, int64_t bins, const void* exchange) {
    if (dtype != BN_F32 && dtype != BN_F64) return fail(BN_ERR_INVALID_ARG, "exchange: dtype must be BN_F32 or BN_F64");
    if (n_attrs < 0 || n_attrs > BN_MAX_ATTR) return fail(BN_ERR_INVALID_ARG, "exchange: n_attrs out of range");
    if (bins < 1 || bins > (int64_t)BN_MAX_BINS) return fail(BN_ERR_INVALID_ARG, "exchange: bins out of range");
    if (!exchange || (uintptr_t)exchange % 8) return fail(BN_ERR_INVALID_ARG, "exchange: buffer missing or not 8-byte aligned");
    return BN_OK;
}

}  // namespace

extern "C" size_t bn_exchange_bytes(int64_t bins, int n_attrs) {
    if (bins < 1 || n_attrs < 0 || n_attrs > BN_MAX_ATTR) return 0;
    return (size_t)bins * 8 * (1 + 3 * (size_t)n_attrs);
}

// Shared body of pack and unpack: one request, one kernel on the context's
// stream, ordered after every buffer's owning stream.
static bn_status exchange_call(bn_context* c, bool pack, void* exchange, int32_t dtype, int n_attrs,
                               int64_t bins, uint32_t ops, const bn_result* in, bn_result* out, int sync,
                               bn_request** req, const char* name) {
    if (!c || (pack ? !in : !out)) return fail(BN_ERR_INVALID_ARG, "%s: NULL argument", name);
    if (!sync && !req) return fail(BN_ERR_INVALID_ARG, "%s: asynchronous call needs req", name);
    bn_status st = check_shape(dtype, n_attrs, bins, exchange);
    if (st != BN_OK) return st;
    if (req) *req = nullptr;
    DeviceGuard g(c->device);
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, exchange) != cudaSuccess || pa.type != cudaMemoryTypeDevice ||
        pa.device != c->device) {
        cudaGetLastError();
        return fail(BN_ERR_DEVICE_MISMATCH, "%s: the exchange buffer must be device memory of device %d", name,
                    c->device);
    }
    std::lock_guard<std::mutex> lk(c->enqueue_mu);
    bn_request* r = new_request(c);
    if (!r) return fail(BN_ERR_NO_MEMORY, "%s: no request slot", name);
    Plan plan(c);
    StateDesc sd;
    memset(&sd, 0, sizeof sd);
    sd.bins = bins;
    sd.n_attrs = n_attrs;
    const bn_result* res = pack ? in : out;
    const uint32_t want = pack ? (uint32_t)BN_OP_ALL : ops;
    sd.do_sum = (want & BN_OP_SUM) ? 1 : 0;
    sd.do_min = (want & BN_OP_MIN) ? 1 : 0;
    sd.do_max = (want & BN_OP_MAX) ? 1 : 0;
    sd.do_avg = (want & BN_OP_AVG) ? 1 : 0;
    void* q = nullptr;
    auto use = [&](const bn_buffer& b, int dt, const char* what, void** o) -> bn_status {
        bn_status s2 = dev_buffer(c, b, bins, dt, what, o);
        if (s2 == BN_OK) s2 = plan.wait_on(b.stream);
        if (s2 == BN_OK && !pack) plan.out_streams.push_back(b.stream);
        return s2;
    };
    st = use(res->count, BN_U64, "count", &q);
    sd.count = static_cast<unsigned long long*>(q);
    for (int a = 0; a < n_attrs && st == BN_OK; ++a) {
        if (pack || sd.do_sum) {
            st = use(res->sum[a], BN_F64, "sum", &q);
            sd.sum[a] = static_cast<double*>(q);
        }
        if (st == BN_OK && (pack || sd.do_min)) st = use(res->min[a], dtype, "min", &sd.mn[a]);
        if (st == BN_OK && (pack || sd.do_max)) st = use(res->max[a], dtype, "max", &sd.mx[a]);
        if (st == BN_OK && sd.do_avg) {
            st = use(res->avg[a], BN_F64, "avg", &q);
            sd.avg[a] = static_cast<double*>(q);
        }
    }
    if (st == BN_OK) {
        const ExchangeView ex = view_of(exchange, bins, n_attrs);
        const int grid = grid_for(bins, c->num_sms);
        if (pack) {
            if (dtype == BN_F64) k_exchange_pack<double><<<grid, 256, 0, c->stream>>>(sd, ex);
            else k_exchange_pack<float><<<grid, 256, 0, c->stream>>>(sd, ex);
        } else {
            if (dtype == BN_F64) k_exchange_unpack<double><<<grid, 256, 0, c->stream>>>(ex, sd);
            else k_exchange_unpack<float><<<grid, 256, 0, c->stream>>>(ex, sd);
        }
        c->launches.fetch_add(1, std::memory_order_relaxed);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, name);
    }
    if (st == BN_OK) st = plan.finish(r);
    if (st != BN_OK) {
        const std::string msg = bn_last_error();
        plan.free_temps();
        cudaEventRecord(r->done, c->stream);
        r->host_status = st;
        bn_request_release(r);
        fail(st, "%s", msg.c_str());
        return st;
    }
    return complete_sync(r, sync, req);
}

extern "C" bn_status bn_exchange_pack(bn_context* c, const bn_result* partial, int32_t dtype, int n_attrs,
                                      int64_t bins, void* exchange, int sync, bn_request** req) {
    return exchange_call(c, true, exchange, dtype, n_attrs, bins, BN_OP_ALL, partial, nullptr, sync, req,
                         "bn_exchange_pack");
}

extern "C" bn_status bn_exchange_unpack(bn_context* c, const void* exchange, int32_t dtype, int n_attrs,
                                        int64_t bins, uint32_t ops, bn_result* out, int sync,
                                        bn_request** req) {
    return exchange_call(c, false, const_cast<void*>(exchange), dtype, n_attrs, bins, ops | BN_OP_COUNT,
                         nullptr, out, sync, req, "bn_exchange_unpack");
}

// Eq. 1 (Sec. 3): d = ((r mod n_u) * s + d_0) mod n_a.
extern "C" bn_status bn_select_device(int rank, int n_use, int stride, int offset, int n_avail, int* device) {
    if (!device) return fail(BN_ERR_INVALID_ARG, "bn_select_device: device is NULL");
    if (rank < 0) return fail(BN_ERR_INVALID_ARG, "bn_select_device: negative rank");
    if (n_avail < 1) return fail(BN_ERR_INVALID_ARG, "bn_select_device: no device available");
    if (n_use <= 0) n_use = n_avail;  // the paper's defaults: n_u = n_a, s = 1, d_0 = 0
    if (stride <= 0) stride = 1;
    const long long d = ((long long)(rank % n_use) * stride + offset) % n_avail;
    *device = (int)(d < 0 ? d + n_avail : d);
    return BN_OK;
}
