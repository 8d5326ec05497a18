// runtime.cu -- the C ABI of libbinning.so (include/binning.h): contexts,
// buffer handles, stream ordering, staging of host data, strategy choice and
// request completion. Kernels live in k_*.cu; this file only plans and
// queues them.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "bn_internal.cuh"
#include "bn_kernels.h"
#include "bn_runtime.h"

using namespace bn;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

bn_status bn::fail(bn_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

bn_status bn::cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? BN_ERR_NO_MEMORY : BN_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

extern "C" const char* bn_last_error(void) { return g_err.c_str(); }
extern "C" const char* bn_version(void) { return "binning 0.1 (sm_103a)"; }

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

// ------------------------------------------------------------------ context

static const int kStatusSlots = 4096;

extern "C" bn_status bn_context_create(int device, const bn_options* opt, bn_context** out) {
    if (!out) return fail(BN_ERR_INVALID_ARG, "bn_context_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev)
        return fail(BN_ERR_INVALID_ARG, "bn_context_create: no CUDA device %d (%d present)", device, ndev);
    DeviceGuard g(device);
    auto* c = new (std::nothrow) bn_context();
    if (!c) return fail(BN_ERR_NO_MEMORY, "bn_context_create: out of host memory");
    c->device = device;
    cudaDeviceProp p;
    e = cudaGetDeviceProperties(&p, device);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaGetDeviceProperties"); }
    c->num_sms = p.multiProcessorCount;
    c->profile = opt && (opt->flags & BN_CTX_PROFILE);
    c->smem_optin = (int)p.sharedMemPerBlockOptin;
    if (opt && opt->stream) {
        c->stream = static_cast<cudaStream_t>(opt->stream);
        c->own_stream = false;
    } else {
        int prio = opt ? opt->stream_priority : 0;
        e = cudaStreamCreateWithPriority(&c->stream, cudaStreamNonBlocking, prio);
        if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaStreamCreateWithPriority"); }
        c->own_stream = true;
    }
    e = cudaDeviceGetDefaultMemPool(&c->pool, device);
    if (e == cudaSuccess) {
        uint64_t thr = (opt && opt->mempool_release_threshold) ? opt->mempool_release_threshold
                                                                : UINT64_MAX;
        cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    e = cudaHostAlloc(reinterpret_cast<void**>(&c->status_host), kStatusSlots * sizeof(int),
                      cudaHostAllocMapped);
    if (e != cudaSuccess) {
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return cuda_fail(e, "cudaHostAlloc(status)");
    }
    e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->status_dev), c->status_host, 0);
    if (e != cudaSuccess) {
        cudaFreeHost(c->status_host);
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return cuda_fail(e, "cudaHostGetDevicePointer(status)");
    }
    memset(c->status_host, 0, kStatusSlots * sizeof(int));
    for (int i = kStatusSlots - 1; i >= 0; --i) c->free_slots.push_back(i);
    *out = c;
    return BN_OK;
}

extern "C" bn_status bn_context_destroy(bn_context* c) {
    if (!c) return BN_OK;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    batch_cache_release(c);
    for (cudaEvent_t ev : c->event_pool) cudaEventDestroy(ev);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    cudaFreeHost(c->status_host);
    delete c;
    return BN_OK;
}

extern "C" bn_status bn_context_stream(bn_context* c, void** stream) {
    if (!c || !stream) return fail(BN_ERR_INVALID_ARG, "bn_context_stream: NULL argument");
    *stream = c->stream;
    return BN_OK;
}

extern "C" bn_status bn_context_profile(bn_context* c, double* total_ms, uint64_t* n,
                                        int32_t* last_strategy) {
    if (!c || !total_ms || !n) return fail(BN_ERR_INVALID_ARG, "bn_context_profile: NULL argument");
    if (last_strategy) *last_strategy = c->last_strategy;
    DeviceGuard g(c->device);
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pairs;
    {
        std::lock_guard<std::mutex> lk(c->prof_mu);
        pairs.swap(c->prof_pairs);
    }
    double tot = 0.0;
    bn_status st = BN_OK;
    for (auto& pr : pairs) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(pr.second);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
        if (e != cudaSuccess && st == BN_OK) st = cuda_fail(e, "bn_context_profile");
        tot += ms;
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    *total_ms = tot;
    *n = pairs.size();
    return st;
}

extern "C" bn_status bn_context_autotune_report(bn_context* c, char* buf, size_t cap) {
    if (!c || !buf || cap == 0) return fail(BN_ERR_INVALID_ARG, "bn_context_autotune_report: bad arguments");
    std::string all;
    {
        std::lock_guard<std::mutex> lk(c->tune_mu);
        for (const std::string& l : c->tune_log) all += l + "\n";
    }
    const size_t k = std::min(all.size(), cap - 1);
    memcpy(buf, all.data(), k);
    buf[k] = '\0';
    return BN_OK;
}

extern "C" bn_status bn_context_launch_count(bn_context* c, uint64_t* n) {
    if (!c || !n) return fail(BN_ERR_INVALID_ARG, "bn_context_launch_count: NULL argument");
    *n = c->launches.load();
    return BN_OK;
}

cudaEvent_t bn_context::get_event() {
    std::lock_guard<std::mutex> lk(pool_mu);
    if (!event_pool.empty()) {
        cudaEvent_t ev = event_pool.back();
        event_pool.pop_back();
        return ev;
    }
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return ev;
}

void bn_context::put_event(cudaEvent_t ev) {
    if (!ev) return;
    std::lock_guard<std::mutex> lk(pool_mu);
    event_pool.push_back(ev);
}

int bn_context::get_slot() {
    std::lock_guard<std::mutex> lk(pool_mu);
    if (free_slots.empty()) return -1;
    int s = free_slots.back();
    free_slots.pop_back();
    status_host[s] = 0;
    return s;
}

void bn_context::put_slot(int s) {
    if (s < 0) return;
    std::lock_guard<std::mutex> lk(pool_mu);
    free_slots.push_back(s);
}

// ------------------------------------------------------------------ requests
bn_request* bn::new_request(bn_context* c) {
    auto* r = new (std::nothrow) bn_request();
    if (!r) return nullptr;
    r->ctx = c;
    r->slot = c->get_slot();
    r->done = c->get_event();
    if (r->slot < 0 || !r->done) {
        c->put_slot(r->slot);
        c->put_event(r->done);
        delete r;
        return nullptr;
    }
    return r;
}

static bn_status request_status_now(bn_request* r) {
    if (r->host_status != BN_OK) return r->host_status;
    if (r->external_done) {
        int st = r->external_done->load(std::memory_order_acquire);
        if (st == BN_NOT_READY) return BN_NOT_READY;
        return (bn_status)st;
    }
    cudaError_t e = cudaEventQuery(r->done);
    if (e == cudaErrorNotReady) return BN_NOT_READY;
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventQuery");
    int st = r->ctx->status_host[r->slot];
    return (bn_status)st;
}

extern "C" bn_status bn_query(bn_request* r) {
    if (!r) return fail(BN_ERR_INVALID_ARG, "bn_query: NULL request");
    DeviceGuard g(r->ctx->device);
    return request_status_now(r);
}

extern "C" bn_status bn_wait(bn_request* r, int64_t timeout_us) {
    if (!r) return fail(BN_ERR_INVALID_ARG, "bn_wait: NULL request");
    DeviceGuard g(r->ctx->device);
    if (timeout_us < 0 && !r->external_done && r->host_status == BN_OK) {
        cudaError_t e = cudaEventSynchronize(r->done);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        return request_status_now(r);
    }
    auto t0 = std::chrono::steady_clock::now();
    int64_t spin = 0;
    for (;;) {
        bn_status st = request_status_now(r);
        if (st != BN_NOT_READY) return st;
        auto el = std::chrono::duration_cast<std::chrono::microseconds>(
                      std::chrono::steady_clock::now() - t0).count();
        if (timeout_us >= 0 && el >= timeout_us)
            return fail(BN_ERR_TIMEOUT, "bn_wait: request still running after %lld us",
                        (long long)timeout_us);
        if (++spin > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

void bn::run_deleters(bn_request* r) {
    for (auto& d : r->deleters) d.fn(d.ptr, d.ctx);
    r->deleters.clear();
}

extern "C" bn_status bn_request_release(bn_request* r) {
    if (!r) return BN_OK;
    DeviceGuard g(r->ctx->device);
    if (r->external_done) {
        while (r->external_done->load(std::memory_order_acquire) == BN_NOT_READY)
            std::this_thread::sleep_for(std::chrono::microseconds(50));
    } else if (r->host_status == BN_OK) {
        cudaEventSynchronize(r->done);
    }
    run_deleters(r);
    if (r->on_release) r->on_release(r);
    r->ctx->put_event(r->done);
    r->ctx->put_slot(r->slot);
    delete r;
    return BN_OK;
}

// Library outputs return to the stream-ordered pool on the stream that
// allocated them (ctx): no device-wide synchronisation, and ordered after
// every kernel the library queued there.
static void lib_free_deleter(void* ptr, void* ctx) {
    if (ptr) cudaFreeAsync(ptr, static_cast<cudaStream_t>(ctx));
}

extern "C" bn_status bn_buffer_release(bn_buffer* b) {
    if (!b) return BN_OK;
    if (b->deleter) b->deleter(b->ptr, b->deleter_ctx);
    memset(b, 0, sizeof *b);
    return BN_OK;
}

// ------------------------------------------------------------------ planning
static int dtype_size(int dt) { return dt == BN_F32 ? 4 : 8; }

bn_status bn::validate_buffer(const bn_context* c, const bn_buffer* b, int64_t n, int dtype,
                              const char* what) {
    if (!b) return fail(BN_ERR_INVALID_ARG, "%s: NULL buffer", what);
    if (b->n != n) return fail(BN_ERR_INVALID_ARG, "%s: length %lld, expected %lld", what,
                               (long long)b->n, (long long)n);
    if (b->dtype != dtype)
        return fail(BN_ERR_INVALID_ARG, "%s: dtype %d, expected %d", what, b->dtype, dtype);
    if (n > 0 && !b->ptr) return fail(BN_ERR_INVALID_ARG, "%s: NULL pointer", what);
    if (b->stride < 0) return fail(BN_ERR_INVALID_ARG, "%s: negative stride", what);
    if (b->device != BN_HOST && b->device != c->device) {
        // another CUDA device of this process: staged (Plan::column)
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || b->device < 0 || b->device >= ndev) {
            cudaGetLastError();
            return fail(BN_ERR_DEVICE_MISMATCH, "%s: buffer on device %d, which this process does not have", what,
                        b->device);
        }
    }
    if (b->ptr && ((uintptr_t)b->ptr % (uintptr_t)dtype_size(dtype)) != 0)
        return fail(BN_ERR_INVALID_ARG, "%s: pointer not aligned to its element size", what);
    return BN_OK;
}

// Host-side mesh set-up for explicit bounds, in the coordinate type T:
// lo_T = (T)lo, hi_T = (T)hi, s_T = (T)res / (hi_T - lo_T).
template <typename T>
static bn_status make_axis_host(double lo, double hi, int res, AxisDesc* d) {
    if (!std::isfinite(lo) || !std::isfinite(hi))
        return fail(BN_ERR_INVALID_ARG, "grid: bounds must be finite");
    volatile T lo_t = (T)lo;
    volatile T hi_t = (T)hi;
    volatile T w = (T)(hi_t - lo_t);
    if (!(w > (T)0) || !std::isfinite((double)w))
        return fail(BN_ERR_INVALID_ARG, "grid: lo must be below hi (after rounding to the data type)");
    volatile T s = (T)((T)res / w);
    if (!(s > (T)0) || !std::isfinite((double)s))
        return fail(BN_ERR_INVALID_ARG, "grid: res / (hi - lo) is not finite");
    d->lo = (double)lo_t;
    d->hi = (double)hi_t;
    d->s = (double)s;
    d->res = res;
    d->closed = 0;
    d->fast = 0;
    d->delta = 0.0f;
    return BN_OK;
}

bn_status bn::make_grid_desc(const bn_grid* g, int dtype, GridDesc* out) {
    if (!g) return fail(BN_ERR_INVALID_ARG, "grid: NULL");
    for (int a = 0; a < 2; ++a)
        if (g->res[a] < 1 || g->res[a] > BN_MAX_RES)
            return fail(BN_ERR_INVALID_ARG, "grid: res[%d] = %d outside [1, %d]", a, g->res[a], BN_MAX_RES);
    if ((int64_t)g->res[0] * g->res[1] > (int64_t)BN_MAX_BINS)
        return fail(BN_ERR_INVALID_ARG, "grid: more than %d bins", BN_MAX_BINS);
    memset(out, 0, sizeof *out);
    out->valid = 1;
    for (int a = 0; a < 2; ++a) {
        out->ax[a].res = g->res[a];
        if (g->auto_bounds) {
            out->ax[a].closed = 1;
            continue;
        }
        bn_status st = dtype == BN_F64 ? make_axis_host<double>(g->lo[a], g->hi[a], g->res[a], &out->ax[a])
                                       : make_axis_host<float>(g->lo[a], g->hi[a], g->res[a], &out->ax[a]);
        if (st != BN_OK) return st;
    }
    return BN_OK;
}

// Stream-ordered temporaries of one request.
void* Plan::alloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    const size_t rounded = (bytes + 255) & ~(size_t)255;
    cudaError_t e = cudaMallocAsync(&p, rounded, stream);
    if (e != cudaSuccess) {
        err = e;
        return nullptr;
    }
    temps.push_back(p);
    temp_bytes += rounded;
    return p;
}

void Plan::free_temps() {
    for (void* p : temps) cudaFreeAsync(p, stream);
    temps.clear();
}

// Order the execution stream after work already queued on stream s of
// another device: the event is created and recorded on that device.
bn_status Plan::wait_on_peer(void* s, int device) {
    cudaEvent_t ev = nullptr;
    cudaError_t e;
    {
        DeviceGuard g(device);
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, static_cast<cudaStream_t>(s));
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev, 0);
    if (ev) cudaEventDestroy(ev);  // released once the wait has been satisfied
    if (e != cudaSuccess) return cuda_fail(e, "stream ordering (peer device)");
    return BN_OK;
}

// Order the execution stream after work already queued on stream s.
bn_status Plan::wait_on(void* s) {
    cudaStream_t st = static_cast<cudaStream_t>(s);
    if (st == stream) return BN_OK;
    for (void* w : waited)
        if (w == s) return BN_OK;
    waited.push_back(s);
    cudaEvent_t ev = ctx->get_event();
    if (!ev) return fail(BN_ERR_CUDA, "cudaEventCreate failed");
    cudaError_t e = cudaEventRecord(ev, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev, 0);
    ctx->put_event(ev);  // safe: a recorded event may be re-recorded later
    if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
    return BN_OK;
}

// A device pointer with the column's data: the buffer itself (zero copy), or
// a contiguous staged copy (host data, or strided device data when the
// caller cannot read strided columns: stride_out == nullptr). With
// stride_out, a strided device column is used in place and its element
// stride returned (1 otherwise).
bn_status Plan::column(const bn_buffer* b, int dtype, const void** out, int64_t* stride_out) {
    const size_t es = dtype_size(dtype);
    const int64_t n = b->n;
    if (n == 0) {
        *out = nullptr;
        return BN_OK;
    }
    const int64_t stride = b->stride <= 1 ? 1 : b->stride;
    if (stride_out) *stride_out = 1;
    if (b->device != BN_HOST && b->device != ctx->device) {
        // another device (location-agnostic access, Sec. 2: moved to the
        // device that runs the work, into a temporary freed with the
        // request): one peer copy of the column's span, after the work
        // queued on its owning stream
        bn_status st = wait_on_peer(b->stream, b->device);
        if (st != BN_OK) return st;
        const size_t span = ((size_t)(n - 1) * stride + 1) * es;
        void* t = alloc(span);
        if (!t) return cuda_fail(err, "cudaMallocAsync(peer column)");
        cudaError_t e = cudaMemcpyPeerAsync(t, ctx->device, b->ptr, b->device, span, stream);
        if (e != cudaSuccess) return cuda_fail(e, "copy column from peer device");
        p2p_bytes += span;
        if (stride == 1 || stride_out) {
            if (stride_out) *stride_out = stride;
            *out = t;
            return BN_OK;
        }
        void* g = alloc((size_t)n * es);
        if (!g) return cuda_fail(err, "cudaMallocAsync(column)");
        e = launch_gather(kc(), dtype, g, t, n, stride);
        if (e != cudaSuccess) return cuda_fail(e, "gather kernel");
        *out = g;
        return BN_OK;
    }
    if (b->device != BN_HOST) {
        bn_status st = wait_on(b->stream);
        if (st != BN_OK) return st;
        if (stride == 1) {
            *out = b->ptr;
            return BN_OK;
        }
        if (stride_out) {
            *out = b->ptr;
            *stride_out = stride;
            return BN_OK;
        }
        void* t = alloc((size_t)n * es);
        if (!t) return cuda_fail(err, "cudaMallocAsync(column)");
        cudaError_t e = launch_gather(kc(), dtype, t, b->ptr, n, stride);
        if (e != cudaSuccess) return cuda_fail(e, "gather kernel");
        *out = t;
        return BN_OK;
    }
    // host memory: the location-agnostic access of Sec. 2. Page-locked host
    // memory is mapped into the device's address space: the kernels read a
    // contiguous page-locked column in place over the host link (each input
    // is read once, coalesced), with no temporary and no separate copy.
    // Other host memory is moved into a temporary.
    if (stride == 1) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, b->ptr) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer) {
            h2d_bytes += (size_t)n * es;
            *out = pa.devicePointer;
            return BN_OK;
        }
        cudaGetLastError();  // an unregistered pointer is not an error here
    }
    void* t = alloc((size_t)n * es);
    if (!t) return cuda_fail(err, "cudaMallocAsync(host column)");
    cudaError_t e;
    if (stride == 1)
        e = cudaMemcpyAsync(t, b->ptr, (size_t)n * es, cudaMemcpyHostToDevice, stream);
    else
        e = cudaMemcpy2DAsync(t, es, b->ptr, (size_t)stride * es, es, (size_t)n,
                              cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy host column");
    h2d_bytes += (size_t)n * es;
    *out = t;
    return BN_OK;
}

// Device storage for one per-bin output: the caller's device buffer, a
// library allocation handed back to the caller, or a temporary (host
// outputs, or state the caller did not ask for). load: copy the caller's
// host data in first (accumulate mode).
bn_status Plan::output(bn_buffer* b, bool wanted, int64_t bins, int dtype, bool load, void** out) {
    const size_t es = dtype_size(dtype);
    if (wanted && b && b->ptr) {
        if (b->n < bins) return fail(BN_ERR_INVALID_ARG, "output buffer holds %lld elements, mesh has %lld",
                                     (long long)b->n, (long long)bins);
        if (b->dtype != dtype) return fail(BN_ERR_INVALID_ARG, "output dtype %d, expected %d", b->dtype, dtype);
        if (b->stride > 1) return fail(BN_ERR_INVALID_ARG, "output buffers must be contiguous");
        if (((uintptr_t)b->ptr % es) != 0) return fail(BN_ERR_INVALID_ARG, "output pointer misaligned");
        if (b->device != BN_HOST && b->device != ctx->device) {
            // another device: a temporary here, copied to the peer buffer when
            // the work is done, ordered before later work on its stream
            int ndev = 0;
            if (cudaGetDeviceCount(&ndev) != cudaSuccess || b->device < 0 || b->device >= ndev) {
                cudaGetLastError();
                return fail(BN_ERR_DEVICE_MISMATCH, "output on device %d, which this process does not have",
                            b->device);
            }
            bn_status st = wait_on_peer(b->stream, b->device);
            if (st != BN_OK) return st;
            void* t = alloc((size_t)bins * es);
            if (!t) return cuda_fail(err, "cudaMallocAsync(peer output)");
            if (load) {
                cudaError_t e = cudaMemcpyPeerAsync(t, ctx->device, b->ptr, b->device, (size_t)bins * es, stream);
                if (e != cudaSuccess) return cuda_fail(e, "copy peer output in");
                p2p_bytes += (size_t)bins * es;
            }
            peer_out.push_back({b->ptr, b->device, b->stream, t, (size_t)bins * es});
            *out = t;
            return BN_OK;
        }
        if (b->device != BN_HOST) {
            bn_status st = wait_on(b->stream);
            if (st != BN_OK) return st;
            out_streams.push_back(b->stream);
            *out = b->ptr;
            return BN_OK;
        }
        void* t = alloc((size_t)bins * es);
        if (!t) return cuda_fail(err, "cudaMallocAsync(output)");
        if (load) {
            cudaError_t e = cudaMemcpyAsync(t, b->ptr, (size_t)bins * es, cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) return cuda_fail(e, "copy host output in");
            h2d_bytes += (size_t)bins * es;
        }
        d2h.push_back({b->ptr, t, (size_t)bins * es});
        *out = t;
        return BN_OK;
    }
    if (wanted && b && !b->ptr) {
        if (load) return fail(BN_ERR_INVALID_ARG, "accumulate needs existing output buffers");
        void* p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, (size_t)bins * es, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(library output)");
        b->ptr = p;
        b->n = bins;
        b->stride = 1;
        b->dtype = dtype;
        b->device = ctx->device;
        b->stream = stream;
        b->alloc = BN_ALLOC_CUDA_ASYNC;
        b->deleter = lib_free_deleter;
        b->deleter_ctx = stream;
        *out = p;
        return BN_OK;
    }
    if (load) return fail(BN_ERR_INVALID_ARG, "accumulate needs count, sum, min and max outputs");
    void* t = alloc((size_t)bins * es);
    if (!t) return cuda_fail(err, "cudaMallocAsync(state)");
    *out = t;
    return BN_OK;
}

bn_status Plan::finish(bn_request* r) {
    for (auto& c : d2h) {
        cudaError_t e = cudaMemcpyAsync(c.host, c.dev, c.bytes, cudaMemcpyDeviceToHost, stream);
        if (e != cudaSuccess) return cuda_fail(e, "copy output to host");
        d2h_bytes += c.bytes;
    }
    for (auto& c : peer_out) {
        cudaError_t e = cudaMemcpyPeerAsync(c.peer, c.device, c.dev, ctx->device, c.bytes, stream);
        if (e != cudaSuccess) return cuda_fail(e, "copy output to peer device");
        p2p_bytes += c.bytes;
    }
    free_temps();
    cudaError_t e = cudaEventRecord(r->done, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    // later work on a peer output's own stream (on its device) waits for it
    for (auto& c : peer_out) {
        DeviceGuard g(c.device);
        e = cudaStreamWaitEvent(static_cast<cudaStream_t>(c.stream), r->done, 0);
        if (e != cudaSuccess) return cuda_fail(e, "order peer output stream");
    }
    for (void* s : out_streams) {
        if (static_cast<cudaStream_t>(s) == stream) continue;
        e = cudaStreamWaitEvent(static_cast<cudaStream_t>(s), r->done, 0);
        if (e != cudaSuccess) return cuda_fail(e, "order output stream");
    }
    return BN_OK;
}

// ------------------------------------------------------------------ binning
// The largest window of a res_x x res_y mesh whose counts and sums fit one
// CTA's shared memory (k_window.cu), about square; false if none fits or
// the attribute count has no window kernel.
static bool window_shape(int rx, int ry, int n_attrs, bool do_sum, int smem_optin, int* wnx, int* wny) {
    if (n_attrs > kWindowMaxAttr) return false;
    int cells = 0;
    while (window_bytes(cells + 64, n_attrs, do_sum) <= (size_t)(smem_optin - 1024)) cells += 64;
    const int side = (int)std::sqrt((double)cells);
    *wnx = std::min(side, rx);
    *wny = std::min(cells / std::max(*wnx, 1), ry);
    return *wnx >= 1 && *wny >= 1;
}

int bn::choose_strategy(const BinArgs& a, int smem_optin, int num_sms, uint32_t ops) {
    const uint32_t forced = ops & BN_STRATEGY_MASK;
    if (forced == BN_STRATEGY_PRIVATE) return BN_STRATEGY_PRIVATE;
    if (forced == BN_STRATEGY_GLOBAL) return BN_STRATEGY_GLOBAL;
    if (forced == BN_STRATEGY_SORT) return BN_STRATEGY_SORT;
    if (forced == BN_STRATEGY_HYBRID) return BN_STRATEGY_HYBRID;
    const size_t smem = private_smem_bytes(a, smem_optin);
    const int64_t B = (int64_t)a.grid.ax[0].res * a.grid.ax[1].res;
    // Privatise when the mesh fits and there are enough particles per CTA
    // copy of the mesh to amortise clearing and merging it.
    if (smem > 0 && a.n >= 2 * B) return BN_STRATEGY_PRIVATE;
    // Bucketed sort + reduce when the mesh state is larger than L2 (so
    // global atomics would go to DRAM), a pass-1 tile feeds few enough
    // buckets (run reservations at most one per four records), and there is
    // enough work to stream.
    const size_t tsz = a.dtype == BN_F64 ? 8 : 4;
    const double state = (double)B * (8 + a.n_attrs * (8 + 2 * tsz));
    SortDesc sd;
    if (state > 128e6 && sort_plan(a, smem_optin, &sd) && 4 * sd.nb <= sd.tp &&
        a.n >= (int64_t)num_sms * sd.tp && a.n >= B / 4)
        return BN_STRATEGY_SORT;
    return BN_STRATEGY_GLOBAL;
}

// An upper bound on the device temporaries enqueue_bin allocates for one
// block (the server charges it to its budget before admitting the block):
// state the caller did not ask for, device copies of host outputs, min/max
// key records and their filter, the sort path's scratch whenever the mesh
// has a sort plan, the mesh descriptor, edge keys and bounds accumulator.
// The block's columns are taken as contiguous device data.
size_t bn::request_temp_bytes(const bn_context* c, const bn_block& b, int dtype, uint32_t ops) {
    auto r256 = [](size_t v) { return (std::max(v, (size_t)16) + 255) & ~(size_t)255; };
    const size_t es = dtype_size(dtype);
    const int64_t B = (int64_t)b.grid.res[0] * b.grid.res[1];
    const bool want_avg = ops & BN_OP_AVG, want_sum = ops & BN_OP_SUM;
    const bool want_min = ops & BN_OP_MIN, want_max = ops & BN_OP_MAX, want_count = ops & BN_OP_COUNT;
    const int A = (want_sum || want_avg || want_min || want_max) ? b.n_attrs : 0;
    const bn_result* o = b.out;
    auto host_or_missing = [&](const bn_buffer& buf, bool wanted) {
        return !wanted || !buf.ptr || buf.device == BN_HOST;
    };
    size_t t = 0;
    if (host_or_missing(o->count, want_count)) t += r256((size_t)B * 8);
    for (int a = 0; a < A; ++a) {
        if ((want_sum || want_avg) && host_or_missing(o->sum[a], want_sum)) t += r256((size_t)B * 8);
        if (want_min && o->min[a].device == BN_HOST) t += r256((size_t)B * es);
        if (want_max && o->max[a].device == BN_HOST) t += r256((size_t)B * es);
        if (want_avg && o->avg[a].device == BN_HOST) t += r256((size_t)B * 8);
    }
    if (A >= 1 && A <= kRecMaxAttr && (want_sum || want_avg)) t += r256((size_t)record_doubles(A) * B * 8);
    if (A > 0 && (want_min || want_max)) {
        t += r256((size_t)key_record_pairs(A, (int)es) * B * 2 * es);
        if (dtype == BN_F64 && A >= 3) t += r256((size_t)filter_record_pairs(A) * B * sizeof(int2));
    }
    BinArgs a;
    memset(&a, 0, sizeof a);
    a.dtype = dtype;
    a.n_attrs = A;
    a.n = b.x.n;
    a.sum_mode = dtype == BN_F64 ? kSumF64 : (ops & BN_SUM_MASK) == BN_SUM_F32 ? kSumF32
                                           : (ops & BN_SUM_MASK) == BN_SUM_F64 ? kSumF64 : kSumF32C;
    a.grid.ax[0].res = b.grid.res[0];
    a.grid.ax[1].res = b.grid.res[1];
    a.st.do_sum = (want_sum || want_avg) ? 1 : 0;
    a.st.do_min = want_min;
    a.st.do_max = want_max;
    SortDesc sd;
    if (sort_plan(a, c->smem_optin, &sd)) t += r256(sort_scratch_bytes(sd, a));
    t += r256(sizeof(GridDesc)) + r256(4 * es);
    if (dtype == BN_F64) t += r256(8 * ((size_t)b.grid.res[0] + 1)) + r256(8 * ((size_t)b.grid.res[1] + 1));
    if (o->bounds.ptr && o->bounds.device == BN_HOST) t += r256(4 * 8);
    return t;
}

bn_status bn::enqueue_bin(bn_context* c, Plan& plan, const bn_buffer* x, const bn_buffer* y,
                          const bn_buffer* attrs, int n_attrs, const bn_grid* grid, uint32_t ops,
                          bn_result* out, int* status_dev) {
    if (!x || !y || !grid || !out) return fail(BN_ERR_INVALID_ARG, "bn_bin_particles: NULL argument");
    if (n_attrs < 0 || n_attrs > BN_MAX_ATTR)
        return fail(BN_ERR_INVALID_ARG, "n_attrs = %d outside [0, %d]", n_attrs, BN_MAX_ATTR);
    if (n_attrs > 0 && !attrs) return fail(BN_ERR_INVALID_ARG, "attrs is NULL");
    const int dtype = x->dtype;
    if (dtype != BN_F32 && dtype != BN_F64)
        return fail(BN_ERR_INVALID_ARG, "coordinates must be BN_F32 or BN_F64");
    const int64_t n = x->n;
    if (n < 0) return fail(BN_ERR_INVALID_ARG, "negative length");
    bn_status st = validate_buffer(c, x, n, dtype, "x");
    if (st == BN_OK) st = validate_buffer(c, y, n, dtype, "y");
    for (int a = 0; a < n_attrs && st == BN_OK; ++a) st = validate_buffer(c, &attrs[a], n, dtype, "attr");
    if (st != BN_OK) return st;
    if ((ops & BN_STRATEGY_MASK) > BN_STRATEGY_HYBRID)
        return fail(BN_ERR_INVALID_ARG, "unknown strategy in ops");
    if ((ops & BN_AGG_MASK) == BN_AGG_MASK) return fail(BN_ERR_INVALID_ARG, "unknown aggregation mode in ops");
    const uint32_t sum_bits = ops & BN_SUM_MASK;
    if (sum_bits == (3u << 8)) return fail(BN_ERR_INVALID_ARG, "unknown sum mode in ops");

    GridDesc gd;
    st = make_grid_desc(grid, dtype, &gd);
    if (st != BN_OK) return st;
    const int64_t B = (int64_t)grid->res[0] * grid->res[1];
    const bool accumulate = (ops & BN_OP_ACCUMULATE) != 0;
    const bool want_avg = (ops & BN_OP_AVG) != 0;
    const bool want_sum = (ops & BN_OP_SUM) != 0;
    const bool want_min = (ops & BN_OP_MIN) != 0;
    const bool want_max = (ops & BN_OP_MAX) != 0;
    const bool want_count = (ops & BN_OP_COUNT) != 0;
    if (accumulate && (!want_count || (n_attrs > 0 && (!want_sum || !want_min || !want_max))))
        return fail(BN_ERR_INVALID_ARG, "BN_OP_ACCUMULATE needs count, sum, min and max");
    if (accumulate && grid->auto_bounds)
        return fail(BN_ERR_INVALID_ARG, "BN_OP_ACCUMULATE needs explicit bounds");
    // the attribute columns were validated above; with no per-attribute
    // operation requested they are neither staged nor read
    if (!want_sum && !want_avg && !want_min && !want_max) n_attrs = 0;

    BinArgs args;
    memset(&args, 0, sizeof args);
    args.dtype = dtype;
    args.n_attrs = n_attrs;
    args.sum_mode = dtype == BN_F64 ? kSumF64
                    : sum_bits == BN_SUM_F32 ? kSumF32
                    : sum_bits == BN_SUM_F64 ? kSumF64
                                             : kSumF32C;
    args.n = n;
    // warp aggregation: on request, else for meshes small enough that a warp
    // of random particles often shares bins (clustered data raises that)
    const uint32_t agg = ops & BN_AGG_MASK;
    args.aggregate = agg == BN_AGG_ON ? 1 : agg == BN_AGG_OFF ? 0
                     : ((int64_t)grid->res[0] * grid->res[1] <= 65536 ? 1 : 0);
    // strided device columns are read in place by the private, global and
    // hybrid kernels; the sort path needs them contiguous
    const bool sort_forced = (ops & BN_STRATEGY_MASK) == BN_STRATEGY_SORT;
    st = plan.column(x, dtype, &args.x, sort_forced ? nullptr : &args.sx);
    if (st == BN_OK) st = plan.column(y, dtype, &args.y, sort_forced ? nullptr : &args.sy);
    for (int a = 0; a < n_attrs && st == BN_OK; ++a)
        st = plan.column(&attrs[a], dtype, &args.a[a], sort_forced ? nullptr : &args.sa[a]);
    if (st != BN_OK) return st;
    bool strided = args.sx > 1 || args.sy > 1;
    for (int a = 0; a < n_attrs; ++a) strided = strided || args.sa[a] > 1;

    StateDesc& sd = args.st;
    sd.bins = B;
    sd.n_attrs = n_attrs;
    sd.do_sum = (want_sum || want_avg) ? 1 : 0;
    sd.do_min = want_min ? 1 : 0;
    sd.do_max = want_max ? 1 : 0;
    sd.do_avg = want_avg ? 1 : 0;
    void* p = nullptr;
    st = plan.output(&out->count, want_count, B, BN_U64, accumulate, &p);
    if (st != BN_OK) return st;
    sd.count = static_cast<unsigned long long*>(p);
    for (int a = 0; a < n_attrs; ++a) {
        if (sd.do_sum) {
            st = plan.output(&out->sum[a], want_sum, B, BN_F64, accumulate, &p);
            if (st != BN_OK) return st;
            sd.sum[a] = static_cast<double*>(p);
        }
        if (want_min) {
            st = plan.output(&out->min[a], true, B, dtype, accumulate, &p);
            if (st != BN_OK) return st;
            sd.mn[a] = p;
        }
        if (want_max) {
            st = plan.output(&out->max[a], true, B, dtype, accumulate, &p);
            if (st != BN_OK) return st;
            sd.mx[a] = p;
        }
        if (want_avg) {
            st = plan.output(&out->avg[a], true, B, BN_F64, false, &p);
            if (st != BN_OK) return st;
            sd.avg[a] = static_cast<double*>(p);
        }
    }
    double* bounds_out = nullptr;
    if (out->bounds.ptr) {
        st = plan.output(&out->bounds, true, 4, BN_F64, false, &p);
        if (st != BN_OK) return st;
        bounds_out = static_cast<double*>(p);
    }

    const KernelCtx kc = plan.kc();
    cudaError_t e;
    args.grid = gd;
    // strategy first: the global strategy keeps min/max as key pairs in a
    // temporary (one read per attribute in the hot loop), written to the
    // outputs by the finalise kernel
    int strat = 0;
    SortDesc sortd;
    void* sort_scratch = nullptr;
    bool trial = false;  // measure the candidates on this call's data first
    std::tuple<int, int, uint32_t, int, int, int> klass;
    const uint32_t forced = ops & BN_STRATEGY_MASK;
    const uint32_t aggbits = ops & BN_AGG_MASK;
    if (n > 0) {
        strat = choose_strategy(args, c->smem_optin, c->num_sms, ops);
        if (!forced) {
            // shape class: dtype, attributes, ops, log2 bins, log2 n, auto bounds
            auto lg = [](int64_t v) { int r = 0; while (v > 1) v >>= 1, ++r; return r; };
            klass = std::make_tuple(dtype, n_attrs, ops & (BN_OP_ALL | BN_SUM_MASK), lg(B), lg(n),
                                    grid->auto_bounds ? 1 : 0);
            std::lock_guard<std::mutex> lk(c->tune_mu);
            auto it = c->tuned.find(klass);
            if (it != c->tuned.end()) {
                strat = it->second.strategy;
                // a class spans a factor of two in bins: a mesh larger than the
                // one the class was tuned on may not fit shared memory
                const bool keys = dtype == BN_F64 && !accumulate && n_attrs > 0 && (want_min || want_max);
                if (strat == BN_STRATEGY_PRIVATE && private_smem_bytes(args, c->smem_optin, keys ? 1 : 0) == 0)
                    strat = BN_STRATEGY_GLOBAL;
                if (!aggbits) args.aggregate = it->second.aggregate;
                if (strat == BN_STRATEGY_GLOBAL && it->second.win_nx > 0 &&
                    it->second.win_x0 + it->second.win_nx <= grid->res[0] &&
                    it->second.win_y0 + it->second.win_ny <= grid->res[1] &&
                    window_bytes(it->second.win_nx * it->second.win_ny, n_attrs, sd.do_sum != 0) <=
                        (size_t)(c->smem_optin - 1024)) {
                    args.win_x0 = it->second.win_x0;
                    args.win_y0 = it->second.win_y0;
                    args.win_nx = it->second.win_nx;
                    args.win_ny = it->second.win_ny;
                    strat = BN_STRATEGY_HYBRID;
                }
            } else if (n >= (int64_t)1 << 16 && !accumulate && plan.may_tune) {
                trial = true;
            }
        }
        if (strided && strat == BN_STRATEGY_SORT) strat = BN_STRATEGY_GLOBAL;  // (tuned on contiguous data)
        // a forced window without a tuned placement sits at the mesh centre
        if (strat == BN_STRATEGY_HYBRID && args.win_nx == 0) {
            int wnx = 0, wny = 0;
            if (!window_shape(grid->res[0], grid->res[1], n_attrs, sd.do_sum != 0, c->smem_optin, &wnx, &wny))
                return fail(BN_ERR_INVALID_ARG, "BN_STRATEGY_HYBRID: at most %d attributes", kWindowMaxAttr);
            args.win_x0 = (grid->res[0] - wnx) / 2;
            args.win_y0 = (grid->res[1] - wny) / 2;
            args.win_nx = wnx;
            args.win_ny = wny;
        }
        // min/max as global key records: the global strategy's state, and
        // for f64 the private strategy's exact keys (behind a shared filter);
        // f64 records of three or more attributes get the 32-bit filter
        const bool global_like = strat == BN_STRATEGY_GLOBAL || strat == BN_STRATEGY_HYBRID;
        const bool keys_private = dtype == BN_F64 && (strat == BN_STRATEGY_PRIVATE || trial);
        if ((global_like || keys_private || trial) && !accumulate && n_attrs > 0 &&
            (want_min || want_max)) {
            sd.mmk = plan.alloc((size_t)key_record_pairs(n_attrs, (int)dtype_size(dtype)) * B * 2 *
                                dtype_size(dtype));
            if (!sd.mmk) return cuda_fail(plan.err, "cudaMallocAsync(min/max keys)");
            if ((global_like || trial) && dtype == BN_F64 && n_attrs >= 3) {
                sd.mmf = plan.alloc((size_t)filter_record_pairs(n_attrs) * B * sizeof(int2));
                if (!sd.mmf) return cuda_fail(plan.err, "cudaMallocAsync(min/max filter)");
            }
        }
        // the global strategy's count and sums as one record per bin: one
        // bulk reduction per particle instead of 1 + n_attrs
        if ((strat == BN_STRATEGY_GLOBAL || trial) && !accumulate && sd.do_sum && n_attrs >= 1 &&
            n_attrs <= kRecMaxAttr) {
            sd.rec = static_cast<double*>(plan.alloc((size_t)record_doubles(n_attrs) * B * sizeof(double)));
            if (!sd.rec) return cuda_fail(plan.err, "cudaMallocAsync(count-and-sums records)");
        }
        if (strat == BN_STRATEGY_PRIVATE && private_smem_bytes(args, c->smem_optin) == 0)
            return fail(BN_ERR_INVALID_ARG, "BN_STRATEGY_PRIVATE: the mesh does not fit in shared memory");
        const bool sort_ok = sort_plan(args, c->smem_optin, &sortd);
        sortd.accumulate = accumulate ? 1 : 0;
        if (strat == BN_STRATEGY_SORT && !sort_ok)
            return fail(BN_ERR_INVALID_ARG, "BN_STRATEGY_SORT: the mesh has too many buckets for the sort path");
        if (strat == BN_STRATEGY_SORT || (trial && sort_ok && !strided)) {
            sort_scratch = plan.alloc(sort_scratch_bytes(sortd, args));
            if (!sort_scratch) return cuda_fail(plan.err, "cudaMallocAsync(sort scratch)");
        }
    }
    args.st = sd;
    void* bounds_acc = nullptr;
    if (grid->auto_bounds) {
        bounds_acc = plan.alloc(4 * dtype_size(dtype));
        if (!bounds_acc) return cuda_fail(plan.err, "cudaMallocAsync(bounds)");
    }
    if (!accumulate || bounds_acc) {
        StateDesc init = sd;
        if (accumulate) init.bins = 0;  // keep the state, only reset bounds_acc
        e = launch_init_state(kc, dtype, init, bounds_acc);
        if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    }
    GridDesc* dev_grid = nullptr;
    if (dtype == BN_F64 || grid->auto_bounds || bounds_out) {
        dev_grid = static_cast<GridDesc*>(plan.alloc(sizeof(GridDesc)));
        long long* e0 = nullptr;
        long long* e1 = nullptr;
        if (dtype == BN_F64) {
            e0 = static_cast<long long*>(plan.alloc(sizeof(long long) * (grid->res[0] + 1)));
            e1 = static_cast<long long*>(plan.alloc(sizeof(long long) * (grid->res[1] + 1)));
        }
        if (!dev_grid || (dtype == BN_F64 && (!e0 || !e1))) return cuda_fail(plan.err, "cudaMallocAsync(grid)");
        if (grid->auto_bounds && n > 0) {
            e = launch_bounds_reduce(kc, dtype, args.x, args.y, n, bounds_acc, args.sx, args.sy);
            if (e != cudaSuccess) return cuda_fail(e, "bounds kernel");
        }
        e = launch_grid_setup(kc, dtype, gd, bounds_acc, dev_grid, e0, e1, bounds_out, status_dev);
        if (e != cudaSuccess) return cuda_fail(e, "grid set-up kernel");
        args.dev_grid = dev_grid;
    }
    args.grid = gd;
    if (n > 0 && trial) {
        // Autotuner: run each candidate particle pass on this call's data,
        // timed with CUDA events (the state is re-initialised before each),
        // keep the fastest for the shape class, then do the real pass.
        struct Cand { int strat, agg; };
        std::vector<Cand> cands;
        if (private_smem_bytes(args, c->smem_optin) > 0) cands.push_back({BN_STRATEGY_PRIVATE, 0});
        cands.push_back({BN_STRATEGY_GLOBAL, 0});
        cands.push_back({BN_STRATEGY_GLOBAL, 1});
        if (sort_scratch && sortd.nb >= 8) cands.push_back({BN_STRATEGY_SORT, 0});  // a few buckets: pointless
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        float best = -1.0f;
        Cand win{strat, args.aggregate};
        std::string times;
        StateDesc last_st = sd;  // the state the last trial pass wrote
        if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
            for (const Cand& cd : cands) {
                BinArgs ta = args;
                ta.aggregate = aggbits == BN_AGG_ON ? 1 : aggbits == BN_AGG_OFF ? 0 : cd.agg;
                // the key records serve the global strategy, and f64 private
                // meshes; the filter only the global strategy
                if (cd.strat == BN_STRATEGY_SORT || (cd.strat == BN_STRATEGY_PRIVATE && dtype != BN_F64))
                    ta.st.mmk = nullptr;
                if (cd.strat != BN_STRATEGY_GLOBAL) ta.st.mmf = nullptr;
                if (cd.strat != BN_STRATEGY_GLOBAL) ta.st.rec = nullptr;
                auto pass = [&]() {
                    return cd.strat == BN_STRATEGY_PRIVATE ? launch_bin_private(kc, ta)
                           : cd.strat == BN_STRATEGY_SORT  ? launch_bin_sort(kc, ta, sortd, sort_scratch)
                                                           : launch_bin_global(kc, ta);
                };
                // one untimed pass first: the first launch of a kernel also
                // loads its module, which must not count against it
                last_st = ta.st;
                e = launch_init_state(kc, dtype, ta.st, nullptr);
                if (e == cudaSuccess) e = pass();
                if (e == cudaSuccess) e = launch_init_state(kc, dtype, ta.st, nullptr);
                if (e == cudaSuccess) e = cudaEventRecord(e0, plan.stream);
                if (e == cudaSuccess) e = pass();
                if (e == cudaSuccess) e = cudaEventRecord(e1, plan.stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = -1.0f;
                if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) break;
                char tb[64];
                snprintf(tb, sizeof tb, " %s%s=%.3fms",
                         cd.strat == BN_STRATEGY_PRIVATE ? "private" : cd.strat == BN_STRATEGY_SORT ? "sort" : "global",
                         cd.strat == BN_STRATEGY_GLOBAL ? (ta.aggregate ? "+agg" : "") : "", ms);
                times += tb;
                if (ms >= 0.0f && (best < 0.0f || ms < best)) {
                    best = ms;
                    win = cd;
                }
            }
        }
        // Global strategy with a shared-memory window over the densest bins:
        // the window is placed on the counts the trials just produced (in situ
        // steps keep their distribution from one step to the next) and kept
        // only if it is faster.
        int wbest[4] = {0, 0, 0, 0};
        int wnx = 0, wny = 0;
        if (e == cudaSuccess && win.strat == BN_STRATEGY_GLOBAL && private_smem_bytes(args, c->smem_optin) == 0 &&
            window_shape(grid->res[0], grid->res[1], n_attrs, sd.do_sum != 0, c->smem_optin, &wnx, &wny)) {
            const int rx = grid->res[0], ry = grid->res[1];
            if (wnx >= 8 && wny >= 8 && (int64_t)wnx * wny < B) {
                std::vector<unsigned long long> cnt((size_t)B);
                // counts kept in count-and-sums records reach the count array
                // through the finalise kernel
                if (last_st.rec) e = launch_finalize(kc, last_st, dtype);
                if (e == cudaSuccess) e = cudaStreamSynchronize(plan.stream);
                if (e == cudaSuccess)
                    e = cudaMemcpy(cnt.data(), sd.count, (size_t)B * 8, cudaMemcpyDeviceToHost);
                if (e == cudaSuccess) {
                    // 2D prefix sums, then every window position
                    std::vector<unsigned long long> P((size_t)(rx + 1) * (ry + 1), 0ull);
                    for (int yy = 0; yy < ry; ++yy)
                        for (int xx = 0; xx < rx; ++xx)
                            P[(size_t)(yy + 1) * (rx + 1) + xx + 1] = cnt[(size_t)yy * rx + xx] +
                                P[(size_t)yy * (rx + 1) + xx + 1] + P[(size_t)(yy + 1) * (rx + 1) + xx] -
                                P[(size_t)yy * (rx + 1) + xx];
                    unsigned long long bestc = 0;
                    for (int yy = 0; yy + wny <= ry; ++yy)
                        for (int xx = 0; xx + wnx <= rx; ++xx) {
                            const unsigned long long cw =
                                P[(size_t)(yy + wny) * (rx + 1) + xx + wnx] - P[(size_t)yy * (rx + 1) + xx + wnx] -
                                P[(size_t)(yy + wny) * (rx + 1) + xx] + P[(size_t)yy * (rx + 1) + xx];
                            if (cw > bestc) {
                                bestc = cw;
                                wbest[0] = xx;
                                wbest[1] = yy;
                            }
                        }
                    // worth trying only if the window holds a good share of the particles
                    if (bestc * 8 >= (unsigned long long)n) {
                        wbest[2] = wnx;
                        wbest[3] = wny;
                        BinArgs ta = args;
                        ta.aggregate = aggbits == BN_AGG_ON ? 1 : aggbits == BN_AGG_OFF ? 0 : win.agg;
                        ta.win_x0 = wbest[0];
                        ta.win_y0 = wbest[1];
                        ta.win_nx = wnx;
                        ta.win_ny = wny;
                        ta.st.rec = nullptr;  // the window kernel updates count and sum directly
                        if (e0) cudaEventDestroy(e0);
                        if (e1) cudaEventDestroy(e1);
                        e0 = e1 = nullptr;
                        if (e == cudaSuccess) e = cudaEventCreate(&e0);
                        if (e == cudaSuccess) e = cudaEventCreate(&e1);
                        float ms = -1.0f;
                        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                            e = launch_init_state(kc, dtype, ta.st, nullptr);
                            if (e == cudaSuccess && rep == 1) e = cudaEventRecord(e0, plan.stream);
                            if (e == cudaSuccess) e = launch_bin_global(kc, ta);
                            if (e == cudaSuccess && rep == 1) e = cudaEventRecord(e1, plan.stream);
                        }
                        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
                        {
                            char tb[96];
                            snprintf(tb, sizeof tb, " global+window[%d,%d %dx%d holding %.0f%%]=%.3fms", wbest[0],
                                     wbest[1], wnx, wny, 100.0 * (double)bestc / (double)n, ms);
                            times += tb;
                        }
                        if (e == cudaSuccess && ms >= 0.0f && ms < best) {
                            best = ms;
                            args.win_x0 = wbest[0];
                            args.win_y0 = wbest[1];
                            args.win_nx = wnx;
                            args.win_ny = wny;
                        } else {
                            wbest[2] = wbest[3] = 0;
                        }
                        if (e0) cudaEventDestroy(e0);
                        if (e1) cudaEventDestroy(e1);
                        e0 = e1 = nullptr;
                    }
                }
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (e != cudaSuccess) return cuda_fail(e, "autotuner trial");
        strat = win.strat;
        if (strat == BN_STRATEGY_GLOBAL && wbest[2] > 0) strat = BN_STRATEGY_HYBRID;
        if (!aggbits) args.aggregate = win.agg;
        {
            std::lock_guard<std::mutex> lk(c->tune_mu);
            c->tuned[klass] = bn_context::Tuned{win.strat, win.agg, wbest[0], wbest[1], wbest[2], wbest[3]};
            char head[160];
            snprintf(head, sizeof head, "dtype=%s attrs=%d bins=2^%d n=2^%d:", dtype == BN_F64 ? "f64" : "f32",
                     n_attrs, std::get<3>(klass), std::get<4>(klass));
            char tail[96];
            snprintf(tail, sizeof tail, " -> %s%s%s",
                     win.strat == BN_STRATEGY_PRIVATE ? "private" : win.strat == BN_STRATEGY_SORT ? "sort" : "global",
                     win.strat == BN_STRATEGY_GLOBAL && win.agg ? "+agg" : "", wbest[2] ? "+window" : "");
            c->tune_log.push_back(std::string(head) + times + tail);
        }
        if (strat == BN_STRATEGY_SORT || (strat == BN_STRATEGY_PRIVATE && dtype != BN_F64)) sd.mmk = nullptr;
        if (strat != BN_STRATEGY_GLOBAL && strat != BN_STRATEGY_HYBRID) sd.mmf = nullptr;
        if (strat != BN_STRATEGY_GLOBAL) sd.rec = nullptr;
        args.st = sd;
        e = launch_init_state(kc, dtype, sd, nullptr);
        if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    }
    if (n > 0) {
        plan.strategy = strat;
        cudaEvent_t t0 = nullptr, t1 = nullptr;
        if (c->profile && cudaEventCreate(&t0) == cudaSuccess && cudaEventCreate(&t1) == cudaSuccess)
            cudaEventRecord(t0, plan.stream);
        e = strat == BN_STRATEGY_PRIVATE ? launch_bin_private(kc, args)
            : strat == BN_STRATEGY_SORT  ? launch_bin_sort(kc, args, sortd, sort_scratch)
                                         : launch_bin_global(kc, args);
        if (t1) {
            cudaEventRecord(t1, plan.stream);
            std::lock_guard<std::mutex> lk(c->prof_mu);
            c->prof_pairs.emplace_back(t0, t1);
        }
        if (e != cudaSuccess) return cuda_fail(e, "binning kernel");
    }
    if (want_avg || sd.mmk || sd.rec) {
        e = launch_finalize(kc, sd, dtype);
        if (e != cudaSuccess) return cuda_fail(e, "finalize kernel");
    }
    return BN_OK;
}

bn_status bn::complete_sync(bn_request* r, int sync, bn_request** req) {
    if (sync) {
        cudaError_t e = cudaEventSynchronize(r->done);
        bn_status st = e == cudaSuccess ? request_status_now(r) : cuda_fail(e, "cudaEventSynchronize");
        if (st == BN_NOT_READY) st = BN_OK;
        if (req) {
            *req = r;
        } else {
            bn_request_release(r);
        }
        if (st < 0 && bn_last_error()[0] == '\0') fail(st, "request failed on the device (status %d)", (int)st);
        return st;
    }
    *req = r;
    return BN_OK;
}

// Fused multi-grid pass (bn_bin_multi): every column is staged or taken in
// place once, each spec gets its mesh descriptor, outputs and initial state
// as a bn_bin_particles call would, and one k_bin_multi launch bins them all.
static bn_status enqueue_multi(bn_context* c, Plan& plan, const bn_buffer* cols, int n_cols,
                               const bn_grid_spec* specs, int n_specs, uint32_t ops, bn_result* outs,
                               int* status_dev) {
    const int dtype = cols[0].dtype;
    const int64_t n = cols[0].n;
    if (dtype != BN_F32 && dtype != BN_F64) return fail(BN_ERR_INVALID_ARG, "bn_bin_multi: dtype must be BN_F32 or BN_F64");
    for (int i = 0; i < n_cols; ++i) {
        bn_status st = validate_buffer(c, &cols[i], n, dtype, "column");
        if (st != BN_OK) return st;
    }
    if (ops & BN_OP_ACCUMULATE) return fail(BN_ERR_INVALID_ARG, "bn_bin_multi: BN_OP_ACCUMULATE is not supported");
    if (ops & BN_STRATEGY_MASK) return fail(BN_ERR_INVALID_ARG, "bn_bin_multi: the fused pass takes no strategy");
    if ((ops & BN_AGG_MASK) == BN_AGG_MASK) return fail(BN_ERR_INVALID_ARG, "unknown aggregation mode in ops");
    if ((ops & BN_SUM_MASK) == (3u << 8)) return fail(BN_ERR_INVALID_ARG, "unknown sum mode in ops");
    const bool want_avg = (ops & BN_OP_AVG) != 0;
    const bool want_sum = (ops & BN_OP_SUM) != 0;
    const bool want_min = (ops & BN_OP_MIN) != 0;
    const bool want_max = (ops & BN_OP_MAX) != 0;
    const bool want_count = (ops & BN_OP_COUNT) != 0;
    const bool attr_ops = want_sum || want_avg || want_min || want_max;
    const uint32_t agg = ops & BN_AGG_MASK;
    for (int k = 0; k < n_specs; ++k) {
        const bn_grid_spec& sp = specs[k];
        if (sp.x < 0 || sp.x >= n_cols || sp.y < 0 || sp.y >= n_cols)
            return fail(BN_ERR_INVALID_ARG, "bn_bin_multi: spec %d: coordinate column out of range", k);
        if (sp.n_attrs < 0 || sp.n_attrs > BN_MAX_ATTR)
            return fail(BN_ERR_INVALID_ARG, "bn_bin_multi: spec %d: n_attrs = %d outside [0, %d]", k, sp.n_attrs, BN_MAX_ATTR);
        for (int a = 0; a < sp.n_attrs; ++a)
            if (sp.attrs[a] < 0 || sp.attrs[a] >= n_cols)
                return fail(BN_ERR_INVALID_ARG, "bn_bin_multi: spec %d: attribute column out of range", k);
        if (sp.grid.auto_bounds) return fail(BN_ERR_INVALID_ARG, "bn_bin_multi: spec %d: automatic bounds are not supported", k);
    }
    std::vector<const void*> colp((size_t)n_cols, nullptr);
    for (int i = 0; i < n_cols; ++i) {
        bn_status st = plan.column(&cols[i], dtype, &colp[i]);
        if (st != BN_OK) return st;
    }
    const KernelCtx kc = plan.kc();
    std::vector<MultiSpec> hs((size_t)n_specs);
    for (int k = 0; k < n_specs; ++k) {
        const bn_grid_spec& sp = specs[k];
        MultiSpec& m = hs[k];
        memset(&m, 0, sizeof m);
        GridDesc gd;
        bn_status st = make_grid_desc(&sp.grid, dtype, &gd);
        if (st != BN_OK) return st;
        const int64_t B = (int64_t)sp.grid.res[0] * sp.grid.res[1];
        GridDesc* dg = static_cast<GridDesc*>(plan.alloc(sizeof(GridDesc)));
        long long* e0 = nullptr;
        long long* e1 = nullptr;
        if (dtype == BN_F64) {
            e0 = static_cast<long long*>(plan.alloc(sizeof(long long) * (sp.grid.res[0] + 1)));
            e1 = static_cast<long long*>(plan.alloc(sizeof(long long) * (sp.grid.res[1] + 1)));
        }
        if (!dg || (dtype == BN_F64 && (!e0 || !e1))) return cuda_fail(plan.err, "cudaMallocAsync(grid)");
        cudaError_t e = launch_grid_setup(kc, dtype, gd, nullptr, dg, e0, e1, nullptr, status_dev);
        if (e != cudaSuccess) return cuda_fail(e, "grid setup kernel");
        const int A = attr_ops ? sp.n_attrs : 0;
        m.grid = dg;
        m.x = colp[sp.x];
        m.y = colp[sp.y];
        for (int a = 0; a < A; ++a) m.a[a] = colp[sp.attrs[a]];
        m.n_attrs = A;
        // combining a warp's same-bin lanes (__match_any_sync) only on request:
        // there is no trial here to show it pays
        m.aggregate = agg == BN_AGG_ON ? 1 : 0;
        StateDesc& sd = m.st;
        sd.bins = B;
        sd.n_attrs = A;
        sd.do_sum = (want_sum || want_avg) ? 1 : 0;
        sd.do_min = want_min ? 1 : 0;
        sd.do_max = want_max ? 1 : 0;
        sd.do_avg = want_avg ? 1 : 0;
        bn_result* out = &outs[k];
        void* p = nullptr;
        st = plan.output(&out->count, want_count, B, BN_U64, false, &p);
        if (st != BN_OK) return st;
        sd.count = static_cast<unsigned long long*>(p);
        for (int a = 0; a < A; ++a) {
            if (sd.do_sum) {
                st = plan.output(&out->sum[a], want_sum, B, BN_F64, false, &p);
                if (st != BN_OK) return st;
                sd.sum[a] = static_cast<double*>(p);
            }
            if (want_min) {
                st = plan.output(&out->min[a], true, B, dtype, false, &p);
                if (st != BN_OK) return st;
                sd.mn[a] = p;
            }
            if (want_max) {
                st = plan.output(&out->max[a], true, B, dtype, false, &p);
                if (st != BN_OK) return st;
                sd.mx[a] = p;
            }
            if (want_avg) {
                st = plan.output(&out->avg[a], true, B, BN_F64, false, &p);
                if (st != BN_OK) return st;
                sd.avg[a] = static_cast<double*>(p);
            }
        }
        // min/max as key records (one or two 256-bit loads per particle for
        // all attributes), written to the outputs by the finalise kernel
        if (A > 0 && (want_min || want_max)) {
            sd.mmk = plan.alloc((size_t)key_record_pairs(A, (int)dtype_size(dtype)) * B * 2 *
                                dtype_size(dtype));
            if (!sd.mmk) return cuda_fail(plan.err, "cudaMallocAsync(min/max keys)");
        }
        // count and sums as one record per bin (one bulk reduction per
        // particle and spec), for the counts the kernel is compiled for
        if (sd.do_sum && A >= 1 && A <= kMultiRecMaxAttr) {
            sd.rec = static_cast<double*>(plan.alloc((size_t)record_doubles(A) * B * sizeof(double)));
            if (!sd.rec) return cuda_fail(plan.err, "cudaMallocAsync(count-and-sums records)");
        }
        e = launch_init_state(kc, dtype, sd, nullptr);
        if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    }
    // the descriptors, grouped by attribute count (one launch per group); a
    // pageable source is copied out before the call returns
    std::vector<MultiSpec> sorted(hs);
    std::stable_sort(sorted.begin(), sorted.end(),
                     [](const MultiSpec& a, const MultiSpec& b) { return a.n_attrs < b.n_attrs; });
    std::vector<int> group_attrs, group_size;
    for (const MultiSpec& m : sorted) {
        if (group_attrs.empty() || group_attrs.back() != m.n_attrs) {
            group_attrs.push_back(m.n_attrs);
            group_size.push_back(0);
        }
        ++group_size.back();
    }
    MultiSpec* ds = static_cast<MultiSpec*>(plan.alloc(sizeof(MultiSpec) * (size_t)n_specs));
    if (!ds) return cuda_fail(plan.err, "cudaMallocAsync(specs)");
    cudaError_t e = cudaMemcpyAsync(ds, sorted.data(), sizeof(MultiSpec) * (size_t)n_specs,
                                    cudaMemcpyHostToDevice, plan.stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy specs");
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (c->profile && cudaEventCreate(&t0) == cudaSuccess && cudaEventCreate(&t1) == cudaSuccess)
        cudaEventRecord(t0, plan.stream);
    e = launch_bin_multi(kc, dtype, ds, group_attrs.data(), group_size.data(), (int)group_attrs.size(), n);
    if (t1) {
        cudaEventRecord(t1, plan.stream);
        std::lock_guard<std::mutex> lk(c->prof_mu);
        c->prof_pairs.emplace_back(t0, t1);
    }
    if (e != cudaSuccess) return cuda_fail(e, "fused multi-grid kernel");
    for (int k = 0; k < n_specs; ++k)
        if (want_avg || hs[k].st.mmk || hs[k].st.rec) {
            e = launch_finalize(kc, hs[k].st, dtype);
            if (e != cudaSuccess) return cuda_fail(e, "finalize kernel");
        }
    plan.strategy = BN_STRATEGY_GLOBAL;
    return BN_OK;
}

extern "C" bn_status bn_bin_multi(bn_context* c, const bn_buffer* cols, int n_cols, const bn_grid_spec* specs,
                                  int n_specs, uint32_t ops, bn_result* outs, int sync, bn_request** req) {
    g_err.clear();
    if (!c || !cols || !specs || !outs) return fail(BN_ERR_INVALID_ARG, "bn_bin_multi: NULL argument");
    if (n_cols < 1 || n_cols > BN_MAX_MULTI_COLS)
        return fail(BN_ERR_INVALID_ARG, "bn_bin_multi: n_cols = %d outside [1, %d]", n_cols, BN_MAX_MULTI_COLS);
    if (n_specs < 1 || n_specs > BN_MAX_MULTI_SPECS)
        return fail(BN_ERR_INVALID_ARG, "bn_bin_multi: n_specs = %d outside [1, %d]", n_specs, BN_MAX_MULTI_SPECS);
    if (!sync && !req) return fail(BN_ERR_INVALID_ARG, "bn_bin_multi: asynchronous call needs req");
    if (req) *req = nullptr;
    DeviceGuard g(c->device);
    std::lock_guard<std::mutex> lk(c->enqueue_mu);
    bn_request* r = new_request(c);
    if (!r) return fail(BN_ERR_NO_MEMORY, "bn_bin_multi: no request slot");
    Plan plan(c);
    bn_status st = enqueue_multi(c, plan, cols, n_cols, specs, n_specs, ops, outs, c->status_dev + r->slot);
    if (st == BN_OK) st = plan.finish(r);
    if (st != BN_OK) {
        std::string msg = g_err;
        plan.free_temps();
        cudaEventRecord(r->done, c->stream);
        r->host_status = st;
        bn_request_release(r);
        g_err = msg;
        return st;
    }
    for (int i = 0; i < n_cols; ++i)
        if (cols[i].deleter) r->deleters.push_back({cols[i].deleter, cols[i].ptr, cols[i].deleter_ctx});
    c->last_strategy = BN_STRATEGY_GLOBAL;
    return complete_sync(r, sync, req);
}

extern "C" bn_status bn_bin_particles(bn_context* c, const bn_buffer* x, const bn_buffer* y,
                                      const bn_buffer* attrs, int n_attrs, const bn_grid* grid,
                                      uint32_t ops, bn_result* out, int sync, bn_request** req) {
    g_err.clear();
    if (!c) return fail(BN_ERR_INVALID_ARG, "bn_bin_particles: NULL context");
    if (!sync && !req) return fail(BN_ERR_INVALID_ARG, "bn_bin_particles: asynchronous call needs req");
    if (req) *req = nullptr;
    DeviceGuard g(c->device);
    std::lock_guard<std::mutex> lk(c->enqueue_mu);
    bn_request* r = new_request(c);
    if (!r) return fail(BN_ERR_NO_MEMORY, "bn_bin_particles: no request slot");
    Plan plan(c);
    bn_status st = enqueue_bin(c, plan, x, y, attrs, n_attrs, grid, ops, out, c->status_dev + r->slot);
    if (st == BN_OK) st = plan.finish(r);
    if (st != BN_OK) {
        std::string msg = g_err;
        plan.free_temps();
        cudaEventRecord(r->done, c->stream);
        r->host_status = st;
        bn_request_release(r);
        g_err = msg;
        return st;
    }
    if (x->deleter) r->deleters.push_back({x->deleter, x->ptr, x->deleter_ctx});
    if (y->deleter) r->deleters.push_back({y->deleter, y->ptr, y->deleter_ctx});
    for (int a = 0; a < n_attrs; ++a)
        if (attrs[a].deleter) r->deleters.push_back({attrs[a].deleter, attrs[a].ptr, attrs[a].deleter_ctx});
    if (plan.strategy) c->last_strategy = plan.strategy;
    return complete_sync(r, sync, req);
}

// ------------------------------------------------------------------ merge
extern "C" bn_status bn_merge_results(bn_context* c, const bn_result* parts, int n_parts,
                                      int32_t dtype, int n_attrs, int64_t bins, uint32_t ops,
                                      bn_result* out, int sync, bn_request** req) {
    g_err.clear();
    if (!c || !parts || !out) return fail(BN_ERR_INVALID_ARG, "bn_merge_results: NULL argument");
    if (!sync && !req) return fail(BN_ERR_INVALID_ARG, "bn_merge_results: asynchronous call needs req");
    if (n_parts < 1) return fail(BN_ERR_INVALID_ARG, "bn_merge_results: no parts");
    if (dtype != BN_F32 && dtype != BN_F64) return fail(BN_ERR_INVALID_ARG, "bn_merge_results: bad dtype");
    if (n_attrs < 0 || n_attrs > BN_MAX_ATTR) return fail(BN_ERR_INVALID_ARG, "bn_merge_results: bad n_attrs");
    if (bins < 1 || bins > BN_MAX_BINS) return fail(BN_ERR_INVALID_ARG, "bn_merge_results: bad bins");
    if (req) *req = nullptr;
    DeviceGuard g(c->device);
    std::lock_guard<std::mutex> lk(c->enqueue_mu);
    bn_request* r = new_request(c);
    if (!r) return fail(BN_ERR_NO_MEMORY, "bn_merge_results: no request slot");
    Plan plan(c);
    const bool want_avg = (ops & BN_OP_AVG) != 0;
    bn_status st = BN_OK;
    std::vector<StateDesc> hp((size_t)n_parts);
    for (int p = 0; p < n_parts && st == BN_OK; ++p) {
        StateDesc& s = hp[p];
        memset(&s, 0, sizeof s);
        s.bins = bins;
        s.n_attrs = n_attrs;
        auto dev_in = [&](const bn_buffer& b, int dt, void** outp) -> bn_status {
            if (!b.ptr || b.n < bins || b.dtype != dt || b.device != c->device || b.stride > 1)
                return fail(BN_ERR_INVALID_ARG, "bn_merge_results: part %d needs contiguous device count/sum/min/max of %lld bins", p, (long long)bins);
            bn_status s2 = plan.wait_on(b.stream);
            *outp = b.ptr;
            return s2;
        };
        void* q = nullptr;
        st = dev_in(parts[p].count, BN_U64, &q);
        s.count = static_cast<unsigned long long*>(q);
        for (int a = 0; a < n_attrs && st == BN_OK; ++a) {
            st = dev_in(parts[p].sum[a], BN_F64, &q);
            s.sum[a] = static_cast<double*>(q);
            if (st == BN_OK) st = dev_in(parts[p].min[a], dtype, &s.mn[a]);
            if (st == BN_OK) st = dev_in(parts[p].max[a], dtype, &s.mx[a]);
        }
    }
    StateDesc sd;
    memset(&sd, 0, sizeof sd);
    sd.bins = bins;
    sd.n_attrs = n_attrs;
    sd.do_sum = 1;
    sd.do_min = 1;
    sd.do_max = 1;
    sd.do_avg = want_avg;
    void* q = nullptr;
    if (st == BN_OK) st = plan.output(&out->count, true, bins, BN_U64, false, &q);
    sd.count = static_cast<unsigned long long*>(q);
    for (int a = 0; a < n_attrs && st == BN_OK; ++a) {
        st = plan.output(&out->sum[a], true, bins, BN_F64, false, &q);
        sd.sum[a] = static_cast<double*>(q);
        if (st == BN_OK) st = plan.output(&out->min[a], true, bins, dtype, false, &sd.mn[a]);
        if (st == BN_OK) st = plan.output(&out->max[a], true, bins, dtype, false, &sd.mx[a]);
        if (st == BN_OK && want_avg) {
            st = plan.output(&out->avg[a], true, bins, BN_F64, false, &q);
            sd.avg[a] = static_cast<double*>(q);
        }
    }
    StateDesc* dparts = nullptr;
    if (st == BN_OK) {
        dparts = static_cast<StateDesc*>(plan.alloc(sizeof(StateDesc) * n_parts));
        if (!dparts) st = cuda_fail(plan.err, "cudaMallocAsync(parts)");
    }
    if (st == BN_OK) {
        // pageable source: the copy completes before cudaMemcpyAsync returns
        cudaError_t e = cudaMemcpyAsync(dparts, hp.data(), sizeof(StateDesc) * n_parts,
                                        cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = launch_merge(c->kc(), dtype, sd, dparts, n_parts);
        if (e == cudaSuccess && want_avg) e = launch_finalize(c->kc(), sd, dtype);
        if (e != cudaSuccess) st = cuda_fail(e, "merge kernels");
    }
    if (st == BN_OK) st = plan.finish(r);
    if (st != BN_OK) {
        std::string msg = g_err;
        plan.free_temps();
        cudaEventRecord(r->done, c->stream);
        r->host_status = st;
        bn_request_release(r);
        g_err = msg;
        return st;
    }
    return complete_sync(r, sync, req);
}
