// server.cu -- the asynchronous in situ method of Sec. 3 as a continuous-
// batching server.
//
// Sec. 3/4.3: with asynchronous execution the in situ code deep-copies the
// data it needs, hands the work to a thread and returns to the simulation at
// once; simulation and analysis then run concurrently. Here:
//   submit   deep-copies the block's columns (device data: a device copy if
//            the memory budget has room now, otherwise a copy into the
//            page-locked staging arena the server allocated at creation;
//            host data: a staging-arena copy), makes each input's owning
//            stream wait for the copy (so the caller may overwrite its
//            buffers with any later work on that stream), queues the
//            request and returns a handle;
//   worker   admits queued requests while their device memory (input copy +
//            state temporaries) fits the budget, groups admitted requests
//            into one batch per launch slot and queues the batch on one of
//            max_inflight low-priority streams -- requests that arrive while
//            other batches run are admitted as memory and slots free up, and
//            their kernels overlap on the device with the running batches
//            and with the caller's own work (the producer);
//   complete when a batch's event fires, each request's memory returns to
//            the budget and its status is published.
// Every request is binned exactly as bn_bin_particles would bin it alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "bn_runtime.h"

using namespace bn;

namespace {

using Clock = std::chrono::steady_clock;

double us_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::micro>(b - a).count();
}

// Page-locked host memory allocated once, handed out first-fit in 256-byte
// units: submit never has to page-lock memory on the request path.
struct Arena {
    char* base = nullptr;
    size_t size = 0;
    std::mutex mu;
    std::map<size_t, size_t> free_;  // offset -> bytes, adjacent runs merged

    static size_t round(size_t n) { return (std::max(n, (size_t)1) + 255) & ~(size_t)255; }
    bool alloc(size_t n, size_t* off) {
        n = round(n);
        std::lock_guard<std::mutex> lk(mu);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, o2 = it->first + n;
            free_.erase(it);
            if (rest) free_[o2] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = round(n);
        std::lock_guard<std::mutex> lk(mu);
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Job {
    bn_request* req = nullptr;
    std::atomic<int> status{BN_NOT_READY};
    bn_block block;           // columns rewritten to point at the copies
    bn_result out;            // the caller's outputs (copied handle set)
    uint32_t ops = 0;
    int dtype = 0;
    int64_t n = 0;
    size_t col_bytes = 0;     // bytes of one column copy
    size_t need = 0;          // device bytes charged to the budget
    bool on_device = false;   // inputs already copied to device memory
    void* dev_copy = nullptr; // device copy of all columns (one allocation)
    void* host_copy = nullptr;// page-locked staging (when not on device)
    int staged = 0;           // 0 device copy, 1 staging arena, 2 own page-locked allocation
    size_t arena_off = 0;
    size_t copy_bytes = 0;
    cudaEvent_t copied = nullptr;
    // timing record (bn_request_timing)
    Clock::time_point t_submit0, t_submit1, t_admit, t_launch, t_done;
    double batch_gpu_us = 0.0;
    int batch_size = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t start = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<Job*> jobs;
    bool busy = false;
};

}  // namespace

struct bn_server {
    bn_context* ctx = nullptr;
    size_t budget = 0;
    int max_batch = 64;
    std::vector<Slot> slots;
    cudaStream_t copy_stream = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job*> queue;  // submitted, waiting for admission
    bool stop = false;
    size_t in_use = 0, peak = 0;
    Arena arena;
    std::atomic<uint64_t> submitted{0}, admitted{0}, completed{0}, failed{0}, launches{0};
    std::atomic<uint64_t> staged{0}, staging_overflow{0}, overdrawn{0};
};

static void job_release_hook(bn_request* r) {
    Job* j = static_cast<Job*>(r->owner);
    if (!j) return;
    if (j->host_copy && j->staged == 2) cudaFreeHost(j->host_copy);
    if (j->copied) r->ctx->put_event(j->copied);
    delete j;
}

static void finish_job(bn_server* s, Job* j, int st) {
    j->t_done = Clock::now();
    // the batch is complete, so its host-to-device copy is too: the staging
    // space can take the next request (a job that failed before launch may
    // still have its copy queued)
    if (j->host_copy && j->staged == 1) {
        if (st < 0) cudaStreamSynchronize(s->copy_stream);
        s->arena.release(j->arena_off, j->copy_bytes);
        j->host_copy = nullptr;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->in_use -= j->need;
    }
    if (st < 0) s->failed++;
    s->completed++;
    j->status.store(st, std::memory_order_release);
    s->cv.notify_all();
}

// Queue one batch on a free slot. Called by the worker with s->mu unlocked.
static void launch_batch(bn_server* s, Slot& slot, std::vector<Job*>& batch) {
    bn_context* c = s->ctx;
    std::lock_guard<std::mutex> lk(c->enqueue_mu);
    Plan plan(c, slot.stream);
    plan.may_tune = false;  // shape classes the context has tuned keep their choice
    cudaEventRecord(slot.start, slot.stream);
    for (Job* j : batch) {
        if (j->copied) cudaStreamWaitEvent(slot.stream, j->copied, 0);
        const size_t before = plan.temp_bytes;
        bn_status st = enqueue_bin(c, plan, &j->block.x, &j->block.y, j->block.attrs,
                                   j->block.n_attrs, &j->block.grid, j->ops, &j->out,
                                   c->status_dev + j->req->slot);
        if (plan.temp_bytes - before > j->need - j->copy_bytes) s->overdrawn++;
        if (st != BN_OK) {
            j->req->host_status = st;
            j->status.store(st, std::memory_order_release);
        }
    }
    // the staged columns are no longer needed once the kernels are queued
    for (Job* j : batch)
        if (j->dev_copy) {
            cudaFreeAsync(j->dev_copy, slot.stream);
            j->dev_copy = nullptr;
        }
    for (auto& cp : plan.d2h)
        cudaMemcpyAsync(cp.host, cp.dev, cp.bytes, cudaMemcpyDeviceToHost, slot.stream);
    plan.d2h.clear();
    plan.free_temps();
    cudaEventRecord(slot.done, slot.stream);
    for (void* os : plan.out_streams)
        if (static_cast<cudaStream_t>(os) != slot.stream)
            cudaStreamWaitEvent(static_cast<cudaStream_t>(os), slot.done, 0);
    s->launches++;
    const Clock::time_point now = Clock::now();
    for (Job* j : batch) {
        j->t_launch = now;
        j->batch_size = (int)batch.size();
    }
    slot.jobs = batch;
    slot.busy = true;
}

static void worker_main(bn_server* s) {
    cudaSetDevice(s->ctx->device);
    for (;;) {
        // 1. retire finished batches
        for (Slot& sl : s->slots) {
            if (!sl.busy) continue;
            cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaErrorNotReady) continue;
            float gpu_ms = 0.0f;
            if (e == cudaSuccess && cudaEventElapsedTime(&gpu_ms, sl.start, sl.done) != cudaSuccess) gpu_ms = 0.0f;
            for (Job* j : sl.jobs) {
                j->batch_gpu_us = 1e3 * (double)gpu_ms;
                int st = j->status.load(std::memory_order_acquire);
                if (st == BN_NOT_READY) {
                    st = e == cudaSuccess ? s->ctx->status_host[j->req->slot] : BN_ERR_CUDA;
                }
                finish_job(s, j, st);
            }
            sl.jobs.clear();
            sl.busy = false;
        }
        // 2. admit and launch
        std::vector<Job*> batch;
        Slot* free_slot = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (Slot& sl : s->slots)
                if (!sl.busy) { free_slot = &sl; break; }
            bool any_busy = false;
            for (Slot& sl : s->slots) any_busy = any_busy || sl.busy;
            if (s->stop && s->queue.empty() && !any_busy) return;
            if (free_slot) {
                while (!s->queue.empty() && (int)batch.size() < s->max_batch) {
                    Job* j = s->queue.front();
                    // device-resident copies were charged at submit
                    if (!j->on_device && s->in_use + j->need > s->budget) break;
                    if (!j->on_device) {
                        s->in_use += j->need;
                        s->peak = std::max(s->peak, s->in_use);
                    }
                    s->queue.pop_front();
                    batch.push_back(j);
                }
            }
            if (batch.empty()) {
                // nothing to launch now: sleep briefly unless work is running
                s->cv.wait_for(lk, std::chrono::microseconds(any_busy ? 20 : 200));
                continue;
            }
        }
        // move pinned-staged inputs to the device
        const Clock::time_point t_admit = Clock::now();
        for (Job* j : batch) {
            s->admitted++;
            j->t_admit = t_admit;
            if (j->on_device) continue;
            void* d = nullptr;
            size_t bytes = j->col_bytes * (2 + j->block.n_attrs);
            cudaError_t e = cudaMallocAsync(&d, bytes ? bytes : 16, s->copy_stream);
            if (e == cudaSuccess && bytes)
                e = cudaMemcpyAsync(d, j->host_copy, bytes, cudaMemcpyHostToDevice, s->copy_stream);
            if (e == cudaSuccess) e = cudaEventRecord(j->copied, s->copy_stream);
            if (e != cudaSuccess) {
                j->req->host_status = BN_ERR_CUDA;
                j->status.store(BN_ERR_CUDA, std::memory_order_release);
                continue;
            }
            j->dev_copy = d;
            char* p = static_cast<char*>(d);
            j->block.x.ptr = p;
            j->block.y.ptr = p + j->col_bytes;
            for (int a = 0; a < j->block.n_attrs; ++a) j->block.attrs[a].ptr = p + (2 + a) * j->col_bytes;
            j->block.x.device = j->block.y.device = s->ctx->device;
            for (int a = 0; a < j->block.n_attrs; ++a) j->block.attrs[a].device = s->ctx->device;
        }
        std::vector<Job*> runnable;
        for (Job* j : batch) {
            if (j->status.load() != BN_NOT_READY) finish_job(s, j, j->status.load());
            else runnable.push_back(j);
        }
        if (!runnable.empty()) launch_batch(s, *free_slot, runnable);
    }
}

extern "C" bn_status bn_server_create(bn_context* c, const bn_server_options* opt, bn_server** out) {
    if (!c || !out) return fail(BN_ERR_INVALID_ARG, "bn_server_create: NULL argument");
    *out = nullptr;
    auto* s = new (std::nothrow) bn_server();
    if (!s) return fail(BN_ERR_NO_MEMORY, "bn_server_create: out of host memory");
    s->ctx = c;
    s->budget = (opt && opt->budget_bytes) ? opt->budget_bytes : ((size_t)40 << 30);
    int inflight = (opt && opt->max_inflight > 0) ? opt->max_inflight : 4;
    s->max_batch = (opt && opt->max_batch > 0) ? opt->max_batch : 64;
    int lo = 0, hi = 0;
    cudaSetDevice(c->device);
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    int prio = (opt && opt->stream_priority) ? opt->stream_priority : lo;  // lo = least urgent
    s->slots.resize((size_t)inflight);
    cudaError_t e = cudaStreamCreateWithPriority(&s->copy_stream, cudaStreamNonBlocking, prio);
    for (Slot& sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, prio);
        if (e == cudaSuccess) e = cudaEventCreate(&sl.start);  // timed: batch_gpu_us
        if (e == cudaSuccess) e = cudaEventCreate(&sl.done);
    }
    // the staging arena: page-locked once, here, not per request
    size_t staging = (opt && opt->staging_bytes) ? opt->staging_bytes
                                                 : std::min(s->budget / 4, (size_t)4 << 30);
    staging = (staging + 255) & ~(size_t)255;
    if (e == cudaSuccess && staging) {
        void* base = nullptr;
        e = cudaHostAlloc(&base, staging, cudaHostAllocDefault);
        if (e == cudaSuccess) {
            s->arena.base = static_cast<char*>(base);
            s->arena.size = staging;
            s->arena.free_[0] = staging;
        }
    }
    if (e != cudaSuccess) {
        for (Slot& sl : s->slots) {
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.start) cudaEventDestroy(sl.start);
            if (sl.done) cudaEventDestroy(sl.done);
        }
        if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
        if (s->arena.base) cudaFreeHost(s->arena.base);
        delete s;
        return cuda_fail(e, "bn_server_create");
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return BN_OK;
}

extern "C" bn_status bn_server_submit(bn_server* s, const bn_block* b, uint32_t ops, bn_request** req) {
    const Clock::time_point t0 = Clock::now();
    if (!s || !b || !req) return fail(BN_ERR_INVALID_ARG, "bn_server_submit: NULL argument");
    *req = nullptr;
    bn_context* c = s->ctx;
    if (!b->out) return fail(BN_ERR_INVALID_ARG, "bn_server_submit: block has no outputs");
    const int dtype = b->x.dtype;
    if (dtype != BN_F32 && dtype != BN_F64) return fail(BN_ERR_INVALID_ARG, "bn_server_submit: bad dtype");
    if (b->n_attrs < 0 || b->n_attrs > BN_MAX_ATTR) return fail(BN_ERR_INVALID_ARG, "bn_server_submit: bad n_attrs");
    const int64_t n = b->x.n;
    bn_status st = validate_buffer(c, &b->x, n, dtype, "x");
    if (st == BN_OK) st = validate_buffer(c, &b->y, n, dtype, "y");
    for (int a = 0; a < b->n_attrs && st == BN_OK; ++a) st = validate_buffer(c, &b->attrs[a], n, dtype, "attr");
    if (st != BN_OK) return st;
    // the deep copy orders itself after the columns' own streams on this
    // device: columns and outputs on other devices go through bn_bin_particles
    auto peer = [&](const bn_buffer& q) { return q.ptr && q.device != BN_HOST && q.device != c->device; };
    bool any_peer = peer(b->x) || peer(b->y) || (b->out && peer(b->out->count));
    for (int a = 0; a < b->n_attrs; ++a)
        any_peer = any_peer || peer(b->attrs[a]) ||
                   (b->out && (peer(b->out->sum[a]) || peer(b->out->min[a]) || peer(b->out->max[a]) ||
                               peer(b->out->avg[a])));
    if (any_peer)
        return fail(BN_ERR_DEVICE_MISMATCH, "bn_server_submit: buffers on another device are not served");
    GridDesc gd;
    st = make_grid_desc(&b->grid, dtype, &gd);
    if (st != BN_OK) return st;
    // outputs must be caller-allocated: the library cannot hand back
    // allocations from the worker thread
    const bool want_avg = ops & BN_OP_AVG, want_sum = ops & BN_OP_SUM;
    if ((ops & BN_OP_COUNT) && !b->out->count.ptr)
        return fail(BN_ERR_INVALID_ARG, "bn_server_submit: outputs must be caller-allocated");
    for (int a = 0; a < b->n_attrs; ++a) {
        if ((want_sum && !b->out->sum[a].ptr) || ((ops & BN_OP_MIN) && !b->out->min[a].ptr) ||
            ((ops & BN_OP_MAX) && !b->out->max[a].ptr) || (want_avg && !b->out->avg[a].ptr))
            return fail(BN_ERR_INVALID_ARG, "bn_server_submit: outputs must be caller-allocated");
    }
    if (ops & BN_OP_ACCUMULATE) return fail(BN_ERR_INVALID_ARG, "bn_server_submit: accumulate is not served");

    const size_t es = dtype == BN_F32 ? 4 : 8;
    auto* j = new (std::nothrow) Job();
    if (!j) return fail(BN_ERR_NO_MEMORY, "bn_server_submit: out of host memory");
    j->block = *b;
    j->out = *b->out;
    j->block.out = &j->out;
    j->ops = ops & ~(uint32_t)BN_OP_ACCUMULATE;
    j->dtype = dtype;
    j->n = n;
    j->t_submit0 = t0;
    j->col_bytes = ((size_t)n * es + 255) & ~(size_t)255;
    const size_t copy_bytes = j->col_bytes * (2 + b->n_attrs);
    j->copy_bytes = copy_bytes;
    j->need = copy_bytes + request_temp_bytes(c, *b, dtype, j->ops);
    if (j->need > s->budget) {
        delete j;
        return fail(BN_ERR_BUDGET, "bn_server_submit: request needs %zu bytes, budget is %zu", j->need, s->budget);
    }
    bn_request* r = new_request(c);
    if (!r) {
        delete j;
        return fail(BN_ERR_NO_MEMORY, "bn_server_submit: no request slot");
    }
    j->req = r;
    r->external_done = &j->status;
    r->owner = j;
    r->on_release = job_release_hook;
    j->copied = c->get_event();

    // The deep copy (Sec. 4.3 asynchronous method): into device memory when
    // the budget has room now, else into pinned host memory.
    bool all_dev = b->x.device != BN_HOST && b->y.device != BN_HOST;
    for (int a = 0; a < b->n_attrs; ++a) all_dev = all_dev && b->attrs[a].device != BN_HOST;
    bool charged = false;
    if (all_dev) {
        // a device copy whenever the budget has room, even behind a queue:
        // staging through host memory while a backlog drains would slow
        // every later request and feed the backlog
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->in_use + j->need <= s->budget) {
            s->in_use += j->need;
            s->peak = std::max(s->peak, s->in_use);
            charged = true;
        }
    }
    const bn_buffer* cols[2 + BN_MAX_ATTR];
    cols[0] = &b->x;
    cols[1] = &b->y;
    for (int a = 0; a < b->n_attrs; ++a) cols[2 + a] = &b->attrs[a];
    const int ncol = 2 + b->n_attrs;
    cudaError_t e = cudaSuccess;
    std::lock_guard<std::mutex> enq(c->enqueue_mu);  // copy stream ordering vs. other submits
    // order the copy stream after every owning stream
    for (int k = 0; k < ncol && e == cudaSuccess; ++k) {
        if (cols[k]->device == BN_HOST) continue;
        cudaEvent_t ev = c->get_event();
        e = cudaEventRecord(ev, static_cast<cudaStream_t>(cols[k]->stream));
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->copy_stream, ev, 0);
        c->put_event(ev);
    }
    void* dst = nullptr;
    if (e == cudaSuccess) {
        if (charged) {
            e = cudaMallocAsync(&dst, copy_bytes ? copy_bytes : 16, s->copy_stream);
        } else if (s->arena.base && s->arena.alloc(copy_bytes, &j->arena_off)) {
            // earlier copies into the same arena range were consumed by
            // batches that completed before the range was released
            dst = s->arena.base + j->arena_off;
            j->staged = 1;
            s->staged++;
        } else {
            // the arena is full or too small: page-lock memory for this one
            e = cudaHostAlloc(&dst, copy_bytes ? copy_bytes : 16, cudaHostAllocDefault);
            j->staged = 2;
            s->staging_overflow++;
        }
    }
    for (int k = 0; k < ncol && e == cudaSuccess && n > 0; ++k) {
        const bn_buffer* col = cols[k];
        char* d = static_cast<char*>(dst) + (size_t)k * j->col_bytes;
        const size_t pitch = (col->stride <= 1 ? 1 : (size_t)col->stride) * es;
        const cudaMemcpyKind kind = col->device == BN_HOST
                                        ? (charged ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost)
                                        : (charged ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
        if (col->device == BN_HOST && !charged) {
            // host to pinned host: a plain CPU copy, done before returning
            if (pitch == es) memcpy(d, col->ptr, (size_t)n * es);
            else for (int64_t i = 0; i < n; ++i) memcpy(d + i * es, static_cast<const char*>(col->ptr) + i * pitch, es);
        } else if (pitch == es) {
            e = cudaMemcpyAsync(d, col->ptr, (size_t)n * es, kind, s->copy_stream);
        } else {
            e = cudaMemcpy2DAsync(d, es, col->ptr, pitch, es, (size_t)n, kind, s->copy_stream);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(j->copied, s->copy_stream);
    // later work on each input's owning stream is ordered after the copy
    for (int k = 0; k < ncol && e == cudaSuccess; ++k)
        if (cols[k]->device != BN_HOST)
            e = cudaStreamWaitEvent(static_cast<cudaStream_t>(cols[k]->stream), j->copied, 0);
    if (e != cudaSuccess) {
        if (charged) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->in_use -= j->need;
        }
        if (dst && !charged) {
            cudaStreamSynchronize(s->copy_stream);  // copies already queued from it
            if (j->staged == 1) s->arena.release(j->arena_off, copy_bytes);
            else cudaFreeHost(dst);
        }
        j->staged = 0;
        j->status.store(BN_ERR_CUDA);
        r->host_status = BN_ERR_CUDA;
        bn_status out = cuda_fail(e, "bn_server_submit: deep copy");
        bn_request_release(r);
        return out;
    }
    if (charged) {
        j->on_device = true;
        j->dev_copy = dst;
    } else {
        j->host_copy = dst;
    }
    if (charged) {
        char* p = static_cast<char*>(dst);
        j->block.x.ptr = p;
        j->block.y.ptr = p + j->col_bytes;
        for (int a = 0; a < b->n_attrs; ++a) j->block.attrs[a].ptr = p + (2 + a) * j->col_bytes;
        j->block.x.device = j->block.y.device = c->device;
        for (int a = 0; a < b->n_attrs; ++a) j->block.attrs[a].device = c->device;
    }
    j->block.x.stride = j->block.y.stride = 1;
    j->block.x.stream = j->block.y.stream = nullptr;
    j->block.x.deleter = j->block.y.deleter = nullptr;
    for (int a = 0; a < b->n_attrs; ++a) {
        j->block.attrs[a].stride = 1;
        j->block.attrs[a].stream = nullptr;
        j->block.attrs[a].deleter = nullptr;
    }
    // copies are ordered by the `copied` event; the legacy stream (nullptr)
    // must not be waited on by the worker, so point the columns at the copy
    // stream, which the worker's slot stream waits on through `copied`
    j->block.x.stream = j->block.y.stream = s->copy_stream;
    for (int a = 0; a < b->n_attrs; ++a) j->block.attrs[a].stream = s->copy_stream;
    j->t_submit1 = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->queue.push_back(j);
    }
    s->submitted++;
    s->cv.notify_all();
    *req = r;
    return BN_OK;
}

extern "C" bn_status bn_server_stats_get(bn_server* s, bn_server_stats* out) {
    if (!s || !out) return fail(BN_ERR_INVALID_ARG, "bn_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted.load();
    out->admitted = s->admitted.load();
    out->completed = s->completed.load();
    out->failed = s->failed.load();
    out->launches = s->launches.load();
    out->bytes_in_use = s->in_use;
    out->peak_bytes = s->peak;
    out->staged = s->staged.load();
    out->staging_overflow = s->staging_overflow.load();
    out->overdrawn = s->overdrawn.load();
    return BN_OK;
}

extern "C" bn_status bn_server_request_timing(bn_request* r, bn_request_timing* out) {
    if (!r || !out || r->on_release != job_release_hook || !r->owner)
        return fail(BN_ERR_INVALID_ARG, "bn_server_request_timing: not a server request");
    const Job* j = static_cast<const Job*>(r->owner);
    if (j->status.load(std::memory_order_acquire) == BN_NOT_READY) return BN_NOT_READY;
    memset(out, 0, sizeof *out);
    out->submit_us = us_between(j->t_submit0, j->t_submit1);
    out->queue_us = us_between(j->t_submit1, j->t_admit);
    out->launch_us = j->batch_size ? us_between(j->t_admit, j->t_launch) : 0.0;
    out->complete_us = j->batch_size ? us_between(j->t_launch, j->t_done) : 0.0;
    out->batch_gpu_us = j->batch_gpu_us;
    out->batch_size = j->batch_size;
    out->staged = j->staged;
    return BN_OK;
}

extern "C" bn_status bn_server_destroy(bn_server* s) {
    if (!s) return BN_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->ctx->device);
    for (Slot& sl : s->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.start);
        cudaEventDestroy(sl.done);
    }
    cudaStreamSynchronize(s->copy_stream);
    cudaStreamDestroy(s->copy_stream);
    // every request has finished, so no arena range is in use any more
    if (s->arena.base) cudaFreeHost(s->arena.base);
    delete s;
    return BN_OK;
}
