// bn_runtime.h -- host-side objects behind the opaque handles of binning.h.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/binning.h"
#include "bn_internal.cuh"
#include "bn_kernels.h"

struct bn_context {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int smem_optin = 0;
    cudaMemPool_t pool = nullptr;
    std::atomic<uint64_t> launches{0};
    std::mutex enqueue_mu;  // one request is planned and queued at a time
    std::mutex pool_mu;     // event pool and status slots
    std::vector<cudaEvent_t> event_pool;
    std::vector<int> free_slots;
    int* status_host = nullptr;  // mapped pinned: the device writes request errors here
    int* status_dev = nullptr;
    int last_strategy = 0;
    bool profile = false;
    // measured strategy choices of single calls, per shape class
    std::mutex tune_mu;
    struct Tuned {
        int strategy, aggregate;
        int win_x0, win_y0, win_nx, win_ny;  // global strategy's shared-memory window
    };
    std::map<std::tuple<int, int, uint32_t, int, int, int>, Tuned> tuned;
    std::vector<std::string> tune_log;  // one line per tuned class
    std::mutex prof_mu;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pairs;

    bn::KernelCtx kc() { return bn::KernelCtx{stream, num_sms, smem_optin, &launches}; }
    cudaEvent_t get_event();
    void put_event(cudaEvent_t ev);
    int get_slot();
    void put_slot(int s);
};

namespace bn {
struct Deleter {
    void (*fn)(void*, void*);
    void* ptr;
    void* ctx;
};
}  // namespace bn

struct bn_request {
    bn_context* ctx = nullptr;
    cudaEvent_t done = nullptr;
    int slot = -1;
    bn_status host_status = BN_OK;  // error found before launch
    std::vector<bn::Deleter> deleters;
    // Server requests complete on the server's streams; the server thread
    // publishes BN_NOT_READY / final status here.
    std::atomic<int>* external_done = nullptr;
    void (*on_release)(bn_request*) = nullptr;
    void* owner = nullptr;
};

namespace bn {

bn_status fail(bn_status st, const char* fmt, ...);
bn_status cuda_fail(cudaError_t e, const char* what);

// Makes `dev` the calling thread's current device for its scope.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Everything one request queues: stream ordering, staged inputs,
// temporaries (freed stream-ordered once the kernels are queued) and
// device-to-host copies of host outputs.
struct Plan {
    struct Copy {
        void* host;
        void* dev;
        size_t bytes;
    };
    bn_context* ctx;
    cudaStream_t stream;  // where this plan's work is queued
    std::vector<void*> temps;
    std::vector<void*> waited;
    std::vector<void*> out_streams;
    std::vector<Copy> d2h;
    struct PeerCopy {  // an output on another device: temporary -> peer at finish
        void* peer;
        int device;
        void* stream;
        void* dev;
        size_t bytes;
    };
    std::vector<PeerCopy> peer_out;
    cudaError_t err = cudaSuccess;
    size_t h2d_bytes = 0, d2h_bytes = 0, p2p_bytes = 0;
    size_t temp_bytes = 0;  // bytes of every temporary alloc() handed out
    int strategy = 0;
    // false: an unseen shape class takes the heuristic strategy instead of
    // timing the candidates (the trials synchronise with the device; a
    // latency-bound caller such as the server must not wait on them)
    bool may_tune = true;

    explicit Plan(bn_context* c) : ctx(c), stream(c->stream) {}
    Plan(bn_context* c, cudaStream_t s) : ctx(c), stream(s) {}
    KernelCtx kc() const { return KernelCtx{stream, ctx->num_sms, ctx->smem_optin, &ctx->launches}; }
    void* alloc(size_t bytes);
    void free_temps();
    bn_status wait_on(void* stream);
    bn_status wait_on_peer(void* stream, int device);
    bn_status column(const bn_buffer* b, int dtype, const void** out, int64_t* stride_out = nullptr);
    bn_status output(bn_buffer* b, bool wanted, int64_t bins, int dtype, bool load, void** out);
    bn_status finish(bn_request* r);
};

bn_request* new_request(bn_context* c);
void run_deleters(bn_request* r);
bn_status validate_buffer(const bn_context* c, const bn_buffer* b, int64_t n, int dtype,
                          const char* what);
bn_status make_grid_desc(const bn_grid* g, int dtype, GridDesc* out);
int choose_strategy(const BinArgs& a, int smem_optin, int num_sms, uint32_t ops);
bn_status enqueue_bin(bn_context* c, Plan& plan, const bn_buffer* x, const bn_buffer* y,
                      const bn_buffer* attrs, int n_attrs, const bn_grid* grid, uint32_t ops,
                      bn_result* out, int* status_dev);
bn_status complete_sync(bn_request* r, int sync, bn_request** req);
size_t request_temp_bytes(const bn_context* c, const bn_block& b, int dtype, uint32_t ops);
void batch_cache_release(bn_context* c);

}  // namespace bn
