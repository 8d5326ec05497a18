// batch.cu -- bn_bin_batch: many independent blocks in one request (the 90
// binning operations per in situ step of Sec. 4.3).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "bn_runtime.h"

using namespace bn;

extern "C" bn_status bn_bin_batch(bn_context* c, const bn_block* blocks, int n_blocks,
                                  uint32_t ops, int sync, bn_request** req) {
    if (!c) return fail(BN_ERR_INVALID_ARG, "bn_bin_batch: NULL context");
    if (!sync && !req) return fail(BN_ERR_INVALID_ARG, "bn_bin_batch: asynchronous call needs req");
    if (n_blocks < 0 || (n_blocks > 0 && !blocks)) return fail(BN_ERR_INVALID_ARG, "bn_bin_batch: bad blocks");
    if (req) *req = nullptr;
    for (int k = 0; k < n_blocks; ++k)
        if (!blocks[k].out) return fail(BN_ERR_INVALID_ARG, "bn_bin_batch: block %d has no outputs", k);
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != c->device) cudaSetDevice(c->device);
    std::lock_guard<std::mutex> lk(c->enqueue_mu);
    bn_request* r = new_request(c);
    if (!r) return fail(BN_ERR_NO_MEMORY, "bn_bin_batch: no request slot");
    Plan plan(c);
    bn_status st = BN_OK;
    for (int k = 0; k < n_blocks && st == BN_OK; ++k) {
        const bn_block& b = blocks[k];
        st = enqueue_bin(c, plan, &b.x, &b.y, b.attrs, b.n_attrs, &b.grid, ops, b.out,
                         c->status_dev + r->slot);
    }
    if (st == BN_OK) st = plan.finish(r);
    if (st != BN_OK) {
        std::string msg = bn_last_error();
        plan.free_temps();
        cudaEventRecord(r->done, c->stream);
        r->host_status = st;
        bn_request_release(r);
        if (cur >= 0 && cur != c->device) cudaSetDevice(cur);
        return fail(st, "%s", msg.c_str());
    }
    for (int k = 0; k < n_blocks; ++k) {
        const bn_block& b = blocks[k];
        if (b.x.deleter) r->deleters.push_back({b.x.deleter, b.x.ptr, b.x.deleter_ctx});
        if (b.y.deleter) r->deleters.push_back({b.y.deleter, b.y.ptr, b.y.deleter_ctx});
        for (int a = 0; a < b.n_attrs; ++a)
            if (b.attrs[a].deleter)
                r->deleters.push_back({b.attrs[a].deleter, b.attrs[a].ptr, b.attrs[a].deleter_ctx});
    }
    st = complete_sync(r, sync, req);
    if (cur >= 0 && cur != c->device) cudaSetDevice(cur);
    return st;
}
