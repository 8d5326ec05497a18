// static_entry.cu -- bn_bin_particles_static: binning that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they want to bin:
// a simulation that has handed the whole GPU to its own memory pool, code
// running inside a section where any cudaMalloc would synchronise the device
// or fail, or a host that must keep its memory use fixed after start-up. For
// them this entry point takes every input and output from the caller and
// keeps the only scratch it needs (mesh descriptor, automatic-bounds
// accumulator, a status word and the f64 bin-edge keys) in one fixed array
// that lives in this file. It calls no cudaMalloc, cudaFree, cudaHostAlloc or
// allocating library routine, creates no stream or event, and uses no
// bn_context.
//
// The array is kStaticScratchBytes (64 KiB) per GPU that loads the library
// and stays allocated until the process exits. Every call shares it and it
// keeps the last call's contents; each call rewrites or clears every part it
// reads. Calls whose work overlaps on the GPU (different streams, or several
// host threads) race on the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "bn_runtime.h"

using namespace bn;

namespace {

constexpr size_t kStaticScratchBytes = 64 * 1024;
constexpr size_t kOffDesc = 0;       // GridDesc (<= 256 bytes)
constexpr size_t kOffBounds = 256;   // 4 values of the coordinate type
constexpr size_t kOffStatus = 512;   // one int
constexpr size_t kOffEdges = 1024;   // f64 edge keys, res_x + 1 then res_y + 1
constexpr size_t kMaxEdgeKeys = (kStaticScratchBytes - kOffEdges) / sizeof(long long);
static_assert(sizeof(GridDesc) <= kOffBounds - kOffDesc, "mesh descriptor overruns its scratch slot");
static_assert(4 * sizeof(double) <= kOffStatus - kOffBounds, "bounds accumulator overruns its scratch slot");
static_assert(kOffStatus + sizeof(int) <= kOffEdges, "status word overruns its scratch slot");
static_assert(kOffDesc % alignof(GridDesc) == 0 && kOffEdges % alignof(long long) == 0, "misaligned slot");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the array on the current device; looked up once per
// device (host code only sees a stand-in for the symbol, not the address).
bn_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(BN_ERR_INVALID_ARG, "bn_bin_particles_static: device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "bn_bin_particles_static: cudaGetSymbolAddress");
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return BN_OK;
}

bn_status check_dev_buffer(const bn_buffer& b, int dev, int64_t min_n, int dtype, const char* what) {
    if (!b.ptr) return fail(BN_ERR_INVALID_ARG, "bn_bin_particles_static: %s missing (outputs must be caller-allocated)", what);
    if (b.device != dev) return fail(BN_ERR_DEVICE_MISMATCH, "bn_bin_particles_static: %s must be device memory of device %d", what, dev);
    if (b.stride > 1) return fail(BN_ERR_INVALID_ARG, "bn_bin_particles_static: %s must be contiguous", what);
    if (b.dtype != dtype) return fail(BN_ERR_INVALID_ARG, "bn_bin_particles_static: %s has dtype %d, expected %d", what, b.dtype, dtype);
    if (b.n < min_n) return fail(BN_ERR_INVALID_ARG, "bn_bin_particles_static: %s holds %lld elements, needs %lld", what, (long long)b.n, (long long)min_n);
    const size_t es = dtype == BN_F32 ? 4 : 8;
    if ((uintptr_t)b.ptr % es) return fail(BN_ERR_INVALID_ARG, "bn_bin_particles_static: %s misaligned", what);
    return BN_OK;
}

}  // namespace

extern "C" bn_status bn_bin_particles_static(const bn_buffer* x, const bn_buffer* y,
                                             const bn_buffer* attrs, int n_attrs,
                                             const bn_grid* grid, uint32_t ops,
                                             const bn_result* out, void* stream, int sync) {
    if (!x || !y || !grid || !out) return fail(BN_ERR_INVALID_ARG, "bn_bin_particles_static: NULL argument");
    if (n_attrs < 0 || n_attrs > BN_MAX_ATTR || (n_attrs > 0 && !attrs))
        return fail(BN_ERR_INVALID_ARG, "bn_bin_particles_static: bad attributes");
    if (ops & (BN_OP_ACCUMULATE | BN_STRATEGY_MASK))
        return fail(BN_ERR_INVALID_ARG, "bn_bin_particles_static: accumulate and strategy flags are not supported");
    const int dtype = x->dtype;
    if (dtype != BN_F32 && dtype != BN_F64) return fail(BN_ERR_INVALID_ARG, "bn_bin_particles_static: bad dtype");
    const int64_t n = x->n;
    if (n < 0) return fail(BN_ERR_INVALID_ARG, "bn_bin_particles_static: negative length");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "bn_bin_particles_static: cudaGetDevice");
    GridDesc gd;
    bn_status st = make_grid_desc(grid, dtype, &gd);
    if (st != BN_OK) return st;
    const int64_t edge_keys = (int64_t)grid->res[0] + grid->res[1] + 2;
    if (dtype == BN_F64 && edge_keys > (int64_t)kMaxEdgeKeys)
        return fail(BN_ERR_INVALID_ARG,
                    "bn_bin_particles_static: f64 mesh needs %lld edge keys, the fixed scratch holds %zu "
                    "(res_x + res_y <= %zu); use bn_bin_particles for larger meshes",
                    (long long)edge_keys, kMaxEdgeKeys, kMaxEdgeKeys - 2);
    if (n > 0) {
        const bn_buffer* cols[2 + BN_MAX_ATTR] = {x, y};
        for (int a = 0; a < n_attrs; ++a) cols[2 + a] = &attrs[a];
        for (int k = 0; k < 2 + n_attrs; ++k) {
            if (cols[k]->n != n) return fail(BN_ERR_INVALID_ARG, "bn_bin_particles_static: column lengths differ");
            st = check_dev_buffer(*cols[k], dev, n, dtype, k == 0 ? "x" : k == 1 ? "y" : "attribute");
            if (st != BN_OK) return st;
        }
    }
    const int64_t B = (int64_t)grid->res[0] * grid->res[1];
    const bool want_sum = ops & BN_OP_SUM, want_avg = ops & BN_OP_AVG;
    const bool want_min = ops & BN_OP_MIN, want_max = ops & BN_OP_MAX;
    // count is the state every other reduction needs, and avg needs sums:
    // both must come from the caller since nothing is allocated here
    st = check_dev_buffer(out->count, dev, B, BN_U64, "count output");
    if (st != BN_OK) return st;
    StateDesc sd;
    memset(&sd, 0, sizeof sd);
    sd.bins = B;
    sd.n_attrs = n_attrs;
    sd.do_sum = (want_sum || want_avg) ? 1 : 0;
    sd.do_min = want_min;
    sd.do_max = want_max;
    sd.do_avg = want_avg;
    sd.count = static_cast<unsigned long long*>(out->count.ptr);
    for (int a = 0; a < n_attrs; ++a) {
        if (sd.do_sum) {
            st = check_dev_buffer(out->sum[a], dev, B, BN_F64, "sum output");
            if (st != BN_OK) return st;
            sd.sum[a] = static_cast<double*>(out->sum[a].ptr);
        }
        if (want_min) {
            st = check_dev_buffer(out->min[a], dev, B, dtype, "min output");
            if (st != BN_OK) return st;
            sd.mn[a] = out->min[a].ptr;
        }
        if (want_max) {
            st = check_dev_buffer(out->max[a], dev, B, dtype, "max output");
            if (st != BN_OK) return st;
            sd.mx[a] = out->max[a].ptr;
        }
        if (want_avg) {
            st = check_dev_buffer(out->avg[a], dev, B, BN_F64, "avg output");
            if (st != BN_OK) return st;
            sd.avg[a] = static_cast<double*>(out->avg[a].ptr);
        }
    }
    double* bounds_out = nullptr;
    if (out->bounds.ptr) {
        st = check_dev_buffer(out->bounds, dev, 4, BN_F64, "bounds output");
        if (st != BN_OK) return st;
        bounds_out = static_cast<double*>(out->bounds.ptr);
    }

    unsigned char* base = nullptr;
    st = scratch_address(dev, &base);
    if (st != BN_OK) return st;
    GridDesc* dev_grid = reinterpret_cast<GridDesc*>(base + kOffDesc);
    void* bounds_acc = grid->auto_bounds ? static_cast<void*>(base + kOffBounds) : nullptr;
    int* status = reinterpret_cast<int*>(base + kOffStatus);
    long long* e0 = reinterpret_cast<long long*>(base + kOffEdges);
    long long* e1 = e0 + (grid->res[0] + 1);

    int sms = 0, optin = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_fail(e, "bn_bin_particles_static: device attributes");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const KernelCtx kc{s, sms, optin, nullptr};

    BinArgs args;
    memset(&args, 0, sizeof args);
    args.dtype = dtype;
    args.n_attrs = n_attrs;
    const uint32_t sum_bits = ops & BN_SUM_MASK;
    args.sum_mode = dtype == BN_F64 ? kSumF64 : sum_bits == BN_SUM_F32 ? kSumF32
                                              : sum_bits == BN_SUM_F64 ? kSumF64 : kSumF32C;
    args.aggregate = B <= 65536 ? 1 : 0;
    args.x = x->ptr;
    args.y = y->ptr;
    for (int a = 0; a < n_attrs; ++a) args.a[a] = attrs[a].ptr;
    args.n = n;
    args.st = sd;
    args.grid = gd;
    // The kernels read the descriptor from the scratch array only when the
    // device computes it (automatic bounds, f64 edge keys) or publishes the
    // bounds; f32 data with explicit bounds passes it by value, as
    // bn_bin_particles does.
    const bool dev_setup = dtype == BN_F64 || grid->auto_bounds || bounds_out;
    args.dev_grid = dev_setup ? dev_grid : nullptr;

    // the status word keeps the previous call's value: clear it first
    e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_init_state(kc, dtype, sd, bounds_acc);
    if (e == cudaSuccess && grid->auto_bounds && n > 0)
        e = launch_bounds_reduce(kc, dtype, args.x, args.y, n, bounds_acc);
    if (e == cudaSuccess && dev_setup)
        e = launch_grid_setup(kc, dtype, gd, bounds_acc, dev_grid, dtype == BN_F64 ? e0 : nullptr,
                              dtype == BN_F64 ? e1 : nullptr, bounds_out, status);
    if (e == cudaSuccess && n > 0) {
        // the sort path needs a large scratch area, so this entry point
        // chooses only between the shared-memory and the global-atomic paths
        int strat = choose_strategy(args, optin, sms, ops);
        e = strat == BN_STRATEGY_PRIVATE ? launch_bin_private(kc, args) : launch_bin_global(kc, args);
    }
    if (e == cudaSuccess && want_avg) e = launch_finalize(kc, sd, dtype);
    if (e != cudaSuccess) return cuda_fail(e, "bn_bin_particles_static: launch");
    if (!sync) return BN_OK;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "bn_bin_particles_static: cudaStreamSynchronize");
    int dst = 0;
    e = cudaMemcpy(&dst, status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "bn_bin_particles_static: read status");
    if (dst != BN_OK) return fail((bn_status)dst, "bn_bin_particles_static: automatic bounds collapsed");
    return BN_OK;
}
