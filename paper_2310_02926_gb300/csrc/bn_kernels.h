// bn_kernels.h -- host-side launchers of the binning kernels. Each returns
// the launch's cudaError_t; all work is queued on KernelCtx::stream.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "bn_internal.cuh"

namespace bn {

struct KernelCtx {
    cudaStream_t stream;
    int num_sms;
    int smem_optin;                       // max dynamic shared memory per block
    std::atomic<uint64_t>* launches;      // launch counter (may be null)
    void count_launch(uint64_t k = 1) const {
        if (launches) launches->fetch_add(k, std::memory_order_relaxed);
    }
};

// Strategy-independent kernels (k_common.cu).
cudaError_t launch_init_state(const KernelCtx& kc, int dtype, const StateDesc& st,
                              void* bounds_acc);
cudaError_t launch_bounds_reduce(const KernelCtx& kc, int dtype, const void* x, const void* y,
                                 int64_t n, void* bounds_acc);
cudaError_t launch_grid_setup(const KernelCtx& kc, int dtype, const GridDesc& host_desc,
                              const void* bounds_acc, GridDesc* dev_desc, long long* edges0,
                              long long* edges1, double* bounds_out, int* status);
cudaError_t launch_finalize(const KernelCtx& kc, const StateDesc& st);
cudaError_t launch_merge(const KernelCtx& kc, int dtype, const StateDesc& out,
                         const StateDesc* dev_parts, int n_parts);
cudaError_t launch_gather(const KernelCtx& kc, int dtype, void* dst, const void* src, int64_t n,
                          int64_t stride);
int host_fast_ok(double lo, double hi, double s, int res);

// Hot loop: one pass over the particles into the per-bin state.
struct BinArgs {
    int dtype;              // BN_F32 / BN_F64
    int n_attrs;
    int sum_mode;           // SumMode (f32 data)
    const void* x;
    const void* y;
    const void* a[kMaxAttr];
    int64_t n;
    GridDesc grid;          // by value (explicit bounds) ...
    const GridDesc* dev_grid;  // ... or read on the device (automatic bounds; null otherwise)
    StateDesc st;
};

// Shared-memory bytes the privatised kernel needs for this mesh, or 0 if
// the mesh does not fit.
size_t private_smem_bytes(const BinArgs& a, int smem_optin);
cudaError_t launch_bin_private(const KernelCtx& kc, const BinArgs& a);
cudaError_t launch_bin_global(const KernelCtx& kc, const BinArgs& a);

}  // namespace bn
