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
                                 int64_t n, void* bounds_acc, int64_t sx = 1, int64_t sy = 1);
cudaError_t launch_grid_setup(const KernelCtx& kc, int dtype, const GridDesc& host_desc,
                              const void* bounds_acc, GridDesc* dev_desc, long long* edges0,
                              long long* edges1, double* bounds_out, int* status);
cudaError_t launch_finalize(const KernelCtx& kc, const StateDesc& st, int dtype);
cudaError_t launch_merge(const KernelCtx& kc, int dtype, const StateDesc& out,
                         const StateDesc* dev_parts, int n_parts);
cudaError_t launch_gather(const KernelCtx& kc, int dtype, void* dst, const void* src, int64_t n,
                          int64_t stride);
double host_fast_delta(double lo, double hi, double s, int res);

// Hot loop: one pass over the particles into the per-bin state.
struct BinArgs {
    int dtype;              // BN_F32 / BN_F64
    int n_attrs;
    int sum_mode;           // SumMode (f32 data)
    int aggregate;          // global strategy: combine same-bin lanes of a warp first
    // global strategy: a window of bins whose count and sums each CTA keeps
    // in shared memory (win_nx == 0: none); bins [win_x0, win_x0 + win_nx) x
    // [win_y0, win_y0 + win_ny) (k_window.cu)
    int win_x0, win_y0, win_nx, win_ny;
    const void* x;
    const void* y;
    const void* a[kMaxAttr];
    // element strides of x, y and the attributes (0 or 1: contiguous). The
    // private, global and window kernels read strided columns in place with
    // scalar loads (a warp's loads of consecutive records cover contiguous
    // memory); the other kernels take contiguous columns only.
    int64_t sx, sy, sa[kMaxAttr];
    int64_t n;
    GridDesc grid;          // by value (explicit bounds) ...
    const GridDesc* dev_grid;  // ... or read on the device (automatic bounds; null otherwise)
    StateDesc st;
};

// Plan of the bucketed sort + reduce (k_sort.cu). Sizes are set by
// sort_plan; the device pointers by launch_bin_sort from one scratch block.
// Record positions are 32-bit: the plan requires n < 2^31 - 2^16.
struct SortDesc {
    int log2bk;        // bins per bucket = 1 << log2bk
    int nb;            // buckets
    int tp;            // particles per pass-1 tile
    int per;           // particles per pass-1 thread (tp / per threads)
    int chunk;         // records per pass-2 work item (at most)
    int accumulate;    // 1: items merge into the existing state (never store a whole bucket)
    int64_t tiles;     // pass-1 tiles
    int64_t slots;     // record slots (= n; attribute column stride)
    int64_t max_items;
    int off_gpos, off_skey, off_sbk, off_sattr;  // pass-1 shared-memory layout
    size_t smem_count, smem_scatter, smem_reduce;
    unsigned short* keys;    // [slots] bin within the bucket, bucket-contiguous
    void* attrs;             // [n_attrs][slots] attribute values, same order
    unsigned* bucket_total;  // [nb] records per bucket
    unsigned* cursor;        // [nb] next free record slot of each bucket
    int4* items;             // [max_items] {bucket, first record, end record, sole}
    int* counters;           // [0] items, [1] next item to take
};

bool sort_plan(const BinArgs& a, int smem_optin, SortDesc* sd);
size_t sort_scratch_bytes(const SortDesc& sd, const BinArgs& a);
// dargs (may be null): a device copy of `a` the kernels read instead of their
// by-value arguments (a, sd still give the launch shape and the scratch).
cudaError_t launch_bin_sort(const KernelCtx& kc, const BinArgs& a, SortDesc sd, void* scratch,
                            const BinArgs* dargs = nullptr);

// One block of a batch as the persistent kernel sees it (k_batch.cu).
struct BatchBlock {
    const void* x;
    const void* y;
    const void* a[kMaxAttr];
    int64_t n;
    int64_t tile;      // particles per work item
    GridDesc g;        // explicit bounds; edges point into the batch scratch (f64)
    StateDesc st;      // the block's outputs
    int strategy;      // BN_STRATEGY_PRIVATE or BN_STRATEGY_GLOBAL
    int aggregate;
    // private blocks whose mesh exceeds shared memory: the mesh is cut into
    // `bands` bands of `band_rows` mesh rows (the last may be shorter), and
    // every band of every tile is a work item of its own (bands <= 1: whole)
    int bands;
    int band_rows;
};

cudaError_t launch_batch_prepare(const KernelCtx& kc, int dtype, BatchBlock* dev_blocks,
                                 const int64_t* dev_bin_start, const int64_t* dev_edge_start,
                                 int nblk, int64_t total_bins, int64_t total_edges);
cudaError_t launch_batch_bin(const KernelCtx& kc, int dtype, int sum_mode, const BatchBlock* blocks,
                             const int4* items, int n_items, int* counter, int n_attrs, size_t smem);
cudaError_t launch_batch_finalize(const KernelCtx& kc, const BatchBlock* dev_blocks,
                                  const int64_t* dev_bin_start, int nblk, int64_t total_bins);
size_t private_mesh_bytes(int dtype, int sum_mode, int64_t bins, int n_attrs, bool s, bool lo, bool hi);

// One binning of a fused multi-grid pass (k_multi.cu), in device memory.
struct MultiSpec {
    const GridDesc* grid;  // device descriptor (f64: with its edge keys)
    const void* x;
    const void* y;
    const void* a[kMaxAttr];
    int32_t n_attrs;
    int32_t aggregate;
    StateDesc st;
};

// Particles per tile of the fused pass: every spec of a tile is binned
// before the next tile, while the tile's columns are still in L1/L2.
constexpr int kMultiTile = 2048;
// Attribute counts the fused pass is compiled for (larger counts take the
// generic kernel, which updates count and sums with separate reductions).
constexpr int kMultiRecMaxAttr = 10;
// dev_specs holds n_groups runs of specs; run g has group_size[g] specs of
// group_attrs[g] attributes each and gets one launch (the kernel is compiled
// per attribute count so that its per-particle arrays stay in registers).
cudaError_t launch_bin_multi(const KernelCtx& kc, int dtype, const MultiSpec* dev_specs,
                             const int* group_attrs, const int* group_size, int n_groups, int64_t n);

// Shared-memory bytes the privatised kernel needs for this mesh, or 0 if
// the mesh does not fit.
// Shared memory of the private strategy's mesh, 0 when it does not fit.
// keys: -1 as a.st says; 0 / 1: f64 min/max without / with global key records.
size_t private_smem_bytes(const BinArgs& a, int smem_optin, int keys = -1);
cudaError_t launch_bin_private(const KernelCtx& kc, const BinArgs& a);
// Global strategy; with a window (a.win_nx > 0) it runs launch_bin_window.
cudaError_t launch_bin_global(const KernelCtx& kc, const BinArgs& a);

// Global strategy with a shared-memory window of win_nx x win_ny bins whose
// counts and sums (96-bit fixed point) each CTA keeps privately (k_window.cu).
constexpr int kWindowMaxAttr = 4;
cudaError_t launch_bin_window(const KernelCtx& kc, const BinArgs& a);
// Shared-memory bytes of a window of `cells` bins.
size_t window_bytes(int cells, int n_attrs, bool do_sum);

// Raise a kernel's dynamic shared-memory limit to the device's opt-in
// maximum (less its static shared memory), once per kernel and device;
// safe to call from several threads.
cudaError_t raise_smem_limit(const void* kernel, int smem_optin);

}  // namespace bn
