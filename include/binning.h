/*
 * binning.h -- C ABI of libbinning.so: particle data binning on one GB300.
 *
 * The operation (Sec. 4.2, "In Situ Data Binning"): two columns of a
 * particle table are the axes of a uniform 2D mesh; each particle's pair of
 * coordinates selects one mesh cell (bin); a per-bin counter gives a
 * histogram and the other columns are reduced per bin by sum, minimum,
 * maximum and average. Mesh bounds are given by the caller or taken as the
 * minimum and maximum of the coordinate columns.
 *
 * Data hand-off follows the data-model extensions of Sec. 2: a buffer handle
 * carries a pointer, length, element type, the device it lives on, an owning
 * stream and the allocator that made it, and may carry a deleter that ties
 * the memory's life to the handle (zero-copy construction with coordinated
 * life cycle, Listing 1). Work is ordered after each input's owning stream;
 * in asynchronous mode a call returns at once and a request handle is
 * queried or waited on, in synchronous mode the call returns after the work
 * completes (stream modes of Sec. 2).
 *
 * Conventions for every entry point:
 *  - Every call returns a bn_status; nothing throws across the ABI. A
 *    negative status is an error and bn_last_error() returns a message for
 *    the calling thread.
 *  - Pointers to structs are borrowed for the duration of the call only.
 *  - A "device buffer" is memory that the context's device can read with
 *    ordinary loads: cudaMalloc/cudaMallocAsync/torch CUDA memory on that
 *    device. A buffer with device == BN_HOST is host memory (pageable or
 *    pinned), reached by the location-agnostic access of Sec. 2 ("PM
 *    Interoperability and Location Agnostic Access"): a contiguous input
 *    column in page-locked (pinned or registered) host memory is read in
 *    place by the kernels over the host link; other host inputs, and host
 *    outputs, go through a device temporary.
 *  - A buffer on a different CUDA device of this process is reached the
 *    same way (location-agnostic access, Sec. 2: GetCUDAAccessible moves
 *    another device's data to the one doing the work): an input column is
 *    copied peer to peer into a temporary of the context's device after the
 *    work queued on its owning stream (on its own device); an output is
 *    written to a temporary and copied to its device when the request
 *    completes, and later work on its owning stream waits for that copy.
 *    The server (bn_server_submit) takes host buffers and buffers of the
 *    context's device only. A device ordinal this process does not have is
 *    rejected with BN_ERR_DEVICE_MISMATCH.
 *
 * Bin layout of every per-bin output: row-major [res_y][res_x], bin
 * b = iy * res_x + ix. Per-attribute outputs are separate buffers.
 *
 * Numerical contract (readings where the paper is silent):
 *  - the bin index is computed in the coordinate's own type T:
 *    lo_T = (T)lo, hi_T = (T)hi, s_T = (T)res / (hi_T - lo_T),
 *    t = (x - lo_T) * s_T, i = min(trunc(t), res - 1), every operation
 *    IEEE round-to-nearest in T and never fused;
 *  - explicit bounds are the half-open [lo, hi); automatic bounds are the
 *    minimum and maximum over the finite coordinates and are closed;
 *  - particles outside the mesh, or with a NaN coordinate, are dropped;
 *  - count is u64; sum and avg are f64; min and max are in T;
 *  - min/max order is IEEE totalOrder (-0 < +0) and skips NaN attributes;
 *    NaN attributes propagate into sum and avg;
 *  - empty bins: count 0, sum +0.0, min +inf, max -inf, avg quiet NaN
 *    (0x7ff8000000000000).
 *  - counts, min and max are exact; sums differ from the exactly rounded
 *    sum only by accumulation order: FP64 accumulation (f64 data, and f32
 *    data in BN_SUM_F64 mode) within a few units of 2^-53 times the
 *    number of terms times the sum of |a|; f32 modes see BN_SUM_*.
 */
#ifndef BINNING_H
#define BINNING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define BN_API __attribute__((visibility("default")))
#else
#define BN_API
#endif

#define BN_MAX_ATTR 16
#define BN_MAX_RES 65536
#define BN_MAX_BINS (1 << 30)
#define BN_HOST (-1)
#define BN_MAX_MULTI_COLS 64  /* columns of one bn_bin_multi call */
#define BN_MAX_MULTI_SPECS 256 /* binnings of one bn_bin_multi call */

typedef enum bn_status {
    BN_OK = 0,
    BN_NOT_READY = 1,            /* bn_query: the request is still running */
    BN_ERR_INVALID_ARG = -1,     /* bad dtype, length mismatch, res out of range, lo >= hi, ... */
    BN_ERR_DEVICE_MISMATCH = -2, /* a buffer's device cannot be used for this call */
    BN_ERR_NO_MEMORY = -3,       /* a device or host allocation failed */
    BN_ERR_BUDGET = -4,          /* a server request can never fit the memory budget */
    BN_ERR_TIMEOUT = -5,         /* bn_wait gave up; the request is still running */
    BN_ERR_CUDA = -6,            /* a CUDA runtime call failed */
    BN_ERR_DEGENERATE = -7,      /* automatic bounds collapsed (no finite coordinate, or min == max) */
    BN_ERR_INTERNAL = -8
} bn_status;

typedef enum bn_dtype { BN_F32 = 1, BN_F64 = 2, BN_U64 = 3 } bn_dtype;

/* Who made a buffer's memory (Sec. 2, svtkAllocator). Informational except
 * for BN_ALLOC_CUDA_ASYNC buffers that the library allocated itself. */
typedef enum bn_allocator {
    BN_ALLOC_EXTERNAL = 0,   /* caller-managed, any allocator */
    BN_ALLOC_TORCH = 1,      /* PyTorch caching allocator */
    BN_ALLOC_CUDA_ASYNC = 2, /* cudaMallocAsync (the library's own outputs) */
    BN_ALLOC_HOST = 3,       /* malloc/new host memory */
    BN_ALLOC_PINNED = 4      /* cudaHostAlloc page-locked host memory */
} bn_allocator;

/*
 * A zero-copy view of one column (Sec. 2, "Zero-copy Data Transfer").
 *   ptr      first element (device pointer, or host pointer if device == BN_HOST)
 *   n        number of elements
 *   stride   elements between consecutive values; 0 or 1 = contiguous
 *   dtype    bn_dtype of the elements
 *   device   CUDA ordinal, or BN_HOST
 *   stream   owning cudaStream_t (NULL = legacy default stream); reads are
 *            ordered after work already queued on it, and outputs become
 *            visible on it when the request completes
 *   alloc    bn_allocator that made the memory
 *   deleter  NULL = borrowed. Otherwise the library calls
 *            deleter(ptr, deleter_ctx) once, when the request that received
 *            the handle is released (inputs) or when bn_buffer_release is
 *            called (outputs): the shared_ptr deleter of Listing 1.
 */
typedef struct bn_buffer {
    void* ptr;
    int64_t n;
    int64_t stride;
    int32_t dtype;
    int32_t device;
    void* stream;
    int32_t alloc;
    int32_t reserved;
    void (*deleter)(void* ptr, void* ctx);
    void* deleter_ctx;
} bn_buffer;

/* The mesh (Sec. 4.2): lo/hi per axis (ignored when auto_bounds != 0) and
 * the number of bins per axis, 1 <= res <= BN_MAX_RES, res_x * res_y <=
 * BN_MAX_BINS. Axis 0 is x, axis 1 is y. */
typedef struct bn_grid {
    double lo[2];
    double hi[2];
    int32_t res[2];
    int32_t auto_bounds;
    int32_t reserved;
} bn_grid;

/* ops: which reductions to produce (Sec. 4.2: count, sum, min, max, average). */
enum {
    BN_OP_COUNT = 1u << 0,
    BN_OP_SUM = 1u << 1,
    BN_OP_MIN = 1u << 2,
    BN_OP_MAX = 1u << 3,
    BN_OP_AVG = 1u << 4,
    BN_OP_ALL = 0x1fu,
    /* Accumulate: the output buffers already hold a result of the same mesh
     * (count, sum, min, max, all present); the new particles are merged into
     * it and avg is recomputed. Successive steps or shards bin into one
     * state this way. */
    BN_OP_ACCUMULATE = 1u << 5,

    /* Sum mode for f32 data (bits 8-9). f64 data always sums in FP64.
     *   BN_SUM_F32C (default): per-CTA FP32 partial sums with a two-sum
     *     compensation term, widened to FP64 only where partials merge;
     *     error about 2^-44 sum|a| per bin plus the FP64 merge.
     *   BN_SUM_F32: plain FP32 per-CTA partials, FP64 merge; error grows
     *     with the number of terms a CTA adds into one bin (about
     *     n_cta_bin * 2^-24 sum|a| at worst).
     *   BN_SUM_F64: every value widened and added in FP64. */
    BN_SUM_F32C = 0u << 8,
    BN_SUM_F32 = 1u << 8,
    BN_SUM_F64 = 2u << 8,
    BN_SUM_MASK = 3u << 8,

    /* Accumulation strategy (bits 12-15); AUTO lets the library choose. */
    BN_STRATEGY_AUTO = 0u << 12,
    BN_STRATEGY_PRIVATE = 1u << 12, /* per-CTA shared-memory copy of the mesh */
    BN_STRATEGY_GLOBAL = 2u << 12,  /* atomics into the global mesh (count and sums of a
                                      * particle as one bulk reduction of the bin's record,
                                      * for 1-4 attributes; warp aggregation optional) */
    BN_STRATEGY_SORT = 3u << 12,    /* tile sort by bin + segmented reduce */
    /* Global atomics with a shared-memory window: every CTA keeps the counts
     * and sums of a rectangle of the densest bins in shared memory (sums as
     * exact fixed-point integers) and merges them at the end; the rest of the
     * mesh takes global atomics. The autotuner places the window on the
     * counts of its trial pass; forced without a tuned placement, the window
     * sits at the mesh centre. At most 4 attributes. */
    BN_STRATEGY_HYBRID = 4u << 12,
    BN_STRATEGY_MASK = 15u << 12,

    /* Warp aggregation in the global-atomic strategy (bits 16-17): lanes of a
     * warp that hit the same bin combine before their atomics. It pays off
     * for clustered data and costs a warp-wide match per step otherwise. */
    BN_AGG_AUTO = 0u << 16,
    BN_AGG_ON = 1u << 16,
    BN_AGG_OFF = 2u << 16,
    BN_AGG_MASK = 3u << 16
};

/*
 * Outputs. Each requested buffer is either caller-allocated (ptr != NULL:
 * a device buffer of the context's device, or a host buffer, contiguous,
 * n >= bins, dtype as below) or left zeroed (ptr == NULL), in which case the
 * library allocates device memory with cudaMallocAsync on the execution
 * stream, fills in the handle (alloc = BN_ALLOC_CUDA_ASYNC, with a deleter),
 * and the caller frees it with bn_buffer_release.
 *   count          u64 [bins]                     (BN_OP_COUNT)
 *   sum[a], avg[a] f64 [bins]                     (BN_OP_SUM, BN_OP_AVG)
 *   min[a], max[a] T   [bins], T the data's dtype (BN_OP_MIN, BN_OP_MAX)
 *   bounds         f64 [4] = lo_x, hi_x, lo_y, hi_y actually used, in T
 *                  widened to f64 (optional; ptr NULL = not wanted); all
 *                  four are quiet NaN when automatic bounds collapsed
 *                  (BN_ERR_DEGENERATE), so a caller that does not read the
 *                  request's status can still tell a failed call
 * Buffers for ops not requested are ignored.
 */
typedef struct bn_result {
    bn_buffer count;
    bn_buffer sum[BN_MAX_ATTR];
    bn_buffer min[BN_MAX_ATTR];
    bn_buffer max[BN_MAX_ATTR];
    bn_buffer avg[BN_MAX_ATTR];
    bn_buffer bounds;
} bn_result;

/* One independent binning problem inside a batch or a server request. */
typedef struct bn_block {
    bn_buffer x;
    bn_buffer y;
    bn_buffer attrs[BN_MAX_ATTR];
    int32_t n_attrs;
    int32_t reserved;
    bn_grid grid;
    bn_result* out;
} bn_block;

/* One binning of a fused multi-grid pass (bn_bin_multi): the columns that
 * are its coordinates and attributes (indices into the call's columns) and
 * its mesh (explicit bounds). */
typedef struct bn_grid_spec {
    int32_t x, y;
    int32_t n_attrs;
    int32_t attrs[BN_MAX_ATTR];
    int32_t reserved;
    bn_grid grid;
} bn_grid_spec;

/* bn_options.flags */
enum {
    /* Record a timing event pair around every hot-loop kernel launch (the
     * particle pass) on the stream it runs on; read with bn_context_profile. */
    BN_CTX_PROFILE = 1
};

typedef struct bn_options {
    void* stream;            /* execute on this cudaStream_t; NULL = the context
                                creates its own non-blocking stream */
    int32_t stream_priority; /* for a context-created stream (0 = default) */
    int32_t flags;           /* BN_CTX_* */
    size_t mempool_release_threshold; /* bytes the stream-ordered pool may keep
                                         cached (0 = keep everything) */
} bn_options;

typedef struct bn_context bn_context;
typedef struct bn_request bn_request;
typedef struct bn_server bn_server;

/* ----------------------------------------------------------------- context */

/* Bind a context to CUDA device `device` (Sec. 2: memory is allocated on the
 * active device; Sec. 3: the in situ code runs on an assigned device).
 * opt may be NULL. Errors: BN_ERR_INVALID_ARG (no such device),
 * BN_ERR_CUDA, BN_ERR_NO_MEMORY. */
BN_API bn_status bn_context_create(int device, const bn_options* opt, bn_context** ctx);

/* Waits for all work of the context, then frees it. NULL is a no-op. */
BN_API bn_status bn_context_destroy(bn_context* ctx);

/* The cudaStream_t the context executes on (for timing with events). */
BN_API bn_status bn_context_stream(bn_context* ctx, void** stream);

/* The autotuner's record: one line per tuned shape class with the measured
 * time of each candidate particle pass and the choice, written into buf
 * (NUL-terminated, truncated to cap bytes). */
BN_API bn_status bn_context_autotune_report(bn_context* ctx, char* buf, size_t cap);

/* Number of kernel launches the context has issued so far. */
BN_API bn_status bn_context_launch_count(bn_context* ctx, uint64_t* launches);

/* With BN_CTX_PROFILE: waits for the recorded hot-loop launches, returns
 * their total device time in milliseconds and their number, and forgets
 * them. Without the flag both are 0. last_strategy (may be NULL) receives
 * the BN_STRATEGY_* value of the most recent particle pass. */
BN_API bn_status bn_context_profile(bn_context* ctx, double* total_ms, uint64_t* launches,
                                    int32_t* last_strategy);

/* ----------------------------------------------------------------- binning */

/*
 * Bin n particles (Sec. 4.2) with coordinates x, y and n_attrs attribute
 * columns onto `grid`, producing the reductions selected in `ops`.
 *   x, y, attrs[0..n_attrs)  same n and dtype (BN_F32 or BN_F64); device
 *                            buffers and contiguous page-locked host
 *                            buffers are read in place (zero copy), other
 *                            host buffers are staged to the device
 *   n_attrs                  0..BN_MAX_ATTR (0: count only); when `ops`
 *                            selects no sum, avg, min or max the columns are
 *                            validated but neither staged nor read
 *   out                      see bn_result; must not be NULL
 *   sync                     1: return after completion (status of the work);
 *                            0: return at once, the work runs asynchronously
 *   req                      receives a request handle when sync == 0 (must
 *                            then be non-NULL); may be NULL when sync == 1
 * Ownership: inputs are borrowed until the request completes (the caller
 * must neither free nor overwrite them before), deleters of input handles
 * run when the request is released. Errors found before launch are returned
 * directly; errors found on the device (BN_ERR_DEGENERATE) are returned by
 * bn_query / bn_wait / a synchronous call. Empty input (n == 0) is valid.
 */
BN_API bn_status bn_bin_particles(bn_context* ctx, const bn_buffer* x, const bn_buffer* y,
                           const bn_buffer* attrs, int n_attrs, const bn_grid* grid,
                           uint32_t ops, bn_result* out, int sync, bn_request** req);

/*
 * bn_bin_particles without any allocation (the paper has no counterpart:
 * this is for callers that cannot allocate). A simulation that has given all
 * device memory to its own pool, code that must not call cudaMalloc (it can
 * synchronise the device or fail at that point), or a process that must keep
 * its memory footprint fixed after start-up can still bin with this call:
 * it allocates no device or host memory, creates no stream or event and needs
 * no bn_context. Its only scratch (mesh descriptor, automatic-bounds
 * accumulator, a status word, the f64 bin-edge keys) is one fixed 64 KiB
 * array that every GPU loading the library holds until the process exits.
 *   x, y, attrs, out  device buffers of the current CUDA device, contiguous;
 *                     count must be given, and sum[a] whenever avg is asked
 *                     for (they hold the running state); other outputs as
 *                     selected by ops. Buffer streams are ignored.
 *   ops               BN_OP_* and BN_SUM_* bits; no accumulate or strategy bits
 *   stream            all work is queued here (NULL = legacy default stream)
 *   sync              1: wait and return the device status (e.g.
 *                     BN_ERR_DEGENERATE); 0: return after queueing, device
 *                     errors are then not reported. After an asynchronous
 *                     call whose automatic bounds collapsed, the outputs
 *                     hold the empty mesh (count 0, sum +0.0, min +inf, max
 *                     -inf, avg NaN), the same as for input with no particle
 *                     inside; give a bounds output to tell the two apart
 *                     (it then holds four NaN)
 * Limit: f64 meshes need res_x + res_y <= 8062 (the edge keys must fit the
 * array); larger meshes are rejected with BN_ERR_INVALID_ARG. f32 meshes
 * have the usual limits.
 * The first call on each device looks up the array's device address; make
 * that first call before any stream capture. Calls share the array and it
 * keeps the last call's contents (each call rewrites what it reads); calls
 * whose work overlaps on the GPU race on it and must be serialised.
 */
BN_API bn_status bn_bin_particles_static(const bn_buffer* x, const bn_buffer* y,
                                         const bn_buffer* attrs, int n_attrs,
                                         const bn_grid* grid, uint32_t ops,
                                         const bn_result* out, void* stream, int sync);

/*
 * Bin many independent blocks, each with its own columns, mesh and outputs,
 * in one persistent launch (the many binning operations per in situ step of
 * Sec. 4.3). Every block follows the rules of bn_bin_particles; all blocks
 * share one dtype, `ops` and n_attrs. The library chooses a strategy per
 * block (its autotuner) unless `ops` names one (BN_STRATEGY_HYBRID blocks
 * run the global strategy: batch blocks have no window). Repeated batches
 * with the same block shapes replay a cached CUDA graph.
 */
BN_API bn_status bn_bin_batch(bn_context* ctx, const bn_block* blocks, int n_blocks, uint32_t ops,
                       int sync, bn_request** req);

/*
 * Fused multi-grid pass: n_specs binnings of the same particles in one
 * launch. Sec. 4.3 bins 10 variables in 9 coordinate systems every step (90
 * binning operations, run one after another in the paper); here the
 * particles are visited in tiles and every spec of a tile is binned before
 * the next tile, so each column is read from memory once however many
 * specs use it.
 *   cols[0..n_cols)     1..BN_MAX_MULTI_COLS columns, same n and dtype,
 *                       device or host memory as for bn_bin_particles
 *   specs[0..n_specs)   1..BN_MAX_MULTI_SPECS binnings; column indices in
 *                       [0, n_cols); explicit bounds only
 *   ops                 as bn_bin_particles, without BN_OP_ACCUMULATE and
 *                       strategy bits (aggregation bits apply)
 *   outs[0..n_specs)    outs[k] receives spec k's result (bn_result rules)
 * Each spec's result equals bn_bin_particles on its columns and grid
 * (counts, min and max exactly; sums to within rounding order). Errors as
 * bn_bin_particles; BN_ERR_INVALID_ARG for an index out of range,
 * automatic bounds, accumulate or a strategy.
 */
BN_API bn_status bn_bin_multi(bn_context* ctx, const bn_buffer* cols, int n_cols,
                              const bn_grid_spec* specs, int n_specs, uint32_t ops,
                              bn_result* outs, int sync, bn_request** req);

/*
 * Combine n_parts finalized results of one mesh into `out` (the cross-rank
 * merge implied by the MPI-parallel binning of Sec. 4.2): counts and sums
 * add, min and max combine, avg = sum / count. Each part must hold count,
 * sum, min and max (device buffers of the context's device); out follows
 * bn_result rules. dtype is the parts' min/max type.
 */
BN_API bn_status bn_merge_results(bn_context* ctx, const bn_result* parts, int n_parts,
                           int32_t dtype, int n_attrs, int64_t bins, uint32_t ops,
                           bn_result* out, int sync, bn_request** req);

/* ----------------------------------------------------------------- ranks */

/*
 * Partial meshes across ranks. Sec. 4.2 parallelises the binning with MPI:
 * each rank bins the bodies of its own subdomain onto the same mesh, and
 * the partial meshes combine. The library packs a rank's result into an
 * exchange buffer of four sections, each combined across ranks by one
 * element-wise collective the caller runs (ncclAllReduce, MPI_Allreduce,
 * torch.distributed.all_reduce):
 *   bytes [0, 8B)            count  u64 [B]      reduce with SUM
 *   bytes [8B, 8B(1+A))      sum    f64 [A][B]   reduce with SUM
 *   bytes [8B(1+A), 8B(1+2A)) minkey s64 [A][B]  reduce with MIN
 *   bytes [8B(1+2A), 8B(1+3A)) maxkey s64 [A][B] reduce with MAX
 * (B bins, A attributes; per-attribute arrays attribute-major). A key is the
 * IEEE totalOrder key of the min or max value as a signed integer (the bits
 * of a non-negative value; a negative value's bits with the 63 (f64) or 31
 * (f32) magnitude bits flipped, f32 keys sign-extended to 64 bits), so
 * integer MIN / MAX are totalOrder min / max: -0 < +0, and the empty-bin
 * values +inf / -inf are the identities. A float MIN / MAX on the values
 * themselves would not order -0 and +0.
 */

/* Bytes of the exchange buffer of a mesh of `bins` bins and n_attrs
 * attributes (0 for arguments out of range). */
BN_API size_t bn_exchange_bytes(int64_t bins, int n_attrs);

/* Pack `partial` (count, sum, min and max of every attribute: device
 * buffers of the context's device, as bn_bin_particles or bn_merge_results
 * wrote them) into `exchange`, a device buffer of bn_exchange_bytes bytes,
 * 8-byte aligned. dtype is the min/max type. Request semantics as
 * bn_bin_particles. */
BN_API bn_status bn_exchange_pack(bn_context* ctx, const bn_result* partial, int32_t dtype, int n_attrs,
                                  int64_t bins, void* exchange, int sync, bn_request** req);

/* After the collective: write count and the outputs `ops` selects (sum,
 * min, max, avg = sum / count, recomputed) from `exchange` into `out`
 * (device buffers of the context's device). */
BN_API bn_status bn_exchange_unpack(bn_context* ctx, const void* exchange, int32_t dtype, int n_attrs,
                                    int64_t bins, uint32_t ops, bn_result* out, int sync, bn_request** req);

/* Automatic device placement (Sec. 3, Eq. 1): the device a rank's in situ
 * work runs on, d = ((rank mod n_use) * stride + offset) mod n_avail.
 * n_use <= 0 and stride <= 0 take the paper's defaults (n_use = n_avail,
 * stride = 1; offset defaults to 0). A negative result of the sum wraps
 * into [0, n_avail). BN_ERR_INVALID_ARG for rank < 0 or n_avail < 1. */
BN_API bn_status bn_select_device(int rank, int n_use, int stride, int offset, int n_avail, int* device);

/* ----------------------------------------------------------------- requests */

/* BN_OK when done without error, BN_NOT_READY while running, else the
 * request's error (Listing 3/4: Synchronize() before using moved data). */
BN_API bn_status bn_query(bn_request* req);

/* Wait up to timeout_us microseconds (< 0: no limit). BN_ERR_TIMEOUT if the
 * request is still running; otherwise as bn_query. The blocking form of
 * bn_query: the Synchronize() the paper's Listings 3 and 4 call before the
 * host touches data produced on a device. */
BN_API bn_status bn_wait(bn_request* req, int64_t timeout_us);

/* Release a request: waits for completion if it is still running, runs the
 * deleters of the input handles it was given (the coordinated life cycle of
 * zero-copy buffers, Listing 1's shared_ptr deleter), frees its temporaries. */
BN_API bn_status bn_request_release(bn_request* req);

/* Free a library-allocated output (calls its deleter) and zero the handle
 * (the shared_ptr deleter of Listing 1: the memory's life ends with its
 * handle). Library outputs return to the stream-ordered pool on the stream
 * that allocated them, after the work queued there, without synchronising
 * the device; release them before destroying the context that made them. A
 * borrowed handle (no deleter) is only zeroed. */
BN_API bn_status bn_buffer_release(bn_buffer* buf);

/* ----------------------------------------------------------------- serving */

typedef struct bn_server_options {
    size_t budget_bytes;     /* device memory the server may hold for admitted
                                requests: input copies + temporaries (an upper
                                bound of what each request's strategy may use) */
    int32_t max_inflight;    /* launches in flight at once (default 4) */
    int32_t max_batch;       /* requests merged into one launch (default 64) */
    int32_t stream_priority; /* of the server's streams (default: lowest) */
    int32_t reserved;
    size_t staging_bytes;    /* page-locked host arena allocated once at
                                creation for the deep copies of requests that
                                do not fit the budget at submit time
                                (0 = min(budget / 4, 4 GiB)) */
} bn_server_options;

typedef struct bn_server_stats {
    uint64_t submitted, admitted, completed, failed;
    uint64_t launches;
    size_t bytes_in_use, peak_bytes;
    uint64_t staged;           /* deep copies placed in the staging arena */
    uint64_t staging_overflow; /* deep copies that found the arena full and
                                  took a page-locked allocation of their own */
    uint64_t overdrawn;        /* requests whose temporaries exceeded what
                                  admission charged (0 unless the accounting
                                  is wrong) */
} bn_server_stats;

/* Where one server request's time went (host clock, microseconds). */
typedef struct bn_request_timing {
    double submit_us;    /* inside bn_server_submit: checks and the deep copy queued */
    double queue_us;     /* submit returned -> admitted by the server */
    double launch_us;    /* admitted -> its batch queued on a stream */
    double complete_us;  /* batch queued -> completion seen by the server */
    double batch_gpu_us; /* device time of its batch, events on the batch's stream
                            (includes waiting for SMs held by other work) */
    int32_t batch_size;  /* requests in its batch */
    int32_t staged;      /* deep copy: 0 device memory, 1 staging arena,
                            2 a page-locked allocation of its own */
} bn_request_timing;

/*
 * The asynchronous in situ method of Sec. 3: a server that deep-copies each
 * submitted block (so the caller may reuse its buffers as soon as submit
 * returns, as with the asynchronous deep copy of Sec. 4.3), admits requests
 * while their memory fits `budget_bytes`, and merges admitted requests into
 * batched launches that overlap on the device with other work (continuous
 * batching). Each request's result is identical to binning its block alone.
 * Server batches never run the autotuner's timed trials (they synchronise
 * with the device and would stall every queued request): a shape class the
 * context has tuned keeps its measured choice, others take the heuristic one.
 */
BN_API bn_status bn_server_create(bn_context* ctx, const bn_server_options* opt, bn_server** srv);

/* Never blocks on the device: copies the block's columns into device memory
 * when the budget has room (device inputs) or into the server's page-locked
 * staging arena (host inputs, or no room yet; only when the arena is full
 * does it allocate page-locked memory, which can take milliseconds), queues
 * the request and returns a request handle to poll or wait on.
 * BN_ERR_BUDGET if the request alone exceeds the budget. Outputs must be
 * caller-allocated (device or host) and must stay valid until the request
 * completes. */
BN_API bn_status bn_server_submit(bn_server* srv, const bn_block* block, uint32_t ops, bn_request** req);

/* The timing record of a completed server request (BN_NOT_READY while it
 * runs; BN_ERR_INVALID_ARG for a request that did not come from a server). */
BN_API bn_status bn_server_request_timing(bn_request* req, bn_request_timing* timing);

BN_API bn_status bn_server_stats_get(bn_server* srv, bn_server_stats* stats);

/* Finishes every queued and running request, then frees the server. */
BN_API bn_status bn_server_destroy(bn_server* srv);

/* ----------------------------------------------------------------- errors */

/* Message for the last error on the calling thread ("" if none). */
BN_API const char* bn_last_error(void);

/* Library version string. */
BN_API const char* bn_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BINNING_H */
