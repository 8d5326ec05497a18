// batch.cu -- bn_bin_batch: many independent blocks in one request (the 90
// binning operations per in situ step of Sec. 4.3).
//
// Fast path (every block's columns and outputs on the context's device,
// contiguous, explicit bounds): one persistent launch over all blocks
// (k_batch.cu) between one init/edge launch and one finalise launch. The
// launches are captured once per plan shape in a CUDA graph; a later batch
// with the same shape (block sizes, meshes, strategies) only rewrites the
// block descriptors, and the arguments of the blocks on the sort path, in
// pinned memory and replays the graph (its copy nodes move them to the
// device; the sort blocks' scratch lives in the plan's memory).
//
// Autotuner: blocks fall into shape classes (dtype, attributes, ops, log2
// of the bin count, log2 of the particle count). The first block of a new
// class is binned once with each candidate strategy (shared-memory private
// mesh if it fits; global atomics with and without warp aggregation) by the
// batch kernel itself, timed with CUDA events, and the fastest is kept for
// the class. CTA tiling follows from the strategy and the block size: a
// private item carries enough particles per bin to amortise clearing and
// merging its mesh, and large blocks are cut so every SM gets work.
//
// Anything else (host or strided columns, automatic bounds, mixed types)
// takes the general path: each block queued as in bn_bin_particles.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "bn_runtime.h"

using namespace bn;

namespace {

struct ClassKey {
    int dtype, n_attrs;
    uint32_t ops;
    int lb, ln;
    bool operator<(const ClassKey& o) const {
        return std::tie(dtype, n_attrs, ops, lb, ln) < std::tie(o.dtype, o.n_attrs, o.ops, o.lb, o.ln);
    }
};

struct Choice {
    int strategy;
    int aggregate;
    int banded;  // private in mesh bands (blocks whose mesh exceeds shared memory)
};

// The most bands a private block's mesh is cut into: each band re-reads the
// tile's coordinates (from L2 after the first band).
constexpr int kMaxBands = 16;

// Cached graph of one plan shape, with the device and pinned memory it uses.
struct BatchGraph {
    std::vector<int64_t> shape;
    cudaGraphExec_t exec = nullptr;
    void* dev = nullptr;
    void* host = nullptr;
    BatchBlock* h_blocks = nullptr;
    BatchBlock* d_blocks = nullptr;
    cudaEvent_t last = nullptr;  // completion of the last replay (pinned buffer reuse)
    uint64_t launches = 0;       // kernels per replay
    // blocks on the sort path: their scratch and a device copy of their
    // arguments (sort_dev), rewritten from sort_args before every replay, so
    // the captured kernels' parameters stay the same from call to call
    void* sort_dev = nullptr;
    BinArgs* sort_args = nullptr;  // pinned, one per sort block
    size_t sort_args_off = 0;
    std::vector<size_t> sort_off;
    std::vector<SortDesc> sort_sd;
    // side streams of the capture: the sort blocks' kernel chains are
    // independent, so they fork off the context stream after the prepare
    // launch and join it before the finalise (parallel graph branches)
    static constexpr int kSide = 4;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork = nullptr, join[kSide] = {};
    ~BatchGraph() {
        if (last) cudaEventSynchronize(last), cudaEventDestroy(last);
        for (int s = 0; s < kSide; ++s) {
            if (side[s]) cudaStreamDestroy(side[s]);
            if (join[s]) cudaEventDestroy(join[s]);
        }
        if (fork) cudaEventDestroy(fork);
        if (exec) cudaGraphExecDestroy(exec);
        if (dev) cudaFree(dev);
        if (host) cudaFreeHost(host);
        if (sort_dev) cudaFree(sort_dev);
        if (sort_args) cudaFreeHost(sort_args);
    }
};

struct BatchCache {
    std::mutex mu;
    std::map<ClassKey, Choice> choices;
    std::map<std::vector<int64_t>, int> lean;  // batch shape -> sort-leaning plan chosen
    std::vector<std::unique_ptr<BatchGraph>> graphs;  // most recent last
};

std::mutex g_cache_mu;
std::map<bn_context*, std::unique_ptr<BatchCache>> g_caches;

BatchCache& cache_of(bn_context* c) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto& p = g_caches[c];
    if (!p) p.reset(new BatchCache());
    return *p;
}

int ilog2(int64_t v) {
    int r = 0;
    while (v > 1) v >>= 1, ++r;
    return r;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Particles per work item for a block and strategy (the CTA tiling).
int64_t choose_tile(int strategy, int64_t n, int64_t bins, int num_sms) {
    if (strategy == BN_STRATEGY_PRIVATE) {
        // at least 8 particles per bin so clearing and merging the mesh is
        // amortised, at least 32K, and no more items than 2 per SM need;
        // at most kLimbMaxAdds (the most one limb-sum mesh may take per bin)
        int64_t t = std::max<int64_t>(8 * bins, 32768);
        t = std::max<int64_t>(t, (n + 2 * num_sms - 1) / (2 * num_sms));
        t = std::min<int64_t>(t, kLimbMaxAdds);
        return std::min<int64_t>(t, std::max<int64_t>(n, 1));
    }
    int64_t t = (n + 4 * num_sms - 1) / (4 * num_sms);
    t = std::min<int64_t>(std::max<int64_t>(t, 16384), 262144);
    return std::max<int64_t>(std::min<int64_t>(t, n), 1);
}

}  // namespace

namespace bn {

// Release the batch caches of a context (called from bn_context_destroy).
void batch_cache_release(bn_context* c) {
    std::unique_ptr<BatchCache> p;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_caches.find(c);
        if (it == g_caches.end()) return;
        p = std::move(it->second);
        g_caches.erase(it);
    }
}

}  // namespace bn

// Everything the fast path needs per block, validated.
struct FastBlock {
    BatchBlock bb;
    int64_t bins;
    int64_t edges;  // f64: res_x + res_y + 2
    ClassKey cls;
};

static bool fast_eligible(bn_context* c, const bn_block* blocks, int n_blocks) {
    if (n_blocks < 1) return false;
    const int dtype = blocks[0].x.dtype;
    const int A = blocks[0].n_attrs;
    for (int k = 0; k < n_blocks; ++k) {
        const bn_block& b = blocks[k];
        if (b.x.dtype != dtype || b.n_attrs != A || b.grid.auto_bounds) return false;
        const bn_buffer* cols[2 + BN_MAX_ATTR] = {&b.x, &b.y};
        for (int a = 0; a < b.n_attrs; ++a) cols[2 + a] = &b.attrs[a];
        for (int j = 0; j < 2 + b.n_attrs; ++j)
            if (cols[j]->n > 0 && (cols[j]->device != c->device || cols[j]->stride > 1)) return false;
        const bn_result* o = b.out;
        const bn_buffer* outs[1 + 4 * BN_MAX_ATTR] = {&o->count};
        int no = 1;
        for (int a = 0; a < b.n_attrs; ++a) {
            outs[no++] = &o->sum[a];
            outs[no++] = &o->min[a];
            outs[no++] = &o->max[a];
            outs[no++] = &o->avg[a];
        }
        for (int j = 0; j < no; ++j)
            if (outs[j]->ptr && (outs[j]->device != c->device || outs[j]->stride > 1)) return false;
    }
    return true;
}

// Queue prepare + persistent bin + finalize for `fb` (used for the graph
// capture and for autotuner trials). Device arrays must be filled.
static cudaError_t queue_batch(const KernelCtx& kc, int dtype, int sum_mode, int n_attrs,
                               BatchBlock* d_blocks, const int64_t* d_bin_start,
                               const int64_t* d_edge_start, const int4* d_items, int* d_counter,
                               int nblk, int n_items, int64_t total_bins, int64_t total_edges,
                               size_t smem, bool want_avg) {
    cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(int), kc.stream);
    if (e == cudaSuccess)
        e = launch_batch_prepare(kc, dtype, d_blocks, d_bin_start, d_edge_start, nblk, total_bins, total_edges);
    if (e == cudaSuccess && n_items > 0)
        e = launch_batch_bin(kc, dtype, sum_mode, d_blocks, d_items, n_items, d_counter, n_attrs, smem);
    if (e == cudaSuccess && want_avg) e = launch_batch_finalize(kc, d_blocks, d_bin_start, nblk, total_bins);
    return e;
}

// Layout of the per-plan device block: descriptors, starts, items, counter, edges.
struct PlanLayout {
    size_t off_blocks, off_bin_start, off_edge_start, off_items, off_counter, off_edges, bytes;
};

static PlanLayout layout_for(int nblk, int n_items, int64_t total_edges) {
    PlanLayout L;
    size_t o = 0;
    L.off_blocks = o;
    o += align256(sizeof(BatchBlock) * nblk);
    L.off_bin_start = o;
    o += align256(sizeof(int64_t) * (nblk + 1));
    L.off_edge_start = o;
    o += align256(sizeof(int64_t) * (nblk + 1));
    L.off_items = o;
    o += align256(sizeof(int4) * std::max(n_items, 1));
    L.off_counter = o;
    o += 256;
    L.off_edges = o;
    o += align256(sizeof(long long) * std::max<int64_t>(total_edges, 1));
    L.bytes = o;
    return L;
}

// Build items, starts and the per-block edge pointers for a plan in `host`
// (pinned, layout L) whose device copy lives at `dev`.
static void fill_plan(std::vector<FastBlock>& fbs, const PlanLayout& L, unsigned char* host,
                      unsigned char* dev, int* n_items_out, int64_t* bins_out, int64_t* edges_out,
                      int dtype) {
    int64_t* bs = reinterpret_cast<int64_t*>(host + L.off_bin_start);
    int64_t* es = reinterpret_cast<int64_t*>(host + L.off_edge_start);
    int4* items = reinterpret_cast<int4*>(host + L.off_items);
    long long* d_edges = reinterpret_cast<long long*>(dev + L.off_edges);
    int64_t bins = 0, edges = 0;
    const int nblk = (int)fbs.size();
    for (int k = 0; k < nblk; ++k) {
        bs[k] = bins;
        es[k] = edges;
        FastBlock& f = fbs[k];
        if (dtype == BN_F64) {
            f.bb.g.edges[0] = d_edges + edges;
            f.bb.g.edges[1] = d_edges + edges + f.bb.g.ax[0].res + 1;
            edges += f.edges;
        }
        bins += f.bins;
    }
    bs[nblk] = bins;
    es[nblk] = edges;
    // items: largest blocks first so the long ones start early
    std::vector<int> order(nblk);
    for (int k = 0; k < nblk; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return fbs[a].bb.n > fbs[b].bb.n; });
    int ni = 0;
    for (int k : order) {
        const FastBlock& f = fbs[k];
        if (f.bb.n == 0 || f.bb.strategy == BN_STRATEGY_SORT) continue;  // sort blocks: own launches
        const int64_t parts = (f.bb.n + f.bb.tile - 1) / f.bb.tile;
        const int nb = std::max(f.bb.bands, 1);
        // a tile's bands next to each other: they run together and read the
        // tile's coordinates from DRAM once
        for (int64_t j = 0; j < parts; ++j)
            for (int band = 0; band < nb; ++band) items[ni++] = make_int4(k, (int)j, band, 0);
    }
    BatchBlock* hb = reinterpret_cast<BatchBlock*>(host + L.off_blocks);
    for (int k = 0; k < nblk; ++k) hb[k] = fbs[k].bb;
    *n_items_out = ni;
    *bins_out = bins;
    *edges_out = edges;
}

static int count_items(const std::vector<FastBlock>& fbs) {
    int64_t ni = 0;
    for (const FastBlock& f : fbs)
        if (f.bb.n > 0 && f.bb.strategy != BN_STRATEGY_SORT)
            ni += (f.bb.n + f.bb.tile - 1) / f.bb.tile * std::max(f.bb.bands, 1);
    return (int)ni;
}

// BinArgs of a block that takes the bucketed sort path. The mesh descriptor
// goes by value; its f64 edge keys point into the batch plan's memory, which
// the prepare launch fills first.
static BinArgs sort_args(const FastBlock& f, int dtype, int n_attrs, int sum_mode) {
    BinArgs a;
    memset(&a, 0, sizeof a);
    a.dtype = dtype;
    a.n_attrs = n_attrs;
    a.sum_mode = sum_mode;
    a.x = f.bb.x;
    a.y = f.bb.y;
    for (int k = 0; k < n_attrs; ++k) a.a[k] = f.bb.a[k];
    a.n = f.bb.n;
    a.grid = f.bb.g;
    a.dev_grid = nullptr;
    a.st = f.bb.st;
    return a;
}

// Time one block alone with one strategy (autotuner trial), on the context
// stream; the block's outputs are overwritten (the batch recomputes them).
static float trial(bn_context* c, FastBlock f, int strategy, int aggregate, int dtype, int sum_mode,
                   int n_attrs, size_t smem, bool want_avg, int bands = 1, int band_rows = 0) {
    f.bb.strategy = strategy;
    f.bb.aggregate = aggregate;
    f.bb.bands = bands;
    f.bb.band_rows = band_rows;
    f.bb.tile = choose_tile(strategy, f.bb.n, bands > 1 ? (int64_t)band_rows * f.bb.g.ax[0].res : f.bins,
                            c->num_sms);
    std::vector<FastBlock> one{f};
    const int n_items = count_items(one);
    PlanLayout L = layout_for(1, n_items, f.edges);
    void* dev = nullptr;
    void* host = nullptr;
    float ms = -1.0f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMallocAsync(&dev, L.bytes, c->stream) != cudaSuccess) return -1.0f;
    if (cudaHostAlloc(&host, L.bytes, cudaHostAllocDefault) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        int ni;
        int64_t bins, edges;
        fill_plan(one, L, static_cast<unsigned char*>(host), static_cast<unsigned char*>(dev), &ni,
                  &bins, &edges, dtype);
        unsigned char* d = static_cast<unsigned char*>(dev);
        const KernelCtx kc{c->stream, c->num_sms, c->smem_optin, nullptr};
        cudaError_t e = cudaMemcpyAsync(dev, host, L.bytes, cudaMemcpyHostToDevice, c->stream);
        SortDesc sd;
        void* sort_scratch = nullptr;
        BinArgs sa;
        if (strategy == BN_STRATEGY_SORT) {
            sa = sort_args(one[0], dtype, n_attrs, sum_mode);
            if (!sort_plan(sa, c->smem_optin, &sd) ||
                cudaMallocAsync(&sort_scratch, sort_scratch_bytes(sd, sa), c->stream) != cudaSuccess)
                e = cudaErrorInvalidValue;
        }
        auto run = [&]() {
            cudaError_t e2 = queue_batch(kc, dtype, sum_mode, n_attrs, reinterpret_cast<BatchBlock*>(d + L.off_blocks),
                                         reinterpret_cast<int64_t*>(d + L.off_bin_start),
                                         reinterpret_cast<int64_t*>(d + L.off_edge_start),
                                         reinterpret_cast<int4*>(d + L.off_items), reinterpret_cast<int*>(d + L.off_counter),
                                         1, ni, bins, edges, smem, false);
            if (e2 == cudaSuccess && strategy == BN_STRATEGY_SORT) e2 = launch_bin_sort(kc, sa, sd, sort_scratch);
            if (e2 == cudaSuccess && want_avg)
                e2 = launch_batch_finalize(kc, reinterpret_cast<BatchBlock*>(d + L.off_blocks),
                                           reinterpret_cast<int64_t*>(d + L.off_bin_start), 1, bins);
            return e2;
        };
        if (e == cudaSuccess) e = run();  // untimed: the first launch also loads the module
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess) e = run();
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (sort_scratch) cudaFreeAsync(sort_scratch, c->stream);
    }
    cudaFreeAsync(dev, c->stream);
    cudaStreamSynchronize(c->stream);
    if (host) cudaFreeHost(host);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return ms;
}

// Find or build (capture once) the graph of the plan `fbs` describes and
// launch it on the context stream.
// The key of a plan's cached graph: everything that fixes its kernels and
// launch shapes.
static std::vector<int64_t> plan_shape(const std::vector<FastBlock>& fbs, int dtype, int A, uint32_t ops) {
    std::vector<int64_t> shape;
    shape.reserve(4 + 6 * fbs.size());
    shape.push_back(dtype);
    shape.push_back(A);
    shape.push_back(ops & ~(uint32_t)BN_STRATEGY_MASK);
    shape.push_back((int64_t)fbs.size());
    for (const FastBlock& f : fbs) {
        shape.push_back(f.bb.n);
        shape.push_back(f.bb.g.ax[0].res);
        shape.push_back(f.bb.g.ax[1].res);
        shape.push_back(f.bb.strategy * 2 + f.bb.aggregate);
        shape.push_back(f.bb.tile);
        shape.push_back(f.bb.bands);
    }
    return shape;
}

static bn_status launch_plan(bn_context* c, BatchCache& cache, std::vector<FastBlock>& fbs, int dtype, int A,
                             uint32_t ops, int sum_mode, bool want_avg, size_t smem) {
    const int n_blocks = (int)fbs.size();
    const std::vector<int64_t> shape = plan_shape(fbs, dtype, A, ops);
    const int n_items = count_items(fbs);
    int64_t total_edges = 0;
    for (const FastBlock& f : fbs) total_edges += f.edges;
    PlanLayout L = layout_for(n_blocks, n_items, total_edges);

    BatchGraph* G = nullptr;
    {
        std::lock_guard<std::mutex> lk(cache.mu);
        for (auto& g : cache.graphs)
            if (g->shape == shape) G = g.get();
    }
    int ni = n_items;
    int64_t bins = 0, edges = 0;
    for (const FastBlock& f : fbs) bins += f.bins;
    edges = total_edges;
    if (!G) {
        std::unique_ptr<BatchGraph> ng(new BatchGraph());
        ng->shape = shape;
        cudaError_t e = cudaMalloc(&ng->dev, L.bytes);
        if (e == cudaSuccess) e = cudaHostAlloc(&ng->host, L.bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ng->last, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "bn_bin_batch: plan memory");
        fill_plan(fbs, L, static_cast<unsigned char*>(ng->host), static_cast<unsigned char*>(ng->dev), &ni,
                  &bins, &edges, dtype);
        ng->h_blocks = reinterpret_cast<BatchBlock*>(static_cast<unsigned char*>(ng->host) + L.off_blocks);
        ng->d_blocks = reinterpret_cast<BatchBlock*>(static_cast<unsigned char*>(ng->dev) + L.off_blocks);
        // the static part (starts, items) goes over once
        e = cudaMemcpy(ng->dev, ng->host, L.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "bn_bin_batch: plan upload");
        std::lock_guard<std::mutex> lk(cache.mu);
        cache.graphs.push_back(std::move(ng));
        if (cache.graphs.size() > 8) cache.graphs.erase(cache.graphs.begin());
        G = cache.graphs.back().get();
    } else {
        // same shape: wait until the pinned descriptors are free, rewrite them
        cudaEventSynchronize(G->last);
        unsigned char* host = static_cast<unsigned char*>(G->host);
        int64_t edge_off = 0;
        for (int k = 0; k < n_blocks; ++k) {
            FastBlock& f = fbs[k];
            if (dtype == BN_F64) {
                long long* d_edges = reinterpret_cast<long long*>(static_cast<unsigned char*>(G->dev) + L.off_edges);
                f.bb.g.edges[0] = d_edges + edge_off;
                f.bb.g.edges[1] = d_edges + edge_off + f.bb.g.ax[0].res + 1;
                edge_off += f.edges;
            }
            reinterpret_cast<BatchBlock*>(host + L.off_blocks)[k] = f.bb;
        }
    }

    // blocks on the sort path: scratch and argument copies in the plan's own
    // memory (sized once per plan shape), arguments rewritten every call
    std::vector<const FastBlock*> sort_blocks;
    for (const FastBlock& f : fbs)
        if (f.bb.strategy == BN_STRATEGY_SORT && f.bb.n > 0) sort_blocks.push_back(&f);
    const size_t n_sorts = sort_blocks.size();
    if (n_sorts && !G->sort_dev) {
        size_t off = 0;
        for (const FastBlock* f : sort_blocks) {
            const BinArgs a = sort_args(*f, dtype, A, sum_mode);
            SortDesc sd;
            if (!sort_plan(a, c->smem_optin, &sd)) return fail(BN_ERR_INTERNAL, "bn_bin_batch: no sort plan");
            G->sort_sd.push_back(sd);
            G->sort_off.push_back(off);
            off += align256(sort_scratch_bytes(sd, a));
        }
        G->sort_args_off = off;
        off += align256(sizeof(BinArgs) * n_sorts);
        cudaError_t e = cudaMalloc(&G->sort_dev, off);
        if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&G->sort_args), sizeof(BinArgs) * n_sorts,
                                                cudaHostAllocDefault);
        if (e != cudaSuccess) return cuda_fail(e, "bn_bin_batch: sort plan memory");
    }
    // the previous replay has released the pinned copies (G->last waited above)
    for (size_t j = 0; j < n_sorts; ++j) G->sort_args[j] = sort_args(*sort_blocks[j], dtype, A, sum_mode);
    unsigned char* sdev = static_cast<unsigned char*>(G->sort_dev);
    BinArgs* d_sort_args = n_sorts ? reinterpret_cast<BinArgs*>(sdev + G->sort_args_off) : nullptr;

    unsigned char* d = static_cast<unsigned char*>(G->dev);
    std::atomic<uint64_t> nlaunch{0};
    const KernelCtx kc{c->stream, c->num_sms, c->smem_optin, &nlaunch};
    // parallel: fork the sort blocks' chains onto the side streams (capture
    // only; a direct launch keeps them on the context stream, in order)
    auto body = [&](bool parallel) {
        cudaError_t e2 = cudaMemcpyAsync(G->d_blocks, G->h_blocks, sizeof(BatchBlock) * n_blocks,
                                         cudaMemcpyHostToDevice, c->stream);
        if (e2 == cudaSuccess) e2 = cudaMemsetAsync(d + L.off_counter, 0, sizeof(int), c->stream);
        if (e2 == cudaSuccess)
            e2 = launch_batch_prepare(kc, dtype, G->d_blocks, reinterpret_cast<int64_t*>(d + L.off_bin_start),
                                      reinterpret_cast<int64_t*>(d + L.off_edge_start), n_blocks, bins, edges);
        if (e2 == cudaSuccess && n_sorts)
            e2 = cudaMemcpyAsync(d_sort_args, G->sort_args, sizeof(BinArgs) * n_sorts, cudaMemcpyHostToDevice,
                                 c->stream);
        const int n_side = parallel ? (int)std::min<size_t>(n_sorts, BatchGraph::kSide) : 0;
        if (e2 == cudaSuccess && n_side > 0) {
            e2 = cudaEventRecord(G->fork, c->stream);
            for (int k = 0; k < n_side && e2 == cudaSuccess; ++k) e2 = cudaStreamWaitEvent(G->side[k], G->fork, 0);
        }
        for (size_t j = 0; j < n_sorts && e2 == cudaSuccess; ++j) {
            KernelCtx kj = kc;
            if (n_side > 0) kj.stream = G->side[j % n_side];
            e2 = launch_bin_sort(kj, G->sort_args[j], G->sort_sd[j], sdev + G->sort_off[j], d_sort_args + j);
        }
        if (e2 == cudaSuccess && ni > 0)
            e2 = launch_batch_bin(kc, dtype, sum_mode, G->d_blocks, reinterpret_cast<int4*>(d + L.off_items), ni,
                                  reinterpret_cast<int*>(d + L.off_counter), A, smem);
        for (int k = 0; k < n_side && e2 == cudaSuccess; ++k) {
            e2 = cudaEventRecord(G->join[k], G->side[k]);
            if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(c->stream, G->join[k], 0);
        }
        if (e2 == cudaSuccess && want_avg)
            e2 = launch_batch_finalize(kc, G->d_blocks, reinterpret_cast<int64_t*>(d + L.off_bin_start), n_blocks, bins);
        return e2;
    };
    const bool capturable = c->stream != nullptr && c->stream != cudaStreamLegacy;
    if (!capturable) {
        // no graph on the legacy stream: launch directly
        cudaError_t e2 = body(false);
        if (e2 != cudaSuccess) return cuda_fail(e2, "bn_bin_batch: launch");
        c->launches.fetch_add(nlaunch.load());
        cudaEventRecord(G->last, c->stream);
        return BN_OK;
    }
    if (!G->exec) {
        // capture once per plan shape: every per-call value (block
        // descriptors, sort arguments) reaches the kernels through the plan's
        // memory, which the graph's copy nodes rewrite from pinned buffers
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaSuccess;
        if (n_sorts && !G->fork) {
            e = cudaEventCreateWithFlags(&G->fork, cudaEventDisableTiming);
            for (int k = 0; k < BatchGraph::kSide && e == cudaSuccess; ++k) {
                e = cudaStreamCreateWithFlags(&G->side[k], cudaStreamNonBlocking);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->join[k], cudaEventDisableTiming);
            }
            if (e != cudaSuccess) return cuda_fail(e, "bn_bin_batch: side streams");
        }
        e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        cudaError_t eb = e == cudaSuccess ? body(n_sorts > 0) : e;
        cudaError_t ee = cudaStreamEndCapture(c->stream, &graph);
        if (e == cudaSuccess) e = eb != cudaSuccess ? eb : ee;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&G->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "bn_bin_batch: graph capture");
        G->launches = nlaunch.load();
    }
    cudaError_t e = cudaGraphLaunch(G->exec, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "bn_bin_batch: graph launch");
    c->launches.fetch_add(G->launches);
    cudaEventRecord(G->last, c->stream);
    return BN_OK;
}

// Mesh bands for a private block whose whole mesh exceeds shared memory:
// the fewest bands of whole rows that fit, rows spread evenly over them
// (bands = 0: not even one row fits, or more than kMaxBands are needed).
struct Bands {
    int bands, rows;
    size_t bytes;
};
static Bands band_layout(const FastBlock& f, int dtype, int sum_mode, int A, bool s, bool lo, bool hi,
                         int dyn_limit) {
    const int rx = f.bb.g.ax[0].res, ry = f.bb.g.ax[1].res;
    auto bytes = [&](int rows) { return private_mesh_bytes(dtype, sum_mode, (int64_t)rows * rx, A, s, lo, hi); };
    int fit = 0;
    for (int lo_r = 1, hi_r = ry; lo_r <= hi_r;) {  // largest row count that fits
        const int mid = lo_r + (hi_r - lo_r) / 2;
        if (bytes(mid) <= (size_t)dyn_limit) fit = mid, lo_r = mid + 1;
        else hi_r = mid - 1;
    }
    if (fit == 0) return Bands{0, 0, 0};
    const int bands = (ry + fit - 1) / fit;
    if (bands > kMaxBands) return Bands{0, 0, 0};
    const int rows = (ry + bands - 1) / bands;
    return Bands{bands, rows, bytes(rows)};
}

static bn_status batch_fast(bn_context* c, const bn_block* blocks, int n_blocks, uint32_t ops,
                            bn_request* r, Plan& plan) {
    const int dtype = blocks[0].x.dtype;
    const uint32_t sum_bits = ops & BN_SUM_MASK;
    const int sum_mode = dtype == BN_F64 ? kSumF64 : sum_bits == BN_SUM_F32 ? kSumF32
                                                   : sum_bits == BN_SUM_F64 ? kSumF64 : kSumF32C;
    const bool want_avg = ops & BN_OP_AVG, want_sum = ops & BN_OP_SUM;
    const bool want_min = ops & BN_OP_MIN, want_max = ops & BN_OP_MAX, want_count = ops & BN_OP_COUNT;
    // attribute columns are validated; with no per-attribute op they are not read
    const int A_in = blocks[0].n_attrs;
    const int A = (want_sum || want_avg || want_min || want_max) ? A_in : 0;
    const uint32_t forced = ops & BN_STRATEGY_MASK;
    const uint32_t agg = ops & BN_AGG_MASK;
    if (ops & BN_OP_ACCUMULATE) return fail(BN_ERR_INVALID_ARG, "bn_bin_batch: accumulate is not supported for batches");
    const int dyn_limit = c->smem_optin - 1024;  // room for static shared memory

    std::vector<FastBlock> fbs((size_t)n_blocks);
    for (int k = 0; k < n_blocks; ++k) {
        const bn_block& b = blocks[k];
        FastBlock& f = fbs[k];
        memset(&f.bb, 0, sizeof f.bb);
        const int64_t n = b.x.n;
        bn_status st = validate_buffer(c, &b.x, n, dtype, "x");
        if (st == BN_OK) st = validate_buffer(c, &b.y, n, dtype, "y");
        for (int a = 0; a < A_in && st == BN_OK; ++a) st = validate_buffer(c, &b.attrs[a], n, dtype, "attr");
        if (st == BN_OK) st = make_grid_desc(&b.grid, dtype, &f.bb.g);
        if (st != BN_OK) return fail(st, "bn_bin_batch: block %d: %s", k, bn_last_error());
        for (int a = 0; a < 2; ++a) {
            AxisDesc& d = f.bb.g.ax[a];
            const double dl = dtype == BN_F64 ? host_fast_delta(d.lo, d.hi, d.s, d.res) : -1.0;
            d.fast = dl >= 0.0 ? 1 : 0;
            float fd = (float)dl;
            if ((double)fd < dl) fd = nextafterf(fd, INFINITY);
            d.delta = dl >= 0.0 ? fd : 0.0f;
        }
        for (int j = 0; j < 2; ++j) plan.wait_on(j == 0 ? b.x.stream : b.y.stream);
        for (int a = 0; a < A; ++a) plan.wait_on(b.attrs[a].stream);
        f.bb.x = b.x.ptr;
        f.bb.y = b.y.ptr;
        for (int a = 0; a < A; ++a) f.bb.a[a] = b.attrs[a].ptr;
        f.bb.n = n;
        f.bins = (int64_t)b.grid.res[0] * b.grid.res[1];
        f.edges = dtype == BN_F64 ? (int64_t)b.grid.res[0] + b.grid.res[1] + 2 : 0;
        StateDesc& sd = f.bb.st;
        sd.bins = f.bins;
        sd.n_attrs = A;
        sd.do_sum = (want_sum || want_avg) ? 1 : 0;
        sd.do_min = want_min;
        sd.do_max = want_max;
        sd.do_avg = want_avg;
        void* p = nullptr;
        st = plan.output(&b.out->count, want_count, f.bins, BN_U64, false, &p);
        sd.count = static_cast<unsigned long long*>(p);
        for (int a = 0; a < A && st == BN_OK; ++a) {
            if (sd.do_sum) {
                st = plan.output(&b.out->sum[a], want_sum, f.bins, BN_F64, false, &p);
                sd.sum[a] = static_cast<double*>(p);
            }
            if (st == BN_OK && want_min) st = plan.output(&b.out->min[a], true, f.bins, dtype, false, &sd.mn[a]);
            if (st == BN_OK && want_max) st = plan.output(&b.out->max[a], true, f.bins, dtype, false, &sd.mx[a]);
            if (st == BN_OK && want_avg) {
                st = plan.output(&b.out->avg[a], true, f.bins, BN_F64, false, &p);
                sd.avg[a] = static_cast<double*>(p);
            }
        }
        if (st != BN_OK) return st;
        f.cls = ClassKey{dtype, A, ops & (BN_OP_ALL | BN_SUM_MASK), ilog2(f.bins), ilog2(std::max<int64_t>(n, 1))};
    }

    // ---- autotuner: strategy per block
    BatchCache& cache = cache_of(c);
    size_t smem = 0;
    for (int k = 0; k < n_blocks; ++k) {
        FastBlock& f = fbs[k];
        const size_t mesh = private_mesh_bytes(dtype, sum_mode, f.bins, A, f.bb.st.do_sum, want_min, want_max);
        const bool fits = mesh <= (size_t)dyn_limit && f.bins <= (1 << 20);
        const Bands bl = fits ? Bands{1, f.bb.g.ax[1].res, mesh}
                              : band_layout(f, dtype, sum_mode, A, f.bb.st.do_sum, want_min, want_max, dyn_limit);
        const bool bandable = !fits && bl.bands >= 2;
        Choice ch{BN_STRATEGY_GLOBAL, f.bins <= 65536 ? 1 : 0, 0};
        if (forced == BN_STRATEGY_PRIVATE) {
            if (!fits && !bandable)
                return fail(BN_ERR_INVALID_ARG, "bn_bin_batch: block %d mesh does not fit shared memory in %d bands",
                            k, kMaxBands);
            ch.strategy = BN_STRATEGY_PRIVATE;
        } else if (forced == BN_STRATEGY_SORT) {
            SortDesc probe;
            ch.strategy = (f.bb.n > 0 && sort_plan(sort_args(f, dtype, A, sum_mode), c->smem_optin, &probe))
                              ? BN_STRATEGY_SORT : BN_STRATEGY_GLOBAL;
        } else if (forced == BN_STRATEGY_GLOBAL || forced == BN_STRATEGY_HYBRID) {
            // (batch blocks have no shared-memory window: a forced window runs global)
            ch.strategy = BN_STRATEGY_GLOBAL;
        } else {
            std::lock_guard<std::mutex> lk(cache.mu);
            auto it = cache.choices.find(f.cls);
            if (it != cache.choices.end()) {
                ch = it->second;
                if (ch.strategy == BN_STRATEGY_PRIVATE && !fits && !bandable) ch.strategy = BN_STRATEGY_GLOBAL;
            } else if (f.bb.n > 0) {
                float best = -1.0f;
                SortDesc probe;
                const bool sort_fits = f.bb.n >= 4 * (int64_t)c->num_sms * 1024 &&
                                       sort_plan(sort_args(f, dtype, A, sum_mode), c->smem_optin, &probe) &&
                                       probe.nb >= 8;
                const int cands[4][2] = {{BN_STRATEGY_PRIVATE, 0}, {BN_STRATEGY_GLOBAL, 0}, {BN_STRATEGY_GLOBAL, 1},
                                         {BN_STRATEGY_SORT, 0}};
                std::string times;
                for (auto& cd : cands) {
                    if (cd[0] == BN_STRATEGY_PRIVATE && !fits && !bandable) continue;
                    if (cd[0] == BN_STRATEGY_SORT && !sort_fits) continue;
                    const bool band = cd[0] == BN_STRATEGY_PRIVATE && !fits;
                    const float ms = trial(c, f, cd[0], cd[1], dtype, sum_mode, A,
                                           cd[0] == BN_STRATEGY_PRIVATE ? bl.bytes : 0, want_avg,
                                           band ? bl.bands : 1, band ? bl.rows : 0);
                    char tb[64];
                    if (band)
                        snprintf(tb, sizeof tb, " private[%d bands]=%.3fms", bl.bands, ms);
                    else
                        snprintf(tb, sizeof tb, " %s%s=%.3fms",
                                 cd[0] == BN_STRATEGY_PRIVATE ? "private" : cd[0] == BN_STRATEGY_SORT ? "sort" : "global",
                                 cd[0] == BN_STRATEGY_GLOBAL && cd[1] ? "+agg" : "", ms);
                    times += tb;
                    if (ms >= 0.0f && (best < 0.0f || ms < best)) {
                        best = ms;
                        ch = Choice{cd[0], cd[1], band ? 1 : 0};
                    }
                }
                cache.choices[f.cls] = ch;
                char head[128];
                snprintf(head, sizeof head, "batch dtype=%s attrs=%d bins=2^%d n=2^%d:", dtype == BN_F64 ? "f64" : "f32",
                         A, f.cls.lb, f.cls.ln);
                std::lock_guard<std::mutex> lk2(c->tune_mu);
                c->tune_log.push_back(std::string(head) + times + " -> " +
                                      (ch.strategy == BN_STRATEGY_PRIVATE ? (ch.banded ? "private in bands" : "private")
                                       : ch.strategy == BN_STRATEGY_SORT ? "sort"
                                       : ch.aggregate ? "global+agg" : "global"));
            }
        }
        if (agg == BN_AGG_ON) ch.aggregate = 1;
        if (agg == BN_AGG_OFF) ch.aggregate = 0;
        f.bb.strategy = ch.strategy;
        f.bb.aggregate = ch.aggregate;
        const bool banded = ch.strategy == BN_STRATEGY_PRIVATE && !fits;
        f.bb.bands = banded ? bl.bands : 1;
        f.bb.band_rows = banded ? bl.rows : f.bb.g.ax[1].res;
        f.bb.tile = choose_tile(ch.strategy, f.bb.n, banded ? (int64_t)bl.rows * f.bb.g.ax[0].res : f.bins,
                                c->num_sms);
        if (ch.strategy == BN_STRATEGY_PRIVATE) smem = std::max(smem, banded ? bl.bytes : mesh);
    }

    // ---- batch-level check of the per-class choices: inside a batch the sort
    // blocks' kernel chains run as parallel graph branches, which a block's
    // trial alone cannot show, so the first call on a batch shape also times
    // the whole batch with every block of at least 2^16 particles on the sort
    // path, and keeps the faster plan for that shape
    if (!forced && n_blocks > 1) {
        std::vector<int64_t> key{dtype, A, (int64_t)(ops & ~(uint32_t)BN_STRATEGY_MASK), n_blocks};
        for (const FastBlock& f : fbs) {
            key.push_back(f.bb.n);
            key.push_back(f.bb.g.ax[0].res);
            key.push_back(f.bb.g.ax[1].res);
        }
        std::vector<FastBlock> lean = fbs;
        size_t lean_smem = 0;
        bool differs = false;
        for (FastBlock& f : lean) {
            SortDesc probe;
            if (f.bb.strategy != BN_STRATEGY_SORT && f.bb.n >= (1 << 16) &&
                sort_plan(sort_args(f, dtype, A, sum_mode), c->smem_optin, &probe)) {
                f.bb.strategy = BN_STRATEGY_SORT;
                f.bb.aggregate = 0;
                f.bb.bands = 1;
                f.bb.band_rows = f.bb.g.ax[1].res;
                f.bb.tile = choose_tile(BN_STRATEGY_SORT, f.bb.n, f.bins, c->num_sms);
                differs = true;
            } else if (f.bb.strategy == BN_STRATEGY_PRIVATE) {
                lean_smem = std::max(lean_smem, private_mesh_bytes(dtype, sum_mode,
                                                                   (int64_t)f.bb.band_rows * f.bb.g.ax[0].res, A,
                                                                   f.bb.st.do_sum, want_min, want_max));
            }
        }
        int use_lean = -1;
        {
            std::lock_guard<std::mutex> lk(cache.mu);
            auto it = cache.lean.find(key);
            if (it != cache.lean.end()) use_lean = it->second;
        }
        if (differs && use_lean < 0) {
            float t[2] = {-1.0f, -1.0f};
            for (int v = 0; v < 2; ++v) {
                std::vector<FastBlock>& fv = v ? lean : fbs;
                const size_t sm = v ? lean_smem : smem;
                cudaEvent_t e0 = nullptr, e1 = nullptr;
                bn_status st = BN_OK;
                if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
                    for (int rep = 0; rep < 2 && st == BN_OK; ++rep)  // builds, then warms the plan
                        st = launch_plan(c, cache, fv, dtype, A, ops, sum_mode, want_avg, sm);
                    if (st == BN_OK) cudaEventRecord(e0, c->stream);
                    if (st == BN_OK) st = launch_plan(c, cache, fv, dtype, A, ops, sum_mode, want_avg, sm);
                    if (st == BN_OK && cudaEventRecord(e1, c->stream) == cudaSuccess &&
                        cudaEventSynchronize(e1) == cudaSuccess)
                        cudaEventElapsedTime(&t[v], e0, e1);
                }
                if (e0) cudaEventDestroy(e0);
                if (e1) cudaEventDestroy(e1);
                if (st != BN_OK) return st;
            }
            use_lean = (t[1] >= 0.0f && t[1] < t[0]) ? 1 : 0;
            {
                // drop the slower plan's graph and memory (its last replay
                // has finished: the timed launch was waited for)
                const std::vector<int64_t> lose = plan_shape(use_lean ? fbs : lean, dtype, A, ops);
                std::lock_guard<std::mutex> lk(cache.mu);
                cache.lean[key] = use_lean;
                for (size_t g = 0; g < cache.graphs.size(); ++g)
                    if (cache.graphs[g]->shape == lose) {
                        cache.graphs.erase(cache.graphs.begin() + (long)g);
                        break;
                    }
            }
            char msg[160];
            snprintf(msg, sizeof msg, "batch of %d blocks: per-class plan=%.3fms sort-leaning plan=%.3fms -> %s",
                     n_blocks, t[0], t[1], use_lean ? "sort-leaning" : "per-class");
            std::lock_guard<std::mutex> lk2(c->tune_mu);
            c->tune_log.push_back(msg);
        }
        if (differs && use_lean == 1) {
            fbs.swap(lean);
            smem = lean_smem;
        }
    }
    (void)r;
    return launch_plan(c, cache, fbs, dtype, A, ops, sum_mode, want_avg, smem);
}

extern "C" bn_status bn_bin_batch(bn_context* c, const bn_block* blocks, int n_blocks,
                                  uint32_t ops, int sync, bn_request** req) {
    if (!c) return fail(BN_ERR_INVALID_ARG, "bn_bin_batch: NULL context");
    if (!sync && !req) return fail(BN_ERR_INVALID_ARG, "bn_bin_batch: asynchronous call needs req");
    if (n_blocks < 0 || (n_blocks > 0 && !blocks)) return fail(BN_ERR_INVALID_ARG, "bn_bin_batch: bad blocks");
    if (req) *req = nullptr;
    for (int k = 0; k < n_blocks; ++k) {
        if (!blocks[k].out) return fail(BN_ERR_INVALID_ARG, "bn_bin_batch: block %d has no outputs", k);
        if (blocks[k].n_attrs < 0 || blocks[k].n_attrs > BN_MAX_ATTR)
            return fail(BN_ERR_INVALID_ARG, "bn_bin_batch: block %d: bad n_attrs", k);
    }
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != c->device) cudaSetDevice(c->device);
    std::lock_guard<std::mutex> lk(c->enqueue_mu);
    bn_request* r = new_request(c);
    if (!r) return fail(BN_ERR_NO_MEMORY, "bn_bin_batch: no request slot");
    Plan plan(c);
    bn_status st = BN_OK;
    if (fast_eligible(c, blocks, n_blocks)) {
        st = batch_fast(c, blocks, n_blocks, ops, r, plan);
    } else {
        for (int k = 0; k < n_blocks && st == BN_OK; ++k) {
            const bn_block& b = blocks[k];
            st = enqueue_bin(c, plan, &b.x, &b.y, b.attrs, b.n_attrs, &b.grid, ops, b.out,
                             c->status_dev + r->slot);
        }
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
