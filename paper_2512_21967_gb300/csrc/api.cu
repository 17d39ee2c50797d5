// C ABI of the BLEST traversal library (declared in include/blest.h).  Host
// code: argument checks, the create pipeline (clean -> symmetry check ->
// reorder -> upload -> device BVSS build -> statistics), traversal launches and
// array export.  Every step of a traversal runs in the device kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "../../include/blest.h"
#include "bfs_launch.h"
#include "host_graph.h"
#include "msbfs_launch.h"

namespace blest {
constexpr int kCtrlBytes = 256;        // layout in device_common.cuh
constexpr int kCtrlClearBytes = 192;
// bitmaps of a handle's traversal state: 3 eager frontiers, V_curr, V_next
constexpr size_t kStateBitmaps = 5;
constexpr int kStickyWord = 48;
}  // namespace blest
using blest::kCtrlBytes;
using blest::kCtrlClearBytes;
using blest::kStateBitmaps;
using blest::kStickyWord;

using blest::Csr;

namespace {
thread_local std::string g_last_error;

blest_status fail(blest_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

blest_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? BLEST_ERR_OOM : BLEST_ERR_CUDA;
}

constexpr int kLevelRecordCap = 1 << 16;
constexpr int32_t kMaxVertices = 1 << 29;

}  // namespace

namespace blest {
// Lets other translation units of the library report through blest_last_error.
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace blest

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
}  // namespace

struct blest_graph {
    int32_t n = 0;
    int64_t nnz = 0;
    blest::DeviceBvss bvss;
    blest::DeviceCompact compact;        // compact layout, built on first use
    std::vector<int32_t> h_new_id;       // empty = identity
    int32_t* d_new_id = nullptr;
    int32_t* d_L = nullptr;              // internal levels (BVSS ids)
    int32_t* d_out = nullptr;            // staging for host-output calls (original ids)
    // [F0 F1 F2 | V_curr | V_next | dirty | control block] in one allocation, so that
    // one memset clears the bitmaps a traversal needs and the control block's counters
    unsigned char* d_state = nullptr;
    size_t bitmap_bytes = 0;             // each bitmap, rounded up to 256 B
    size_t dirty_bytes = 0;              // 1 bit per bitmap word, rounded up to 256 B
    uint32_t* d_vcur = nullptr;          // V_curr
    uint32_t* d_vnext = nullptr;         // V_next
    uint32_t* d_dirty = nullptr;
    uint32_t* d_F = nullptr;             // 3 bitmaps, bitmap_bytes apart (eager frontier)
    unsigned long long* d_Q = nullptr;   // 3 * qcap
    unsigned int qcap = 0;
    unsigned int* d_ctrl = nullptr;      // 256-byte control block (device_common.cuh layout)
    int32_t* d_level_sizes = nullptr;
    unsigned long long* d_level_times = nullptr;
    unsigned long long* d_arrive = nullptr;   // 4 * kLevelRecordCap: first (stage 1, sweep), then last
    int32_t* d_old_of = nullptr;         // BVSS id -> original id (direct level writes, parent output)
    int32_t* d_cand = nullptr;           // parent candidates (BVSS ids), made on first use
    int32_t* d_parents = nullptr;
    bool need_internal_levels = false;   // the next traversal must leave L cleared for unreached rows
    int32_t* d_roots = nullptr;
    int64_t roots_cap = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t last_stream = nullptr;
    int sms = 0;
    // options
    int update_opt = BLEST_UPDATE_AUTO;
    int pull = BLEST_PULL_POPC;
    int ms_pull = BLEST_PULL_POPC;       // multi-source pull back-end
    int ms_chunk = blest::kMsbfsChunk;   // sources per multi-source launch
    int ms_blocks_per_sm = 0;            // 0 = blocks_per_sm
    int ms_levels = 0;                   // BLEST_OPT_MS_LEVELS: 0 auto, 1 vertex-major, 2 bit planes
    int ms_filter = 2;                   // BLEST_OPT_MS_VISITED_FILTER
    // sharded traversal in progress (blest_shard_*): rank, ranks, next level, output, rows reached
    int32_t shard_rank = -1, shard_world = 0, shard_level = 0;
    int32_t* shard_out = nullptr;
    unsigned int shard_reached = 0;
    int blocks_per_sm = 0;
    int64_t timeout_us = 2000000;
    int record = 0;
    int unroll = 2;
    int minb = 2;
    // defaults: the variant the autotuner picks on social-like graphs (lazy levels);
    // eager levels ignore the lazy-only ones
    int filter = 4;
    int depth = 2;
    int layout = 0;
    int sched = 1;
    int phantom = 0;
    // results
    blest_stats stats{};
    blest_run_info info{};
    std::vector<int64_t> offsets;        // batch handles: graph g owns [offsets[g], offsets[g+1])
    blest::MsbfsState ms;
    // captured batch traversal (blest_batch_graph_capture)
    cudaGraph_t cgraph = nullptr;
    cudaGraphExec_t cgraph_exec = nullptr;
    int32_t* d_graph_roots = nullptr;
    int32_t* h_graph_roots = nullptr;    // pinned
    int32_t graph_nroots = 0;
    cudaEvent_t graph_done = nullptr;

    int nwords() const { return (n + 31) / 32; }
    int resolved_update() const {
        if (update_opt == BLEST_UPDATE_EAGER || update_opt == BLEST_UPDATE_LAZY) return update_opt;
        return stats.update;
    }
    // multi-source level layout: 1 = bit planes, 0 = vertex-major; AUTO takes planes
    // on graphs the Section 5 rule updates lazily (U_div > 25,000: low diameter,
    // where a vertex gains bits at few distinct levels)
    int ms_levels_layout() const {
        if (ms_levels == 1) return 0;
        if (ms_levels == 2) return 1;
        return stats.update == BLEST_UPDATE_LAZY ? 1 : 0;
    }
};

namespace {

void free_handle(blest_graph* h) {
    blest::free_compact_device(h->compact);
    if (!h) return;
    blest::free_bvss_device(h->bvss);
    blest::free_msbfs_state(h->ms);
    cudaFree(h->d_new_id);
    cudaFree(h->d_L);
    cudaFree(h->d_out);
    cudaFree(h->d_state);
    cudaFree(h->d_Q);
    cudaFree(h->d_level_sizes);
    cudaFree(h->d_level_times);
    cudaFree(h->d_arrive);
    cudaFree(h->d_old_of);
    cudaFree(h->d_cand);
    cudaFree(h->d_parents);
    cudaFree(h->d_roots);
    if (h->cgraph_exec) cudaGraphExecDestroy(h->cgraph_exec);
    if (h->cgraph) cudaGraphDestroy(h->cgraph);
    cudaFree(h->d_graph_roots);
    if (h->h_graph_roots) cudaFreeHost(h->h_graph_roots);
    if (h->graph_done) cudaEventDestroy(h->graph_done);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// Device part of create: upload the relabelled CSR, build BVSS, allocate state.
blest_status init_device(blest_graph* h) {
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e, "cudaDeviceGetAttribute");
    if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    return BLEST_OK;
}

// Traversal state of a handle whose BVSS is on the device, and the vertex order.
blest_status alloc_state(blest_graph* h, const std::vector<int32_t>& new_id) {
    cudaError_t e;
    const size_t nw = (size_t)h->nwords();
    h->qcap = (unsigned int)std::max<int64_t>(h->bvss.nvss, 1);
#define BLEST_ALLOC(ptr, bytes, what) \
    if ((e = cudaMalloc(&(ptr), (bytes))) != cudaSuccess) return cuda_fail(e, what);
    BLEST_ALLOC(h->d_L, sizeof(int32_t) * std::max<size_t>(h->n, 1), "cudaMalloc(levels)");
    BLEST_ALLOC(h->d_out, sizeof(int32_t) * std::max<size_t>(h->n, 1), "cudaMalloc(out)");
    h->bitmap_bytes = (sizeof(uint32_t) * std::max<size_t>(nw, 1) + 255) / 256 * 256;
    h->dirty_bytes = (sizeof(uint32_t) * ((std::max<size_t>(nw, 1) + 31) / 32) + 255) / 256 * 256;
    BLEST_ALLOC(h->d_state, kStateBitmaps * h->bitmap_bytes + h->dirty_bytes + kCtrlBytes, "cudaMalloc(bitmaps)");
    h->d_F = reinterpret_cast<uint32_t*>(h->d_state);
    h->d_vcur = reinterpret_cast<uint32_t*>(h->d_state + 3 * h->bitmap_bytes);
    h->d_vnext = reinterpret_cast<uint32_t*>(h->d_state + 4 * h->bitmap_bytes);
    h->d_dirty = reinterpret_cast<uint32_t*>(h->d_state + kStateBitmaps * h->bitmap_bytes);
    h->d_ctrl = reinterpret_cast<unsigned int*>(h->d_state + kStateBitmaps * h->bitmap_bytes + h->dirty_bytes);
    BLEST_ALLOC(h->d_Q, sizeof(unsigned long long) * 3 * (size_t)h->qcap, "cudaMalloc(queues)");
    BLEST_ALLOC(h->d_level_sizes, sizeof(int32_t) * kLevelRecordCap, "cudaMalloc(level record)");
    BLEST_ALLOC(h->d_level_times, sizeof(unsigned long long) * (2 * (size_t)kLevelRecordCap + 2), "cudaMalloc(level times)");
    BLEST_ALLOC(h->d_arrive, sizeof(unsigned long long) * 4 * (size_t)kLevelRecordCap, "cudaMalloc(level arrivals)");
#undef BLEST_ALLOC
    cudaMemsetAsync(h->d_ctrl, 0, kCtrlBytes, h->stream);
    if (!new_id.empty()) {
        h->h_new_id = new_id;
        std::vector<int32_t> old_of((size_t)h->n);
        for (int32_t v = 0; v < h->n; ++v) old_of[(size_t)new_id[(size_t)v]] = v;
        if ((e = cudaMalloc(&h->d_new_id, sizeof(int32_t) * (size_t)h->n)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(new_id)");
        if ((e = cudaMalloc(&h->d_old_of, sizeof(int32_t) * (size_t)h->n)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(old_of)");
        cudaMemcpyAsync(h->d_new_id, new_id.data(), sizeof(int32_t) * (size_t)h->n, cudaMemcpyHostToDevice, h->stream);
        cudaMemcpyAsync(h->d_old_of, old_of.data(), sizeof(int32_t) * (size_t)h->n, cudaMemcpyHostToDevice, h->stream);
        // the host copy must live until the upload is done
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e, "upload order");
    }
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e, "create");
    return BLEST_OK;
}

blest_status finish_create(blest_graph* h, const Csr& g, const std::vector<int32_t>& new_id, double t_order) {
    double t0 = now_s();
    cudaError_t e;
    blest_status bs = init_device(h);
    if (bs) return bs;
    h->n = g.n;
    h->nnz = g.nnz();
    int32_t *d_rp = nullptr, *d_ci = nullptr;
    if ((e = cudaMalloc(&d_rp, sizeof(int32_t) * ((size_t)g.n + 1))) != cudaSuccess) return cuda_fail(e, "cudaMalloc(row_ptr)");
    if ((e = cudaMalloc(&d_ci, sizeof(int32_t) * (size_t)std::max<int64_t>(h->nnz, 1))) != cudaSuccess) {
        cudaFree(d_rp);
        return cuda_fail(e, "cudaMalloc(col_idx)");
    }
    cudaMemcpyAsync(d_rp, g.rp.data(), sizeof(int32_t) * ((size_t)g.n + 1), cudaMemcpyHostToDevice, h->stream);
    if (h->nnz) cudaMemcpyAsync(d_ci, g.ci.data(), sizeof(int32_t) * (size_t)h->nnz, cudaMemcpyHostToDevice, h->stream);
    const char* err = nullptr;
    int rc = blest::build_bvss_device(d_rp, d_ci, g.n, h->nnz, h->stream, h->bvss, &err);
    cudaFree(d_rp);
    cudaFree(d_ci);
    if (rc) return fail((blest_status)rc, std::string("BVSS build: ") + (err ? err : "?"));
    if (h->bvss.nvss >= (int64_t)1 << 31) return fail(BLEST_ERR_TOO_LARGE, "more than 2^31 virtual slice sets");
    double udiv = 0.0;
    rc = blest::update_divergence_device(h->bvss, h->stream, &udiv, &err);
    if (rc) return fail((blest_status)rc, std::string("update divergence: ") + (err ? err : "?"));
    if ((bs = alloc_state(h, new_id)) != BLEST_OK) return bs;

    const size_t nw = (size_t)h->nwords();
    blest_stats& s = h->stats;
    s.n = g.n;
    s.nnz = h->nnz;
    s.num_slice_sets = h->bvss.nss;
    s.num_vss = h->bvss.nvss;
    s.num_slices = 128 * h->bvss.nvss;
    s.unpadded_slices = h->bvss.unpadded;
    s.connectivity_bits = 8 * h->bvss.unpadded;
    s.update_divergence = udiv;
    s.compression_ratio = h->bvss.unpadded ? (double)h->nnz / (double)(8 * h->bvss.unpadded) : 0.0;
    s.bvss_bytes = (int64_t)h->bvss.nvss * (128 * 4 + 32 * 4 + 4 + 4) + ((int64_t)h->bvss.nss + 1) * 4;
    s.state_bytes = (int64_t)g.n * 8 + (int64_t)nw * 4 * 5 + (int64_t)h->qcap * 24 + 128 + kLevelRecordCap * 4;
    s.update = udiv > 25000.0 ? BLEST_UPDATE_LAZY : BLEST_UPDATE_EAGER;
    s.order_seconds = t_order;
    s.build_seconds += now_s() - t0;
    return BLEST_OK;
}

blest_status prepare_graph(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, blest_order order,
                           const blest_create_params* params, int threads, Csr& clean, std::vector<int32_t>& new_id,
                           int32_t* order_used, double* t_order, double* t_clean) {
    if (order < BLEST_ORDER_NONE || order > BLEST_ORDER_AUTO) return fail(BLEST_ERR_INVALID_ARG, "unknown order");
    if (n < 0) return fail(BLEST_ERR_INVALID_ARG, "n must be >= 0");
    if (n > kMaxVertices) return fail(BLEST_ERR_TOO_LARGE, "more than 2^29 vertices");
    int32_t window = params && params->window > 0 ? params->window : 65536;
    if (window % 8 != 0) return fail(BLEST_ERR_INVALID_ARG, "window must be a multiple of 8");
    double t0 = now_s();
    std::string err;
    int rc = blest::clean_csr(n, row_ptr, col_idx, threads, clean, err);
    if (rc) return fail((blest_status)rc, err);
    if (!(params && params->skip_symmetry_check)) {
        int64_t bu = -1, bv = -1;
        if (!blest::is_symmetric(clean, threads, &bu, &bv))
            return fail(BLEST_ERR_NOT_SYMMETRIC, "edge (" + std::to_string(bu) + ", " + std::to_string(bv) +
                                                     ") has no reverse edge");
    }
    *t_clean = now_s() - t0;
    t0 = now_s();
    int32_t ord = order;
    if (ord == BLEST_ORDER_AUTO) ord = blest::is_social_like(clean) ? BLEST_ORDER_COMPRESS : BLEST_ORDER_BANDWIDTH;
    new_id.clear();
    if (ord == BLEST_ORDER_COMPRESS)
        blest::order_compress(clean, 8, window, threads, new_id, params && params->prepass == 1 ? 1 : 0);
    else if (ord == BLEST_ORDER_BANDWIDTH) blest::order_rcm(clean, new_id, threads);
    *order_used = ord;
    *t_order = now_s() - t0;
    return BLEST_OK;
}

// The compact layout is derived from the padded BVSS the first time it is asked for.
blest_status ensure_compact(blest_graph* h) {
    if (h->compact.goff || h->bvss.nss == 0) return BLEST_OK;
    const char* err = nullptr;
    const int rc = blest::build_compact_device(h->bvss, h->stream, h->compact, &err);
    if (rc) return fail((blest_status)rc, err ? err : "compact layout build failed");
    return BLEST_OK;
}

int pick_grid(blest_graph* h, int update, int pull, int unroll, int minb, int depth, int layout) {
    int maxb = blest::bfs_max_blocks_per_sm(update, pull, unroll, minb, depth, layout);
    if (maxb <= 0) return 0;
    int b = h->blocks_per_sm > 0 ? std::min(h->blocks_per_sm, maxb) : maxb;
    return b * h->sms;
}

// Enqueue one single-frontier traversal from the (BVSS-order) roots, writing
// levels in original ids into d_out (device, n int32).
blest_status enqueue_traversal(blest_graph* h, const std::vector<int32_t>& roots, int32_t* d_out, cudaStream_t st,
                               const int32_t* d_roots_preloaded = nullptr, int32_t n_preloaded = 0) {
    if (h->n == 0) return BLEST_OK;
    cudaError_t e;
    blest::BfsLaunch L;
    L.update = h->resolved_update() == BLEST_UPDATE_EAGER ? 1 : 2;
    L.pull = h->pull;
    L.unroll = h->unroll;
    L.minb = h->minb;
    L.filter = h->filter;
    if (L.update == 1 && L.filter >= 2) L.filter = 1;     // V_next is not used by the eager update
    L.sched = h->sched;
    // the TMA ring exists for the lazy kernel compiled for 2 blocks per SM
    L.depth = (L.update == 2 && L.minb == 2) ? h->depth : 0;
    if (L.depth == 0 && L.unroll > 2) L.unroll = 2;       // unroll 4 exists only for the TMA ring
    if (L.depth == 4 && L.unroll > 2) L.unroll = 2;       // a 4-stage ring holds two groups of 2
    if ((L.depth == 2 || L.depth == 3) && L.unroll > 2) L.unroll = 2;   // the register pipelines exist for 1 and 2
    // the compact layout serves the lazy register paths (depth 0 or 2) at 2 blocks per SM
    L.layout = (h->layout == 1 && L.update == 2 && L.minb == 2 && (L.depth == 0 || L.depth == 2) && h->compact.goff) ? 1 : 0;
    L.grid = pick_grid(h, L.update, L.pull, L.unroll, L.minb, L.depth, L.layout);
    if (L.grid <= 0) return fail(BLEST_ERR_CUDA, "no co-resident grid for the traversal kernel");
    L.n = h->n;
    L.qcap = h->qcap;
    L.real_ptrs = h->bvss.real_ptrs;
    L.row_ids = h->bvss.row_ids;
    L.masks = h->bvss.masks;
    L.goff = h->compact.goff;
    L.rows_c = h->compact.rows;
    L.masks_c = h->compact.masks;
    L.new_id = h->d_new_id;
    L.levels_internal = h->d_new_id ? h->d_L : d_out;
    // a lazy traversal with a reordering writes levels straight to out (cleared to
    // -1 before the launch) and needs no unpermute; the parent pass needs L
    L.direct = (L.update == 2 && h->d_new_id && h->d_old_of && !h->need_internal_levels) ? 1 : 0;
    L.old_of = h->d_old_of;
    L.vcur = h->d_vcur;
    L.vnext = h->d_vnext;
    L.dirty = h->d_dirty;
    for (int i = 0; i < 3; ++i) {
        L.F[i] = reinterpret_cast<uint32_t*>(h->d_state + i * h->bitmap_bytes);
        L.Q[i] = h->d_Q + i * (size_t)h->qcap;
    }
    L.ctrl = h->d_ctrl;
    L.level_sizes = h->record ? h->d_level_sizes : nullptr;
    L.level_times = h->d_level_times;
    L.arrive_first = h->d_arrive;
    L.arrive_last = h->d_arrive + 2 * kLevelRecordCap;
    L.level_cap = kLevelRecordCap;
    L.nroots = (int32_t)roots.size();
    if (d_roots_preloaded) {
        // roots already on the device (a captured launch reads them from there)
        L.nroots = n_preloaded;
        L.roots_device = d_roots_preloaded;
    } else if (roots.size() > (size_t)blest::kInlineRoots) {
        if ((int64_t)roots.size() > h->roots_cap) {
            cudaFree(h->d_roots);
            h->d_roots = nullptr;
            h->roots_cap = 0;
            if ((e = cudaMalloc(&h->d_roots, sizeof(int32_t) * roots.size())) != cudaSuccess) return cuda_fail(e, "cudaMalloc(roots)");
            h->roots_cap = (int64_t)roots.size();
        }
        if ((e = cudaMemcpyAsync(h->d_roots, roots.data(), sizeof(int32_t) * roots.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "copy roots");
        L.roots_device = h->d_roots;
    } else {
        for (size_t i = 0; i < roots.size(); ++i) L.roots_host[i] = roots[i];
    }
    if (d_roots_preloaded && n_preloaded <= blest::kInlineRoots) {
        // the kernel takes inline roots below kInlineRoots; a captured launch must read the device list
        return fail(BLEST_ERR_INTERNAL, "device roots need more than the inline count");
    }
    L.out = d_out;
    L.timeout_ns = (uint64_t)h->timeout_us * 1000ull;
    L.phantom = h->phantom ? 1u : 0u;
    // [F (eager only) | V_curr | V_next | dirty | control block up to the sticky status word]
    const size_t skip = L.update == 1 ? 0 : 3 * h->bitmap_bytes;
    cudaMemsetAsync(h->d_state + skip, 0, kStateBitmaps * h->bitmap_bytes + h->dirty_bytes - skip + kCtrlClearBytes, st);
    cudaMemsetAsync(L.direct ? d_out : L.levels_internal, 0xFF, sizeof(int32_t) * (size_t)h->n, st);
    if (L.level_sizes) {
        cudaMemsetAsync(L.arrive_first, 0xFF, sizeof(unsigned long long) * 2 * kLevelRecordCap, st);
        cudaMemsetAsync(L.arrive_last, 0, sizeof(unsigned long long) * 2 * kLevelRecordCap, st);
    }
    if ((e = blest::launch_bfs_kernel(L, st)) != cudaSuccess) return cuda_fail(e, "traversal launch");
    h->last_stream = st;
    h->info.update = L.update == 1 ? BLEST_UPDATE_EAGER : BLEST_UPDATE_LAZY;
    h->info.pull = L.pull;
    h->info.grid_blocks = L.grid;
    h->info.threads_per_block = blest::bfs_threads_per_block();
    h->info.recorded = -1;  // resolved in blest_get_run_info
    h->info.output_path = !h->d_new_id ? 0 : (L.direct ? 1 : 2);
    return BLEST_OK;
}

// Launch description of one step of a sharded traversal (lazy update, padded
// layout, register double buffer, 2 blocks per SM; the steps are separate launches).
blest::BfsLaunch shard_launch(blest_graph* h) {
    blest::BfsLaunch L;
    L.update = 2;
    L.filter = h->filter;
    L.depth = 2;
    L.n = h->n;
    L.qcap = h->qcap;
    L.real_ptrs = h->bvss.real_ptrs;
    L.row_ids = h->bvss.row_ids;
    L.masks = h->bvss.masks;
    L.new_id = h->d_new_id;
    L.direct = h->d_new_id && h->d_old_of ? 1 : 0;
    L.old_of = h->d_old_of;
    L.levels_internal = h->d_new_id ? h->d_L : h->shard_out;
    L.out = h->shard_out;
    L.vcur = h->d_vcur;
    L.vnext = h->d_vnext;
    for (int i = 0; i < 3; ++i) {
        L.F[i] = reinterpret_cast<uint32_t*>(h->d_state + i * h->bitmap_bytes);
        L.Q[i] = h->d_Q + i * (size_t)h->qcap;
    }
    L.ctrl = h->d_ctrl;
    L.timeout_ns = (uint64_t)h->timeout_us * 1000ull;
    L.grid = 2 * h->sms;
    return L;
}

blest_status map_sources(blest_graph* h, const int32_t* srcs, int32_t k, std::vector<int32_t>& roots) {
    roots.resize((size_t)k);
    for (int32_t i = 0; i < k; ++i) {
        int32_t s = srcs[i];
        if (s < 0 || s >= h->n) return fail(BLEST_ERR_INVALID_ARG, "source " + std::to_string(s) + " outside [0, n)");
        roots[i] = h->h_new_id.empty() ? s : h->h_new_id[s];
    }
    return BLEST_OK;
}

blest_status sync_status(blest_graph* h) {
    cudaError_t e;
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if (h->last_stream && h->last_stream != h->stream)
        if ((e = cudaStreamSynchronize(h->last_stream)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if (!h->d_ctrl) return BLEST_OK;
    unsigned int sticky = 0;
    if ((e = cudaMemcpy(&sticky, h->d_ctrl + kStickyWord, sizeof(unsigned int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "read status");
    if (sticky) {
        cudaMemset(h->d_ctrl + kStickyWord, 0, sizeof(unsigned int));
        if (sticky == BLEST_ERR_TIMEOUT) return fail(BLEST_ERR_TIMEOUT, "a grid barrier timed out");
        if (sticky == BLEST_ERR_INTERNAL) return fail(BLEST_ERR_INTERNAL, "device-side consistency check failed");
        return fail((blest_status)sticky, "device error");
    }
    return BLEST_OK;
}

}  // namespace

namespace blest {
cudaError_t launch_distance_stats(const int32_t* lv, int32_t k, int64_t n, unsigned long long* acc, int* ecc,
                                  cudaStream_t st);   // stats.cu
cudaError_t launch_parents(const int32_t* v2r, const int32_t* row_ids, const uint32_t* masks, int64_t nvss,
                           const int32_t* L, const int32_t* old_of, const int32_t* new_id, int32_t n, int32_t* cand,
                           int32_t* out, cudaStream_t st);   // parents.cu
// Read-only view of a handle's device arrays for the query server (server.cu).
struct HandleView {
    int32_t n;
    int32_t nss;
    int64_t nvss;
    const int32_t* real_ptrs;
    const int32_t* row_ids;
    const uint32_t* masks;
    const int32_t* new_id_dev;
    const int32_t* new_id_host;
    int sms;
    int levels_layout;
};
bool handle_view(blest_handle h, HandleView* v) {
    if (!h || !v || h->n == 0) return false;
    v->n = h->n;
    v->nss = h->bvss.nss;
    v->nvss = h->bvss.nvss;
    v->real_ptrs = h->bvss.real_ptrs;
    v->row_ids = h->bvss.row_ids;
    v->masks = h->bvss.masks;
    v->new_id_dev = h->d_new_id;
    v->new_id_host = h->h_new_id.empty() ? nullptr : h->h_new_id.data();
    v->sms = h->sms;
    v->levels_layout = h->ms_levels_layout();
    return true;
}
}  // namespace blest

// ---------------------------------------------------------------- checkpoint helpers

namespace {

struct CheckpointHeader {
    char magic[8];          // "BLESTG1"
    int32_t version;        // 1
    int32_t n;
    int64_t nnz;
    int32_t nss;
    int32_t has_new_id;
    int64_t nvss;
    int64_t unpadded;
    int64_t num_offsets;    // batch handles: graph boundaries (0 for a single graph)
};

template <class T>
bool write_all(FILE* f, const T* p, size_t count) {
    return count == 0 || std::fwrite(p, sizeof(T), count, f) == count;
}

template <class T>
bool read_all(FILE* f, T* p, size_t count) {
    return count == 0 || std::fread(p, sizeof(T), count, f) == count;
}

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src, size_t at_least, cudaStream_t st) {
    cudaError_t e = cudaMalloc(dst, sizeof(T) * std::max(src.size(), at_least));
    if (e == cudaSuccess && !src.empty())
        e = cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, st);
    return e;
}

}  // namespace

extern "C" {

const char* blest_status_string(blest_status s) {
    switch (s) {
        case BLEST_OK: return "BLEST_OK";
        case BLEST_ERR_INVALID_ARG: return "BLEST_ERR_INVALID_ARG";
        case BLEST_ERR_NOT_SYMMETRIC: return "BLEST_ERR_NOT_SYMMETRIC";
        case BLEST_ERR_TOO_LARGE: return "BLEST_ERR_TOO_LARGE";
        case BLEST_ERR_OOM: return "BLEST_ERR_OOM";
        case BLEST_ERR_CUDA: return "BLEST_ERR_CUDA";
        case BLEST_ERR_TIMEOUT: return "BLEST_ERR_TIMEOUT";
        case BLEST_ERR_INTERNAL: return "BLEST_ERR_INTERNAL";
    }
    return "BLEST_ERR_UNKNOWN";
}

const char* blest_last_error(void) { return g_last_error.c_str(); }

blest_status blest_graph_create_ex(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, blest_order order,
                                   const blest_create_params* params, blest_handle* out) {
    if (!out) return fail(BLEST_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    const int threads = blest::host_threads(params ? params->threads : 0);
    Csr clean;
    std::vector<int32_t> new_id;
    int32_t used = order;
    double t_order = 0, t_clean = 0;
    blest_status s = prepare_graph(n, row_ptr, col_idx, order, params, threads, clean, new_id, &used, &t_order, &t_clean);
    if (s) return s;
    std::unique_ptr<blest_graph, void (*)(blest_graph*)> h(new blest_graph(), free_handle);
    Csr relabelled;
    const Csr* g = &clean;
    if (!new_id.empty()) {
        double t0 = now_s();
        blest::relabel_csr(clean, new_id, threads, relabelled);
        t_clean += now_s() - t0;
        g = &relabelled;
    }
    h->stats.build_seconds = t_clean;
    s = finish_create(h.get(), *g, new_id, t_order);
    if (s) return s;
    h->stats.order = used;
    *out = h.release();
    return BLEST_OK;
}

// ---------------------------------------------------------------- checkpoint

blest_status blest_graph_save(blest_handle h, const char* path) {
    if (!h || !path) return fail(BLEST_ERR_INVALID_ARG, "NULL argument");
    blest_status s = sync_status(h);
    if (s) return s;
    const blest::DeviceBvss& b = h->bvss;
    std::vector<int32_t> rp((size_t)b.nss + 1), v2r((size_t)b.nvss), rows(128 * (size_t)b.nvss), cnt((size_t)b.nvss);
    std::vector<uint32_t> masks(32 * (size_t)b.nvss);
    cudaError_t e = cudaSuccess;
    if (b.real_ptrs) e = cudaMemcpy(rp.data(), b.real_ptrs, 4 * rp.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && b.nvss > 0) {
        if ((e = cudaMemcpy(v2r.data(), b.v2r, 4 * v2r.size(), cudaMemcpyDeviceToHost)) == cudaSuccess &&
            (e = cudaMemcpy(rows.data(), b.row_ids, 4 * rows.size(), cudaMemcpyDeviceToHost)) == cudaSuccess &&
            (e = cudaMemcpy(masks.data(), b.masks, 4 * masks.size(), cudaMemcpyDeviceToHost)) == cudaSuccess)
            e = cudaMemcpy(cnt.data(), b.vss_count, 4 * cnt.size(), cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return cuda_fail(e, "read BVSS for saving");
    CheckpointHeader hd{};
    std::memcpy(hd.magic, "BLESTG1", 8);
    hd.version = 1;
    hd.n = h->n;
    hd.nnz = h->nnz;
    hd.nss = b.nss;
    hd.has_new_id = h->h_new_id.empty() ? 0 : 1;
    hd.nvss = b.nvss;
    hd.unpadded = b.unpadded;
    hd.num_offsets = (int64_t)h->offsets.size();
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(BLEST_ERR_INVALID_ARG, std::string("cannot open ") + path + " for writing");
    bool ok = write_all(f, &hd, 1) && write_all(f, &h->stats, 1) &&
              write_all(f, h->offsets.data(), h->offsets.size()) &&
              write_all(f, h->h_new_id.data(), h->h_new_id.size()) && write_all(f, rp.data(), rp.size()) &&
              write_all(f, v2r.data(), v2r.size()) && write_all(f, rows.data(), rows.size()) &&
              write_all(f, masks.data(), masks.size()) && write_all(f, cnt.data(), cnt.size());
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(BLEST_ERR_INVALID_ARG, std::string("short write to ") + path);
    return BLEST_OK;
}

blest_status blest_graph_load(const char* path, blest_handle* out) {
    if (!out || !path) return fail(BLEST_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(BLEST_ERR_INVALID_ARG, std::string("cannot open ") + path);
    std::unique_ptr<FILE, int (*)(FILE*)> closer(f, std::fclose);
    CheckpointHeader hd{};
    blest_stats st{};
    if (!read_all(f, &hd, 1) || std::memcmp(hd.magic, "BLESTG1", 8) != 0 || hd.version != 1)
        return fail(BLEST_ERR_INVALID_ARG, "not a version-1 BLEST graph file");
    if (hd.n < 0 || hd.n > kMaxVertices || hd.nss != (hd.n + 7) / 8 || hd.nnz < 0 || hd.nnz >= ((int64_t)1 << 31) ||
        hd.nvss < 0 || hd.nvss >= ((int64_t)1 << 31) || hd.unpadded < 0 || hd.unpadded > 128 * hd.nvss ||
        hd.num_offsets < 0 || hd.num_offsets > (int64_t)hd.n + 2 || (hd.has_new_id != 0 && hd.has_new_id != 1))
        return fail(BLEST_ERR_INVALID_ARG, "inconsistent sizes in the file header");
    const size_t n = (size_t)hd.n, nss = (size_t)hd.nss, nvss = (size_t)hd.nvss;
    std::vector<int64_t> offsets((size_t)hd.num_offsets);
    std::vector<int32_t> new_id(hd.has_new_id ? n : 0), rp(nss + 1), v2r(nvss), rows(128 * nvss), cnt(nvss);
    std::vector<uint32_t> masks(32 * nvss);
    if (!read_all(f, &st, 1) || !read_all(f, offsets.data(), offsets.size()) ||
        !read_all(f, new_id.data(), new_id.size()) || !read_all(f, rp.data(), rp.size()) ||
        !read_all(f, v2r.data(), v2r.size()) || !read_all(f, rows.data(), rows.size()) ||
        !read_all(f, masks.data(), masks.size()) || !read_all(f, cnt.data(), cnt.size()))
        return fail(BLEST_ERR_INVALID_ARG, "the file is shorter than its header says");
    // every index the kernels follow is checked before anything reaches the device
    if (!new_id.empty()) {
        std::vector<char> seen(n, 0);
        for (int32_t v : new_id) {
            if (v < 0 || (size_t)v >= n || seen[(size_t)v]) return fail(BLEST_ERR_INVALID_ARG, "new_id is not a permutation");
            seen[(size_t)v] = 1;
        }
    }
    if (!offsets.empty()) {
        if (offsets.front() != 0 || offsets.back() != hd.n) return fail(BLEST_ERR_INVALID_ARG, "bad graph offsets");
        for (size_t i = 1; i < offsets.size(); ++i)
            if (offsets[i] < offsets[i - 1]) return fail(BLEST_ERR_INVALID_ARG, "bad graph offsets");
    }
    if (rp[0] != 0 || (int64_t)rp[nss] != hd.nvss) return fail(BLEST_ERR_INVALID_ARG, "bad realPtrs");
    int64_t unpadded = 0;
    for (size_t sidx = 0; sidx < nss; ++sidx) {
        if (rp[sidx + 1] < rp[sidx]) return fail(BLEST_ERR_INVALID_ARG, "realPtrs not monotone");
        const uint32_t colmask = (8 * sidx + 8 <= n) ? 0xFFu : ((1u << (n - 8 * sidx)) - 1u);   // columns < n
        for (int64_t nu = rp[sidx]; nu < rp[sidx + 1]; ++nu) {
            const int c = cnt[(size_t)nu];
            const bool last = nu + 1 == rp[sidx + 1];
            if (v2r[(size_t)nu] != (int32_t)sidx || c < 1 || c > 128 || (!last && c != 128))
                return fail(BLEST_ERR_INVALID_ARG, "bad virtualToReal or VSS count");
            unpadded += c;
            for (int k = 0; k < 128; ++k) {
                const int lane = k & 31, sub = k >> 5;
                const int32_t u = rows[(size_t)nu * 128 + 4 * lane + sub];
                const uint32_t m = (masks[(size_t)nu * 32 + lane] >> (8 * sub)) & 0xFFu;
                if (u < 0 || (size_t)u >= n) return fail(BLEST_ERR_INVALID_ARG, "row id out of range");
                if ((k < c && m == 0) || (k >= c && m != 0) || (m & ~colmask))
                    return fail(BLEST_ERR_INVALID_ARG, "mask inconsistent with the VSS count or the columns");
            }
        }
    }
    if (unpadded != hd.unpadded) return fail(BLEST_ERR_INVALID_ARG, "unpadded slice count mismatch");

    std::unique_ptr<blest_graph, void (*)(blest_graph*)> h(new blest_graph(), free_handle);
    blest_status bs = init_device(h.get());
    if (bs) return bs;
    h->n = hd.n;
    h->nnz = hd.nnz;
    h->offsets = offsets;
    blest::DeviceBvss& b = h->bvss;
    b.n = hd.n;
    b.nss = hd.nss;
    b.nvss = hd.nvss;
    b.unpadded = hd.unpadded;
    cudaError_t e;
    if ((e = upload(&b.real_ptrs, rp, 1, h->stream)) != cudaSuccess || (e = upload(&b.v2r, v2r, 1, h->stream)) != cudaSuccess ||
        (e = upload(&b.row_ids, rows, 1, h->stream)) != cudaSuccess || (e = upload(&b.masks, masks, 1, h->stream)) != cudaSuccess ||
        (e = upload(&b.vss_count, cnt, 1, h->stream)) != cudaSuccess)
        return cuda_fail(e, "upload BVSS");
    if ((bs = alloc_state(h.get(), new_id)) != BLEST_OK) return bs;
    h->stats = st;
    *out = h.release();
    return BLEST_OK;
}

blest_status blest_graph_create(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, blest_order order,
                                blest_handle* out) {
    return blest_graph_create_ex(n, row_ptr, col_idx, order, nullptr, out);
}

blest_status blest_batch_create(int32_t num_graphs, const int32_t* n_each, const int32_t* const* row_ptrs,
                                const int32_t* const* col_idxs, const int32_t* orders,
                                const blest_create_params* params, blest_handle* out) {
    if (!out) return fail(BLEST_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (num_graphs < 0 || (num_graphs > 0 && (!n_each || !row_ptrs || !col_idxs || !orders)))
        return fail(BLEST_ERR_INVALID_ARG, "bad batch description");
    const int threads = blest::host_threads(params ? params->threads : 0);
    std::vector<int64_t> offsets(1, 0);
    for (int32_t g = 0; g < num_graphs; ++g) {
        if (n_each[g] < 0) return fail(BLEST_ERR_INVALID_ARG, "graph with n < 0");
        offsets.push_back(offsets.back() + n_each[g]);
    }
    if (offsets.back() > kMaxVertices) return fail(BLEST_ERR_TOO_LARGE, "more than 2^29 vertices in the batch");
    const int32_t N = (int32_t)offsets.back();
    Csr uni;
    uni.n = N;
    uni.rp.assign((size_t)N + 1, 0);
    std::vector<int32_t> new_id((size_t)N);
    std::vector<Csr> parts((size_t)num_graphs);
    std::vector<std::vector<int32_t>> ids((size_t)num_graphs);
    // Graphs are cleaned, checked, reordered and relabelled on the host threads:
    // a graph holding more than an even share of the batch's entries alone with
    // all threads, the others concurrently with one thread each, largest first.
    // An order does not depend on the thread count, so neither does the handle.
    // The first failing graph (by index) is reported.
    std::vector<blest_status> status((size_t)num_graphs, BLEST_OK);
    std::vector<std::string> errors((size_t)num_graphs);
    std::vector<int32_t> by_size((size_t)num_graphs);
    for (int32_t g = 0; g < num_graphs; ++g) by_size[(size_t)g] = g;
    auto entries = [&](int32_t g) -> int64_t { return n_each[g] > 0 && row_ptrs[g] ? row_ptrs[g][n_each[g]] : 0; };
    std::stable_sort(by_size.begin(), by_size.end(), [&](int32_t a, int32_t b) { return entries(a) > entries(b); });
    const int workers = std::max(1, std::min(threads, num_graphs));
    auto prepare_one = [&](int32_t g, int inner) {
        // runs on worker threads: an exception escaping here would terminate the process,
        // so a failed host allocation becomes this graph's error status
        try {
            int32_t used = 0;
            double to = 0, tc = 0;
            Csr clean;
            blest_status s = prepare_graph(n_each[g], row_ptrs[g], col_idxs[g], (blest_order)orders[g], params,
                                           inner, clean, ids[(size_t)g], &used, &to, &tc);
            if (s) {
                status[(size_t)g] = s;
                errors[(size_t)g] = g_last_error;   // this thread's own message
                return;
            }
            if (!ids[(size_t)g].empty()) blest::relabel_csr(clean, ids[(size_t)g], inner, parts[(size_t)g]);
            else parts[(size_t)g] = std::move(clean);
        } catch (const std::bad_alloc&) {
            status[(size_t)g] = BLEST_ERR_OOM;
            errors[(size_t)g] = "host memory exhausted while preparing the graph";
        } catch (const std::exception& ex) {
            status[(size_t)g] = BLEST_ERR_INTERNAL;
            errors[(size_t)g] = std::string("host preparation failed: ") + ex.what();
        }
    };
    const double t0 = now_s();
    // graphs above an even share of the batch's entries take all threads, one at a time
    int64_t all_entries = 0;
    for (int32_t g = 0; g < num_graphs; ++g) all_entries += entries(g);
    int32_t first_small = 0;
    while (first_small < num_graphs && workers > 1 &&
           entries(by_size[(size_t)first_small]) * workers > all_entries)
        prepare_one(by_size[(size_t)first_small++], threads);
    // the rest run concurrently, one thread each
    std::atomic<int32_t> next(first_small);
    auto work = [&]() {
        for (;;) {
            const int32_t k = next.fetch_add(1);
            if (k >= num_graphs) break;
            prepare_one(by_size[(size_t)k], 1);
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < workers; ++t) pool.emplace_back(work);
    work();
    for (auto& th : pool) th.join();
    const double t_order = now_s() - t0, t_clean = 0;
    int64_t total = 0;
    for (int32_t g = 0; g < num_graphs; ++g) {
        if (status[(size_t)g]) return fail(status[(size_t)g], "graph " + std::to_string(g) + ": " + errors[(size_t)g]);
        total += parts[(size_t)g].nnz();
        if (total >= ((int64_t)1 << 31)) return fail(BLEST_ERR_TOO_LARGE, "batch has 2^31 or more entries");
    }
    uni.ci.resize((size_t)total);
    int64_t pos = 0;
    for (int32_t g = 0; g < num_graphs; ++g) {
        const int64_t off = offsets[g];
        const Csr& p = parts[g];
        for (int32_t v = 0; v < p.n; ++v) {
            uni.rp[off + v + 1] = uni.rp[off + v] + (p.rp[v + 1] - p.rp[v]);
            new_id[off + v] = (int32_t)(off + (ids[g].empty() ? v : ids[g][v]));
        }
        for (int64_t e = 0; e < p.nnz(); ++e) uni.ci[pos++] = (int32_t)(p.ci[e] + off);
        parts[g] = Csr();
    }
    std::unique_ptr<blest_graph, void (*)(blest_graph*)> h(new blest_graph(), free_handle);
    h->stats.build_seconds = t_clean;
    blest_status s = finish_create(h.get(), uni, new_id, t_order);
    if (s) return s;
    h->stats.order = num_graphs > 0 ? orders[0] : BLEST_ORDER_NONE;
    h->offsets = offsets;
    *out = h.release();
    return BLEST_OK;
}

void blest_destroy(blest_handle h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->last_stream && h->last_stream != h->stream) cudaStreamSynchronize(h->last_stream);
    free_handle(h);
}

blest_status blest_set_option(blest_handle h, int32_t key, int64_t value) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    switch (key) {
        case BLEST_OPT_UPDATE:
            if (value < BLEST_UPDATE_AUTO || value > BLEST_UPDATE_LAZY) break;
            h->update_opt = (int)value;
            return BLEST_OK;
        case BLEST_OPT_PULL:
            if (value != BLEST_PULL_POPC && value != BLEST_PULL_MMA) break;
            h->pull = (int)value;
            return BLEST_OK;
        case BLEST_OPT_BLOCKS_PER_SM:
            if (value < 0 || value > 64) break;
            h->blocks_per_sm = (int)value;
            return BLEST_OK;
        case BLEST_OPT_BARRIER_TIMEOUT_US:
            if (value < 1 || value > 600000000) break;
            h->timeout_us = value;
            return BLEST_OK;
        case BLEST_OPT_RECORD_LEVELS:
            if (value != 0 && value != 1) break;
            h->record = (int)value;
            return BLEST_OK;
        case BLEST_OPT_UNROLL:
            if (value != 1 && value != 2 && value != 4) break;
            h->unroll = (int)value;
            return BLEST_OK;
        case BLEST_OPT_VISITED_FILTER:
            if (value < 0 || value > 4) break;
            h->filter = (int)value;
            return BLEST_OK;
        case BLEST_OPT_MIN_BLOCKS:
            if (value != 2 && value != 3) break;
            h->minb = (int)value;
            return BLEST_OK;
        case BLEST_OPT_STAGE_DEPTH:
            if (value != 0 && value != 2 && value != 3 && value != 4 && value != 8) break;
            h->depth = (int)value;
            return BLEST_OK;
        case BLEST_OPT_LAYOUT: {
            if (value != 0 && value != 1) break;
            if (value == 1) {
                blest_status st = ensure_compact(h);
                if (st) return st;
            }
            h->layout = (int)value;
            return BLEST_OK;
        }
        case BLEST_OPT_SCHEDULE:
            if (value != 0 && value != 1) break;
            h->sched = (int)value;
            return BLEST_OK;
        case BLEST_OPT_TEST_PHANTOM_BLOCK:
            if (value != 0 && value != 1) break;
            h->phantom = (int)value;
            return BLEST_OK;
        case BLEST_OPT_MS_PULL:
            if (value != BLEST_PULL_POPC && value != BLEST_PULL_MMA) break;
            h->ms_pull = (int)value;
            return BLEST_OK;
        case BLEST_OPT_MS_CHUNK:
            if (value != 64 && value != 128 && value != 256) break;
            h->ms_chunk = (int)value;
            return BLEST_OK;
        case BLEST_OPT_MS_BLOCKS_PER_SM:
            if (value < 0 || value > 64) break;
            h->ms_blocks_per_sm = (int)value;
            return BLEST_OK;
        case BLEST_OPT_MS_LEVELS:
            if (value < 0 || value > 2) break;
            h->ms_levels = (int)value;
            return BLEST_OK;
        case BLEST_OPT_MS_VISITED_FILTER:
            if (value < 0 || value > 2) break;
            h->ms_filter = (int)value;
            return BLEST_OK;
        default:
            return fail(BLEST_ERR_INVALID_ARG, "unknown option key");
    }
    return fail(BLEST_ERR_INVALID_ARG, "option value out of range");
}

blest_status blest_get_stats(blest_handle h, blest_stats* out) {
    if (!h || !out) return fail(BLEST_ERR_INVALID_ARG, "NULL argument");
    *out = h->stats;
    return BLEST_OK;
}

blest_status blest_bfs_device(blest_handle h, int32_t src, int32_t* d_levels, void* stream) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (h->n == 0 || src < 0 || src >= h->n) return fail(BLEST_ERR_INVALID_ARG, "source outside [0, n)");
    if (!d_levels) return fail(BLEST_ERR_INVALID_ARG, "levels is NULL");
    std::vector<int32_t> roots;
    blest_status s = map_sources(h, &src, 1, roots);
    if (s) return s;
    return enqueue_traversal(h, roots, d_levels, stream ? (cudaStream_t)stream : h->stream);
}

blest_status blest_bfs_multiroot_device(blest_handle h, const int32_t* srcs, int32_t k, int32_t* d_levels, void* stream) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (k < 0 || (k > 0 && !srcs)) return fail(BLEST_ERR_INVALID_ARG, "bad source list");
    if (h->n > 0 && !d_levels) return fail(BLEST_ERR_INVALID_ARG, "levels is NULL");
    std::vector<int32_t> roots;
    blest_status s = map_sources(h, srcs, k, roots);
    if (s) return s;
    cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
    if (k == 0) {
        if (h->n > 0) cudaMemsetAsync(d_levels, 0xFF, sizeof(int32_t) * (size_t)h->n, st);
        return BLEST_OK;
    }
    return enqueue_traversal(h, roots, d_levels, st);
}

blest_status blest_sync(blest_handle h) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    return sync_status(h);
}

blest_status blest_bfs(blest_handle h, int32_t src, int32_t* levels) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (!levels) return fail(BLEST_ERR_INVALID_ARG, "levels is NULL");
    blest_status s = blest_bfs_device(h, src, h->d_out, h->stream);
    if (s) return s;
    cudaError_t e = cudaMemcpyAsync(levels, h->d_out, sizeof(int32_t) * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy levels");
    return sync_status(h);
}

blest_status blest_bfs_parents(blest_handle h, int32_t src, int32_t* levels, int32_t* parents) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (!levels || !parents) return fail(BLEST_ERR_INVALID_ARG, "levels or parents is NULL");
    cudaError_t e;
    const size_t bytes = sizeof(int32_t) * (size_t)std::max(h->n, 1);
    if (!h->d_cand && (e = cudaMalloc(&h->d_cand, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(parents)");
    if (!h->d_parents && (e = cudaMalloc(&h->d_parents, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(parents)");
    if (!h->h_new_id.empty() && !h->d_old_of) {
        std::vector<int32_t> old_of((size_t)h->n);
        for (int32_t v = 0; v < h->n; ++v) old_of[h->h_new_id[v]] = v;
        if ((e = cudaMalloc(&h->d_old_of, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(old_of)");
        if ((e = cudaMemcpy(h->d_old_of, old_of.data(), bytes, cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "copy old_of");
    }
    h->need_internal_levels = true;
    blest_status s = blest_bfs_device(h, src, h->d_out, h->stream);
    h->need_internal_levels = false;
    if (s) return s;
    const int32_t* L = h->d_new_id ? h->d_L : h->d_out;   // levels in BVSS ids
    if ((e = blest::launch_parents(h->bvss.v2r, h->bvss.row_ids, h->bvss.masks, h->bvss.nvss, L, h->d_old_of,
                                   h->d_new_id, h->n, h->d_cand, h->d_parents, h->stream)) != cudaSuccess)
        return cuda_fail(e, "parents launch");
    if ((e = cudaMemcpyAsync(levels, h->d_out, sizeof(int32_t) * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(parents, h->d_parents, sizeof(int32_t) * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
        return cuda_fail(e, "copy results");
    return sync_status(h);
}

blest_status blest_bfs_multiroot(blest_handle h, const int32_t* srcs, int32_t k, int32_t* levels) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (h->n > 0 && !levels) return fail(BLEST_ERR_INVALID_ARG, "levels is NULL");
    blest_status s = blest_bfs_multiroot_device(h, srcs, k, h->d_out, h->stream);
    if (s) return s;
    if (h->n > 0) {
        cudaError_t e = cudaMemcpyAsync(levels, h->d_out, sizeof(int32_t) * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "copy levels");
    }
    return sync_status(h);
}

blest_status blest_batch_bfs(blest_handle h, const int32_t* srcs_local, int32_t* levels) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (h->offsets.empty()) return fail(BLEST_ERR_INVALID_ARG, "not a batch handle");
    const int32_t G = (int32_t)h->offsets.size() - 1;
    if (G > 0 && !srcs_local) return fail(BLEST_ERR_INVALID_ARG, "srcs is NULL");
    std::vector<int32_t> glob;
    for (int32_t g = 0; g < G; ++g) {
        const int64_t ng = h->offsets[g + 1] - h->offsets[g];
        if (ng == 0) continue;   // an empty graph has no source
        if (srcs_local[g] < 0 || srcs_local[g] >= ng) return fail(BLEST_ERR_INVALID_ARG, "source outside its graph");
        glob.push_back((int32_t)(h->offsets[g] + srcs_local[g]));
    }
    return blest_bfs_multiroot(h, glob.data(), (int32_t)glob.size(), levels);
}

blest_status blest_batch_graph_capture(blest_handle h, int32_t* d_levels) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (h->offsets.empty()) return fail(BLEST_ERR_INVALID_ARG, "not a batch handle");
    if (h->n > 0 && !d_levels) return fail(BLEST_ERR_INVALID_ARG, "levels is NULL");
    const int32_t G = (int32_t)h->offsets.size() - 1;
    std::vector<int32_t> first;   // a default source per non-empty graph
    for (int32_t g = 0; g < G; ++g)
        if (h->offsets[g + 1] > h->offsets[g]) first.push_back((int32_t)h->offsets[g]);
    const int32_t nr = (int32_t)first.size();
    // the captured kernel reads its sources from a device list; keep at least
    // kInlineRoots + 1 entries by repeating the first source (a repeated root is harmless)
    const int32_t cap = std::max<int32_t>(nr, blest::kInlineRoots + 1);
    if (nr == 0) return fail(BLEST_ERR_INVALID_ARG, "batch has no vertex");
    cudaError_t e;
    if (h->cgraph_exec) { cudaGraphExecDestroy(h->cgraph_exec); h->cgraph_exec = nullptr; }
    if (h->cgraph) { cudaGraphDestroy(h->cgraph); h->cgraph = nullptr; }
    cudaFree(h->d_graph_roots);
    h->d_graph_roots = nullptr;
    if (h->h_graph_roots) { cudaFreeHost(h->h_graph_roots); h->h_graph_roots = nullptr; }
    if ((e = cudaMalloc(&h->d_graph_roots, sizeof(int32_t) * cap)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(graph roots)");
    if ((e = cudaHostAlloc(&h->h_graph_roots, sizeof(int32_t) * cap, cudaHostAllocDefault)) != cudaSuccess)
        return cuda_fail(e, "cudaHostAlloc(graph roots)");
    if (!h->graph_done && (e = cudaEventCreateWithFlags(&h->graph_done, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate");
    for (int32_t i = 0; i < cap; ++i) {
        const int32_t v = first[i < nr ? i : 0];
        h->h_graph_roots[i] = h->h_new_id.empty() ? v : h->h_new_id[v];
    }
    h->graph_nroots = cap;
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if ((e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamBeginCapture");
    blest_status s = BLEST_OK;
    e = cudaMemcpyAsync(h->d_graph_roots, h->h_graph_roots, sizeof(int32_t) * cap, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) s = cuda_fail(e, "capture: copy roots");
    if (!s) s = enqueue_traversal(h, {}, d_levels, h->stream, h->d_graph_roots, cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->stream, &graph);
    if (!s && e != cudaSuccess) s = cuda_fail(e, "cudaStreamEndCapture");
    if (s) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    h->cgraph = graph;
    if ((e = cudaGraphInstantiate(&h->cgraph_exec, graph, 0)) != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return BLEST_OK;
}

blest_status blest_batch_graph_launch(blest_handle h, const int32_t* srcs_local, void* stream) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (!h->cgraph_exec) return fail(BLEST_ERR_INVALID_ARG, "no captured batch traversal on this handle");
    const int32_t G = (int32_t)h->offsets.size() - 1;
    if (G > 0 && !srcs_local) return fail(BLEST_ERR_INVALID_ARG, "srcs is NULL");
    cudaError_t e;
    // the pinned source list is read by the previous replay's copy: wait for it
    if ((e = cudaEventSynchronize(h->graph_done)) != cudaSuccess) return cuda_fail(e, "wait for previous replay");
    int32_t i = 0;
    for (int32_t g = 0; g < G; ++g) {
        const int64_t ng = h->offsets[g + 1] - h->offsets[g];
        if (ng == 0) continue;
        if (srcs_local[g] < 0 || srcs_local[g] >= ng) return fail(BLEST_ERR_INVALID_ARG, "source outside its graph");
        const int32_t v = (int32_t)(h->offsets[g] + srcs_local[g]);
        h->h_graph_roots[i++] = h->h_new_id.empty() ? v : h->h_new_id[v];
    }
    for (int32_t j = i; j < h->graph_nroots; ++j) h->h_graph_roots[j] = h->h_graph_roots[0];
    cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
    if ((e = cudaGraphLaunch(h->cgraph_exec, st)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    if ((e = cudaEventRecord(h->graph_done, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    h->last_stream = st;
    return BLEST_OK;
}

blest_status blest_msbfs_device(blest_handle h, const int32_t* srcs, int32_t k, int32_t* d_levels, void* stream) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (k < 0 || (k > 0 && !srcs)) return fail(BLEST_ERR_INVALID_ARG, "bad source list");
    if (k == 0) return BLEST_OK;
    if (!d_levels) return fail(BLEST_ERR_INVALID_ARG, "levels is NULL");
    std::vector<int32_t> roots;
    blest_status s = map_sources(h, srcs, k, roots);
    if (s) return s;
    cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
    blest::MsbfsLaunchCommon c;
    c.n = h->n;
    c.nss = h->bvss.nss;
    c.nvss = h->bvss.nvss;
    c.real_ptrs = h->bvss.real_ptrs;
    c.row_ids = h->bvss.row_ids;
    c.masks = h->bvss.masks;
    c.new_id = h->d_new_id;
    c.ctrl = h->d_ctrl;
    c.sms = h->sms;
    c.blocks_per_sm = h->ms_blocks_per_sm ? h->ms_blocks_per_sm : h->blocks_per_sm;
    c.timeout_ns = (uint64_t)h->timeout_us * 1000ull;
    c.phantom = h->phantom ? 1u : 0u;
    c.level_sizes = h->record ? h->d_level_sizes : nullptr;
    c.level_cap = kLevelRecordCap;
    c.pull = h->ms_pull;
    c.chunk = h->ms_chunk;
    c.levels_layout = h->ms_levels_layout();
    c.visited_filter = h->ms_filter;
    const char* err = nullptr;
    int rc = blest::run_msbfs(h->ms, c, roots, d_levels, st, &err);
    if (rc) return fail((blest_status)rc, std::string("msbfs: ") + (err ? err : "?"));
    h->last_stream = st;
    h->info.update = BLEST_UPDATE_LAZY;
    h->info.pull = h->ms_pull;
    h->info.recorded = -1;
    return BLEST_OK;
}

blest_status blest_msbfs(blest_handle h, const int32_t* srcs, int32_t k, int32_t* levels) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (k < 0 || (k > 0 && (!srcs || !levels))) return fail(BLEST_ERR_INVALID_ARG, "bad arguments");
    if (k == 0) return BLEST_OK;
    int32_t* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int32_t) * (size_t)k * (size_t)std::max(h->n, 1));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(msbfs levels)");
    blest_status s = blest_msbfs_device(h, srcs, k, d, h->stream);
    if (!s) {
        e = cudaMemcpyAsync(levels, d, sizeof(int32_t) * (size_t)k * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) s = cuda_fail(e, "copy levels");
    }
    blest_status s2 = sync_status(h);
    cudaFree(d);
    return s ? s : s2;
}

blest_status blest_distance_stats(blest_handle h, const int32_t* srcs, int32_t k, int64_t* reached,
                                  int64_t* sum_dist, int32_t* ecc) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (k < 0 || (k > 0 && (!srcs || !reached || !sum_dist || !ecc))) return fail(BLEST_ERR_INVALID_ARG, "bad arguments");
    if (k == 0) return BLEST_OK;
    std::vector<int32_t> roots;
    blest_status s = map_sources(h, srcs, k, roots);   // validates the whole list before any work
    if (s) return s;
    // sources in batches whose level rows fit in 4 GiB (at most 256, one multi-source launch)
    const int64_t n = std::max<int64_t>(h->n, 1);
    const int32_t batch = (int32_t)std::max<int64_t>(1, std::min<int64_t>({256, k, ((int64_t)4 << 30) / (4 * n)}));
    int32_t* d_lv = nullptr;
    unsigned long long* d_acc = nullptr;
    int* d_ecc = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&d_lv, sizeof(int32_t) * (size_t)batch * (size_t)n)) != cudaSuccess ||
        (e = cudaMalloc(&d_acc, sizeof(unsigned long long) * 2 * (size_t)batch)) != cudaSuccess ||
        (e = cudaMalloc(&d_ecc, sizeof(int) * (size_t)batch)) != cudaSuccess) {
        cudaFree(d_lv);
        cudaFree(d_acc);
        return cuda_fail(e, "cudaMalloc(distance stats)");
    }
    std::vector<unsigned long long> acc(2 * (size_t)batch);
    for (int32_t b0 = 0; b0 < k && !s; b0 += batch) {
        const int32_t kb = std::min(batch, k - b0);
        s = blest_msbfs_device(h, srcs + b0, kb, d_lv, h->stream);
        if (s) break;
        if ((e = blest::launch_distance_stats(d_lv, kb, h->n, d_acc, d_ecc, h->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(acc.data(), d_acc, sizeof(unsigned long long) * 2 * (size_t)kb,
                                 cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(ecc + b0, d_ecc, sizeof(int) * (size_t)kb, cudaMemcpyDeviceToHost, h->stream)) !=
                cudaSuccess) {
            s = cuda_fail(e, "distance stats");
            break;
        }
        if ((s = sync_status(h)) != BLEST_OK) break;
        for (int32_t i = 0; i < kb; ++i) {
            reached[b0 + i] = (int64_t)acc[i];
            sum_dist[b0 + i] = (int64_t)acc[kb + i];
        }
    }
    sync_status(h);
    cudaFree(d_lv);
    cudaFree(d_acc);
    cudaFree(d_ecc);
    return s;
}

blest_status blest_get_run_info(blest_handle h, blest_run_info* info, int32_t* queue_sizes, int32_t cap) {
    if (!h || !info) return fail(BLEST_ERR_INVALID_ARG, "NULL argument");
    blest_status s = sync_status(h);
    if (s) return s;
    unsigned int ctrl[16];
    cudaError_t e = cudaMemcpy(ctrl, h->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read run info");
    h->info.levels = (int32_t)ctrl[6];
    h->info.recorded = h->record ? std::min<int32_t>(h->info.levels, kLevelRecordCap) : 0;
    *info = h->info;
    if (queue_sizes && cap > 0 && h->info.recorded > 0) {
        int32_t m = std::min(cap, h->info.recorded);
        e = cudaMemcpy(queue_sizes, h->d_level_sizes, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "read level record");
    }
    return BLEST_OK;
}

blest_status blest_autotune_msbfs(blest_handle h, const int32_t* srcs, int32_t k, blest_ms_tune_result* out) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (k < 1 || !srcs) return fail(BLEST_ERR_INVALID_ARG, "autotune needs at least one source");
    if (h->n == 0) return fail(BLEST_ERR_INVALID_ARG, "empty graph");
    std::vector<int32_t> roots;
    blest_status s = map_sources(h, srcs, k, roots);
    if (s) return s;
    // launch sizes that give different launches for k sources
    std::vector<int> chunks{blest::kMsbfsChunk};
    if (k > 64) chunks.push_back(64);
    if (k > 128) chunks.push_back(128);
    int32_t* d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_out, sizeof(int32_t) * (size_t)k * (size_t)h->n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(autotune levels)");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaFree(d_out);
        return cuda_fail(e, "cudaEventCreate");
    }
    const int saved_pull = h->ms_pull, saved_chunk = h->ms_chunk, saved_bps = h->ms_blocks_per_sm;
    const int saved_levels = h->ms_levels, saved_filter = h->ms_filter;
    double best = 1e300, best_pull[2] = {-1.0, -1.0};
    int bp = saved_pull, bc = saved_chunk, bb = saved_bps, bl = saved_levels, bf = saved_filter, timed = 0;
    for (int pull : {BLEST_PULL_POPC, BLEST_PULL_MMA})
        for (int chunk : chunks)
            for (int bps : {0, 1, 2})   // blocks per SM above what fits run as many as fit
            for (int levels : {1, 2})    // vertex-major, bit planes
            for (int filt : {1, 2, 0}) { // V_curr or V_next test before each mark, or none
                if (s) break;
                // one layout and the default test are enough to time the MMA
                if (pull == BLEST_PULL_MMA && (levels != 2 || filt != 1)) continue;
                h->ms_pull = pull;
                h->ms_chunk = chunk;
                h->ms_blocks_per_sm = bps;
                h->ms_levels = levels;
                h->ms_filter = filt;
                for (int pass = 0; pass < 2 && !s; ++pass) {
                    if (pass == 1) cudaEventRecord(e0, h->stream);
                    s = blest_msbfs_device(h, srcs, k, d_out, h->stream);
                }
                if (s) break;
                cudaEventRecord(e1, h->stream);
                if ((s = sync_status(h)) != BLEST_OK) break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ++timed;
                if (best_pull[pull] < 0 || ms < best_pull[pull]) best_pull[pull] = ms;
                if (ms < best) { best = ms; bp = pull; bc = chunk; bb = bps; bl = levels; bf = filt; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_out);
    if (s) {
        h->ms_pull = saved_pull; h->ms_chunk = saved_chunk; h->ms_blocks_per_sm = saved_bps;
        h->ms_levels = saved_levels;
        h->ms_filter = saved_filter;
        return s;
    }
    h->ms_pull = bp; h->ms_chunk = bc; h->ms_blocks_per_sm = bb; h->ms_levels = bl; h->ms_filter = bf;
    if (out) {
        out->pull = bp; out->chunk = bc; out->blocks_per_sm = bb; out->levels = bl; out->visited_filter = bf;
        out->candidates = timed;
        out->best_ms = best; out->popc_ms = best_pull[0]; out->mma_ms = best_pull[1];
    }
    return BLEST_OK;
}

// Shared by blest_autotune (k single-source traversals per timing) and
// blest_autotune_multiroot (one traversal from all k roots per timing).
static blest_status autotune_impl(blest_handle h, const int32_t* srcs, int32_t k, bool multiroot,
                                  blest_tune_result* out) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (k < 1 || !srcs) return fail(BLEST_ERR_INVALID_ARG, "autotune needs at least one source");
    if (h->n == 0) return fail(BLEST_ERR_INVALID_ARG, "empty graph");
    std::vector<int32_t> roots;
    blest_status s = map_sources(h, srcs, k, roots);
    if (s) return s;
    struct Cand { int update, pull, unroll, minb, filter, bps, depth, layout = 0, sched = 0; };
    std::vector<Cand> cands;
    for (int u : {BLEST_UPDATE_EAGER, BLEST_UPDATE_LAZY})
        for (int p : {BLEST_PULL_POPC, BLEST_PULL_MMA})
            for (int r : {1, 2})
                for (int m : {2, 3})
                    for (int f = 0; f <= (u == BLEST_UPDATE_LAZY ? 4 : 1); ++f)
                        for (int b : {0, 1}) cands.push_back({u, p, r, m, f, b, 0});
    for (int f : {0, 1, 2, 3, 4})
        for (int b : {0, 1}) {
            for (int p : {BLEST_PULL_POPC, BLEST_PULL_MMA})
                for (int r : {1, 2}) {
                    cands.push_back({BLEST_UPDATE_LAZY, p, r, 2, f, b, 2});
                    cands.push_back({BLEST_UPDATE_LAZY, p, r, 2, f, b, 2, 0, 1});   // static + dynamic tail
                    if (p == BLEST_PULL_POPC && f > 0) {                        // tiles two groups ahead
                        cands.push_back({BLEST_UPDATE_LAZY, p, r, 2, f, b, 3, 0, 0});
                        cands.push_back({BLEST_UPDATE_LAZY, p, r, 2, f, b, 3, 0, 1});
                    }
                    // compact layout (register paths)
                    if (b == 0) {
                        cands.push_back({BLEST_UPDATE_LAZY, p, r, 2, f, b, 0, 1});
                        cands.push_back({BLEST_UPDATE_LAZY, p, r, 2, f, b, 2, 1});
                        cands.push_back({BLEST_UPDATE_LAZY, p, r, 2, f, b, 2, 1, 1});
                    }
                }
            cands.push_back({BLEST_UPDATE_LAZY, BLEST_PULL_POPC, 1, 2, f, b, 4});
            cands.push_back({BLEST_UPDATE_LAZY, BLEST_PULL_POPC, 2, 2, f, b, 4});
            cands.push_back({BLEST_UPDATE_LAZY, BLEST_PULL_POPC, 1, 2, f, b, 8});
            cands.push_back({BLEST_UPDATE_LAZY, BLEST_PULL_POPC, 2, 2, f, b, 8});
            cands.push_back({BLEST_UPDATE_LAZY, BLEST_PULL_POPC, 4, 2, f, b, 8});
            cands.push_back({BLEST_UPDATE_LAZY, BLEST_PULL_MMA, 1, 2, f, b, 4});
            cands.push_back({BLEST_UPDATE_LAZY, BLEST_PULL_MMA, 2, 2, f, b, 8});
        }
    struct Opts { int update_opt, pull, unroll, minb, filter, blocks_per_sm, depth, layout, sched; };
    const Opts saved{h->update_opt, h->pull, h->unroll, h->minb, h->filter, h->blocks_per_sm, h->depth, h->layout,
                     h->sched};
    if ((s = ensure_compact(h)) != BLEST_OK) return s;
    cudaEvent_t e0, e1;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(e, "cudaEventCreate"); }
    double best = 1e300, rule = -1.0;
    Cand bestc = cands[0];
    const int rule_update = h->stats.update;
    int timed = 0;
    // mean device time per traversal of one candidate (one untimed pass first); < 0 on error
    auto time_one = [&](const Cand& c) -> double {
        h->update_opt = c.update; h->pull = c.pull; h->unroll = c.unroll; h->minb = c.minb;
        h->filter = c.filter; h->blocks_per_sm = c.bps; h->depth = c.depth; h->layout = c.layout;
        h->sched = c.sched;
        std::vector<int32_t> one(1);
        for (int pass = 0; pass < 2 && !s; ++pass) {
            if (pass == 1) cudaEventRecord(e0, h->stream);
            if (multiroot) {
                s = enqueue_traversal(h, roots, h->d_out, h->stream);
                continue;
            }
            for (int32_t i = 0; i < k && !s; ++i) {
                one[0] = roots[i];
                s = enqueue_traversal(h, one, h->d_out, h->stream);
            }
        }
        if (s) return -1.0;
        cudaEventRecord(e1, h->stream);
        if ((s = sync_status(h)) != BLEST_OK) return -1.0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ++timed;
        const double per = multiroot ? (double)ms : (double)ms / k;
        if (per < best) { best = per; bestc = c; }
        return per;
    };
    // stage 1: the update scheme, from a few representative variants of each and
    // the Section 5 rule's plain kernel; stage 2: every variant of the scheme that won
    const Cand probes[] = {{BLEST_UPDATE_EAGER, BLEST_PULL_POPC, 1, 2, 0, 0, 0},
                           {BLEST_UPDATE_EAGER, BLEST_PULL_POPC, 2, 2, 1, 0, 0},
                           {BLEST_UPDATE_LAZY, BLEST_PULL_POPC, 2, 2, 3, 0, 2, 0, 1},
                           {BLEST_UPDATE_LAZY, BLEST_PULL_POPC, 2, 2, 1, 0, 0},
                           {rule_update, BLEST_PULL_POPC, 2, 2, 0, 0, 0}};
    for (int i = 0; i < 5 && !s; ++i) {
        const double per = time_one(probes[i]);
        if (i == 4) rule = per;
    }
    const int scheme = bestc.update;
    for (const Cand& c : cands) {
        if (s) break;
        if (c.update != scheme) continue;
        time_one(c);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->update_opt = saved.update_opt; h->pull = saved.pull; h->unroll = saved.unroll; h->minb = saved.minb;
    h->filter = saved.filter; h->blocks_per_sm = saved.blocks_per_sm; h->depth = saved.depth;
    h->layout = saved.layout;
    h->sched = saved.sched;
    if (s) return s;
    h->update_opt = bestc.update; h->pull = bestc.pull; h->unroll = bestc.unroll; h->minb = bestc.minb;
    h->filter = bestc.filter; h->blocks_per_sm = bestc.bps; h->depth = bestc.depth; h->layout = bestc.layout;
    h->sched = bestc.sched;
    if (out) {
        out->update = bestc.update; out->pull = bestc.pull; out->unroll = bestc.unroll; out->min_blocks = bestc.minb;
        out->visited_filter = bestc.filter; out->blocks_per_sm = bestc.bps; out->stage_depth = bestc.depth;
        out->layout = bestc.layout;
        out->schedule = bestc.sched;
        out->candidates = (int32_t)timed;
        out->best_ms = best; out->rule_ms = rule;
    }
    return BLEST_OK;
}

blest_status blest_autotune(blest_handle h, const int32_t* srcs, int32_t k, blest_tune_result* out) {
    return autotune_impl(h, srcs, k, false, out);
}

blest_status blest_autotune_multiroot(blest_handle h, const int32_t* srcs, int32_t k, blest_tune_result* out) {
    return autotune_impl(h, srcs, k, true, out);
}

blest_status blest_get_level_arrivals(blest_handle h, int32_t phase, uint64_t* first_ns, uint64_t* last_ns,
                                      int32_t cap) {
    if (!h || (cap > 0 && (!first_ns || !last_ns))) return fail(BLEST_ERR_INVALID_ARG, "NULL argument");
    if (phase != 0 && phase != 1) return fail(BLEST_ERR_INVALID_ARG, "phase must be 0 (stage 1) or 1 (sweep)");
    blest_status s = sync_status(h);
    if (s) return s;
    const int32_t m = std::min<int32_t>(cap, kLevelRecordCap);
    if (m > 0) {
        const size_t off = (size_t)phase * kLevelRecordCap;
        cudaError_t e = cudaMemcpy(first_ns, h->d_arrive + off, sizeof(uint64_t) * (size_t)m, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(last_ns, h->d_arrive + 2 * kLevelRecordCap + off, sizeof(uint64_t) * (size_t)m,
                           cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "read level arrivals");
    }
    return BLEST_OK;
}

blest_status blest_get_level_times(blest_handle h, uint64_t* times_ns, int32_t cap) {
    if (!h || (cap > 0 && !times_ns)) return fail(BLEST_ERR_INVALID_ARG, "NULL argument");
    blest_status s = sync_status(h);
    if (s) return s;
    unsigned int ctrl[16];
    cudaError_t e = cudaMemcpy(ctrl, h->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read run info");
    const int32_t levels = (int32_t)ctrl[6];
    if (!h->record) return fail(BLEST_ERR_INVALID_ARG, "level recording is off (BLEST_OPT_RECORD_LEVELS)");
    const int32_t m = std::min<int32_t>(cap, 2 * std::min<int32_t>(levels, kLevelRecordCap - 2) + 4);
    if (m > 0) {
        e = cudaMemcpy(times_ns, h->d_level_times, sizeof(uint64_t) * (size_t)m, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "read level times");
    }
    return BLEST_OK;
}

int64_t blest_export_size(blest_handle h, int32_t which) {
    if (!h) return -1;
    switch (which) {
        case BLEST_ARRAY_REAL_PTRS: return 4 * ((int64_t)h->bvss.nss + 1);
        case BLEST_ARRAY_VIRTUAL_TO_REAL: return 4 * h->bvss.nvss;
        case BLEST_ARRAY_ROW_IDS: return 4 * 128 * h->bvss.nvss;
        case BLEST_ARRAY_MASKS: return 4 * 32 * h->bvss.nvss;
        case BLEST_ARRAY_NEW_ID: return 4 * (int64_t)h->n;
        case BLEST_ARRAY_VSS_COUNT: return 4 * h->bvss.nvss;
        case BLEST_ARRAY_COMPACT_OFFSETS: return 4 * ((int64_t)h->bvss.nss + 1);
        case BLEST_ARRAY_COMPACT_ROWS:
        case BLEST_ARRAY_COMPACT_MASKS: {
            if (ensure_compact(h)) return -1;
            return (which == BLEST_ARRAY_COMPACT_ROWS ? 16 : 4) * h->compact.groups;
        }
    }
    return -1;
}

blest_status blest_export(blest_handle h, int32_t which, void* host_out, int64_t bytes) {
    if (!h || (!host_out && bytes > 0)) return fail(BLEST_ERR_INVALID_ARG, "NULL argument");
    int64_t need = blest_export_size(h, which);
    if (need < 0) return fail(BLEST_ERR_INVALID_ARG, "unknown array");
    if (bytes != need) return fail(BLEST_ERR_INVALID_ARG, "byte count does not match the array size");
    if (need == 0) return BLEST_OK;
    const void* src = nullptr;
    switch (which) {
        case BLEST_ARRAY_REAL_PTRS: src = h->bvss.real_ptrs; break;
        case BLEST_ARRAY_VIRTUAL_TO_REAL: src = h->bvss.v2r; break;
        case BLEST_ARRAY_ROW_IDS: src = h->bvss.row_ids; break;
        case BLEST_ARRAY_MASKS: src = h->bvss.masks; break;
        case BLEST_ARRAY_VSS_COUNT: src = h->bvss.vss_count; break;
        case BLEST_ARRAY_COMPACT_OFFSETS:
        case BLEST_ARRAY_COMPACT_ROWS:
        case BLEST_ARRAY_COMPACT_MASKS: {
            blest_status cs = ensure_compact(h);
            if (cs) return cs;
            src = which == BLEST_ARRAY_COMPACT_OFFSETS ? (const void*)h->compact.goff
                : which == BLEST_ARRAY_COMPACT_ROWS ? (const void*)h->compact.rows : (const void*)h->compact.masks;
            break;
        }
        case BLEST_ARRAY_NEW_ID:
            if (h->h_new_id.empty()) {
                int32_t* o = (int32_t*)host_out;
                for (int32_t v = 0; v < h->n; ++v) o[v] = v;
            } else {
                std::memcpy(host_out, h->h_new_id.data(), (size_t)need);
            }
            return BLEST_OK;
    }
    blest_status s = sync_status(h);
    if (s) return s;
    cudaError_t e = cudaMemcpy(host_out, src, (size_t)need, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "export");
    return BLEST_OK;
}

blest_status blest_compute_order(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, blest_order order,
                                 const blest_create_params* params, int32_t* new_id) {
    if (n > 0 && !new_id) return fail(BLEST_ERR_INVALID_ARG, "new_id is NULL");
    const int threads = blest::host_threads(params ? params->threads : 0);
    Csr clean;
    std::vector<int32_t> ids;
    int32_t used = 0;
    double to = 0, tc = 0;
    blest_status s = prepare_graph(n, row_ptr, col_idx, order, params, threads, clean, ids, &used, &to, &tc);
    if (s) return s;
    for (int32_t v = 0; v < n; ++v) new_id[v] = ids.empty() ? v : ids[v];
    return BLEST_OK;
}

int32_t blest_is_social(int32_t n, const int32_t* row_ptr, const int32_t* col_idx) {
    Csr clean;
    std::string err;
    int rc = blest::clean_csr(n, row_ptr, col_idx, blest::host_threads(0), clean, err);
    if (rc) {
        g_last_error = err;
        return -rc;
    }
    return blest::is_social_like(clean) ? 1 : 0;
}

blest_status blest_shard_begin(blest_handle h, int32_t rank, int32_t world, int32_t src, int32_t* d_levels,
                               void* stream) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (world < 1 || rank < 0 || rank >= world) return fail(BLEST_ERR_INVALID_ARG, "rank must be in [0, world)");
    if (!h->offsets.empty()) return fail(BLEST_ERR_INVALID_ARG, "a batch handle has no sharded traversal");
    if (h->n == 0) return fail(BLEST_ERR_INVALID_ARG, "empty graph");
    if (!d_levels) return fail(BLEST_ERR_INVALID_ARG, "levels is NULL");
    std::vector<int32_t> roots;
    blest_status s = map_sources(h, &src, 1, roots);
    if (s) return s;
    cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
    h->shard_rank = rank;
    h->shard_world = world;
    h->shard_out = d_levels;
    h->shard_level = 1;
    h->shard_reached = 1;   // the level-0 sweep gives the root its level
    blest::BfsLaunch L = shard_launch(h);
    cudaError_t e;
    // [V_curr | V_next | dirty | control block up to the sticky status word]
    const size_t skip = 3 * h->bitmap_bytes;
    if ((e = cudaMemsetAsync(h->d_state + skip, 0, kStateBitmaps * h->bitmap_bytes + h->dirty_bytes - skip +
                                                       kCtrlClearBytes, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(L.direct ? d_levels : L.levels_internal, 0xFF, sizeof(int32_t) * (size_t)h->n, st)) !=
            cudaSuccess ||
        (e = blest::launch_shard_step(L, blest::kShardRoot, 0, world, rank, roots[0], nullptr, st)) != cudaSuccess ||
        (e = blest::launch_shard_step(L, blest::kShardSweep, 0, world, rank, 0, nullptr, st)) != cudaSuccess)
        return cuda_fail(e, "shard: level 0");
    h->last_stream = st;
    return BLEST_OK;
}

blest_status blest_shard_pull(blest_handle h, uint32_t* d_words, void* stream) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (h->shard_rank < 0) return fail(BLEST_ERR_INVALID_ARG, "no sharded traversal begun on this handle");
    if (!d_words) return fail(BLEST_ERR_INVALID_ARG, "words is NULL");
    cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
    blest::BfsLaunch L = shard_launch(h);
    cudaError_t e;
    if ((e = blest::launch_shard_step(L, blest::kShardPull, h->shard_level, h->shard_world, h->shard_rank, 0,
                                      nullptr, st)) != cudaSuccess ||
        (e = blest::launch_shard_step(L, blest::kShardWordsOut, h->shard_level, h->shard_world, h->shard_rank, 0,
                                      d_words, st)) != cudaSuccess)
        return cuda_fail(e, "shard: pull");
    h->last_stream = st;
    return BLEST_OK;
}

blest_status blest_shard_merge(uint32_t* d_dst, const uint32_t* d_src, int64_t words, int32_t count, void* stream) {
    if (words < 0 || count < 1 || (words > 0 && (!d_dst || !d_src))) return fail(BLEST_ERR_INVALID_ARG, "bad arguments");
    if (words == 0) return BLEST_OK;
    cudaError_t e = blest::launch_or_words(d_dst, d_src, words, count, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "shard: merge");
    return BLEST_OK;
}

blest_status blest_shard_sweep(blest_handle h, const uint32_t* d_merged, void* stream) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (h->shard_rank < 0) return fail(BLEST_ERR_INVALID_ARG, "no sharded traversal begun on this handle");
    if (!d_merged) return fail(BLEST_ERR_INVALID_ARG, "merged is NULL");
    cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
    blest::BfsLaunch L = shard_launch(h);
    cudaError_t e;
    if ((e = blest::launch_shard_step(L, blest::kShardWordsIn, h->shard_level, h->shard_world, h->shard_rank, 0,
                                      const_cast<uint32_t*>(d_merged), st)) != cudaSuccess ||
        (e = blest::launch_shard_step(L, blest::kShardSweep, h->shard_level, h->shard_world, h->shard_rank, 0,
                                      nullptr, st)) != cudaSuccess)
        return cuda_fail(e, "shard: sweep");
    h->last_stream = st;
    return BLEST_OK;
}

blest_status blest_shard_more(blest_handle h, int32_t* more) {
    if (!h) return fail(BLEST_ERR_INVALID_ARG, "NULL handle");
    if (h->shard_rank < 0) return fail(BLEST_ERR_INVALID_ARG, "no sharded traversal begun on this handle");
    if (!more) return fail(BLEST_ERR_INVALID_ARG, "more is NULL");
    blest_status s = sync_status(h);
    if (s) return s;
    unsigned int ctrl[16];
    cudaError_t e;
    if ((e = cudaMemcpy(ctrl, h->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "shard: read counters");
    const unsigned int reached = ctrl[7];   // Ctrl::reached
    *more = reached > h->shard_reached ? 1 : 0;
    h->shard_reached = reached;
    h->shard_level += 1;
    if (!*more) h->shard_rank = -1;   // the traversal is over; d_levels holds every level
    return BLEST_OK;
}

blest_status blest_shard_finish(blest_handle h, const uint32_t* d_merged, int32_t* more, void* stream) {
    if (!more) return fail(BLEST_ERR_INVALID_ARG, "more is NULL");
    blest_status s = blest_shard_sweep(h, d_merged, stream);
    if (s) return s;
    return blest_shard_more(h, more);
}

blest_status blest_debug_pull(const uint32_t* d_masks, const uint8_t* d_alpha, int32_t tiles, int32_t pull,
                              uint8_t* d_hits) {
    if (tiles < 0 || (tiles > 0 && (!d_masks || !d_alpha || !d_hits))) return fail(BLEST_ERR_INVALID_ARG, "bad arguments");
    if (pull != BLEST_PULL_POPC && pull != BLEST_PULL_MMA) return fail(BLEST_ERR_INVALID_ARG, "unknown pull");
    if (tiles == 0) return BLEST_OK;
    cudaError_t e = blest::launch_debug_pull(d_masks, d_alpha, tiles, pull, d_hits, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "debug pull");
    return BLEST_OK;
}

}  // extern "C"
