// Query server with continuous batching (host runtime; the traversals are the
// multi-source kernel of msbfs_kernel.cu).
//
// A server keeps a set of graph handles resident and runs one scheduler
// thread.  Clients submit queries (graph, k sources, output buffer) at any
// time.  The scheduler repeatedly
//   * retires finished launches: each query of the launch gets its status and
//     completion time, and the launch's device memory is returned;
//   * forms new launches while a launch slot is free: it takes the graph whose
//     oldest waiting query is oldest, packs that graph's waiting queries in
//     arrival order into one multi-source launch of at most max_batch_sources
//     sources, and admits it only if its device memory (levels k x n, bit
//     matrices, queues) fits under memory_cap_bytes next to the launches
//     already in flight; the memory comes from the stream-ordered allocator and
//     goes back when the launch retires.  A long graph (its previous launch ran
//     more than narrow_levels levels) is passed over while long_slots of its kind
//     are in flight, so that the other graphs' short launches find a slot.
// Queries arriving while launches run join the next launch of their graph, and
// launches of different graphs (or of the same graph) run concurrently on
// their own streams; each launch uses a persistent grid of blocks_per_sm
// blocks per SM so that several fit on the GPU at once.  Every query's levels
// are exactly those of blest_msbfs on its own.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/blest.h"
#include "msbfs_launch.h"

namespace blest {
void set_last_error(const std::string& msg);   // api.cu
// Read-only view of a handle for the server (api.cu).
struct HandleView {
    int32_t n;
    int32_t nss;
    int64_t nvss;
    const int32_t* real_ptrs;
    const int32_t* row_ids;
    const uint32_t* masks;
    const int32_t* new_id_dev;
    const int32_t* new_id_host;   // NULL = identity
    int sms;
    int levels_layout;            // multi-source level layout (0 vertex-major, 1 bit planes)
};
bool handle_view(blest_handle h, HandleView* v);
}  // namespace blest

namespace {

using clk = std::chrono::steady_clock;

blest_status fail(blest_status s, const std::string& m) {
    blest::set_last_error(m);
    return s;
}

struct Query {
    uint64_t ticket = 0;
    int32_t graph = 0;
    std::vector<int32_t> roots;      // BVSS ids
    int32_t* levels = nullptr;       // caller's output (host or device), k * n int32, may be NULL
    clk::time_point t_submit;
    clk::time_point t_done;
    blest_status status = BLEST_OK;
    bool done = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    unsigned int* d_ctrl = nullptr;  // 256-byte control block of the launch
    unsigned int* h_status = nullptr;  // pinned: [0] the sticky status word, [1] the launch's level count
    int32_t graph = -1;                // graph of the launch in flight
    bool busy = false;
    bool long_launch = false;          // the graph counted as long when the launch started
    std::vector<Query*> batch;
    int32_t* d_levels = nullptr;
    blest::MsbfsState ms;
    int64_t bytes = 0;
};

constexpr int kStickyWord = 48;   // control-block layout of device_common.cuh

}  // namespace

struct blest_server {
    std::vector<blest_handle> graphs;
    std::vector<blest::HandleView> views;
    blest_server_params p{};
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work;   // new queries or shutdown
    std::condition_variable cv_done;   // a query finished
    std::vector<std::deque<Query*>> pending;
    std::vector<int32_t> last_levels;  // per graph: levels of its last finished launch (0 = none yet)
    std::unordered_map<uint64_t, std::unique_ptr<Query>> queries;
    uint64_t next_ticket = 1;
    int64_t mem_used = 0, mem_peak = 0;
    int64_t launches = 0, sources_launched = 0, queries_done = 0;
    bool stop = false;
    bool paused = false;
    std::string worker_error;
    std::thread worker;
    int dev = 0;
};

namespace {

// While any server lives, the device's default stream-ordered pool keeps up to
// the largest memory cap cached between launches (its release threshold).  The
// first server saves the threshold it found; the last one to go restores it and
// returns the cached memory.
std::mutex g_pool_mu;
int g_pool_users = 0;
uint64_t g_pool_saved = 0;

void pool_acquire(int dev, int64_t cap) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    uint64_t cur = 0;
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur);
    if (g_pool_users++ == 0) g_pool_saved = cur;
    uint64_t thr = std::max<uint64_t>(cur, (uint64_t)cap);
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
}

void pool_release(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (g_pool_users == 0 || --g_pool_users > 0) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    uint64_t thr = g_pool_saved;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    cudaMemPoolTrimTo(pool, 0);
}

int64_t launch_bytes(const blest::HandleView& v, int k) {
    const int W = blest::msbfs_words(k);
    int64_t b = (int64_t)k * v.n * 4;                          // levels
    b += 3 * (int64_t)v.n * W * 8;                            // V_curr, V_next, frontier
    b += 3 * std::max<int64_t>(v.nvss, 1) * 8;                // queues
    if (v.levels_layout == 1) b += blest::msbfs_plane_words(v.n, k) * 8;   // level bit planes in BVSS ids
    else b += blest::msbfs_level_entries(v.n, k) * 4;                   // vertex-major levels in BVSS ids
    b += (int64_t)k * 4 + 4 * 256;                             // roots, alignment slack
    b += ((int64_t)v.nss + 31) / 32 * 4;                       // dirty slice sets
    return b;
}

template <class T>
cudaError_t alloc_async(T*& p, int64_t count, cudaStream_t st) {
    return cudaMallocAsync(reinterpret_cast<void**>(&p), sizeof(T) * (size_t)std::max<int64_t>(count, 1), st);
}

cudaError_t alloc_launch(Slot& s, const blest::HandleView& v, int k) {
    const int64_t words = (int64_t)v.n * blest::msbfs_words(k);
    cudaError_t e;
    blest::MsbfsState& m = s.ms;
    m = blest::MsbfsState();
    m.caller_owned = true;   // stream-ordered pool memory: the launcher must not reallocate it
    if ((e = alloc_async(s.d_levels, (int64_t)k * v.n, s.stream)) != cudaSuccess) return e;
    if ((e = alloc_async(m.vcur, words, s.stream)) != cudaSuccess) return e;
    if ((e = alloc_async(m.vnext, words, s.stream)) != cudaSuccess) return e;
    if ((e = alloc_async(m.front, words, s.stream)) != cudaSuccess) return e;
    m.words_cap = words;
    if ((e = alloc_async(m.Q, 3 * std::max<int64_t>(v.nvss, 1), s.stream)) != cudaSuccess) return e;
    m.qcap = std::max<int64_t>(v.nvss, 1);
    if (v.levels_layout == 1) {
        const int64_t pw = blest::msbfs_plane_words(v.n, k);
        if ((e = alloc_async(m.planes, pw, s.stream)) != cudaSuccess) return e;
        m.planes_cap = pw;
    } else {
        const int64_t lev = blest::msbfs_level_entries(v.n, k);
        if ((e = alloc_async(m.lint, lev, s.stream)) != cudaSuccess) return e;
        m.lint_cap = lev;
    }
    if ((e = alloc_async(m.roots, k, s.stream)) != cudaSuccess) return e;
    m.roots_cap = k;
    const int64_t dwords = ((int64_t)v.nss + 31) / 32;
    if ((e = alloc_async(m.dirty, dwords, s.stream)) != cudaSuccess) return e;
    m.dirty_cap = dwords;
    return cudaSuccess;
}

void free_launch(Slot& s) {
    blest::MsbfsState& m = s.ms;
    for (void* p : {(void*)s.d_levels, (void*)m.vcur, (void*)m.vnext, (void*)m.front, (void*)m.Q, (void*)m.lint, (void*)m.planes,
                    (void*)m.roots, (void*)m.dirty})
        if (p) cudaFreeAsync(p, s.stream);
    s.d_levels = nullptr;
    m = blest::MsbfsState();
}

// Retire finished launches (caller holds the lock).  Returns true if any.
bool retire(blest_server* sv) {
    bool any = false;
    for (Slot& s : sv->slots) {
        if (!s.busy) continue;
        const cudaError_t q = cudaEventQuery(s.done);
        if (q == cudaErrorNotReady) continue;
        blest_status st = BLEST_OK;
        if (q != cudaSuccess) st = BLEST_ERR_CUDA;
        else if (s.h_status[0]) st = (blest_status)s.h_status[0];
        if (q == cudaSuccess && s.graph >= 0) sv->last_levels[(size_t)s.graph] = (int32_t)s.h_status[1];
        const auto now = clk::now();
        for (Query* r : s.batch) {
            r->status = st;
            r->t_done = now;
            r->done = true;
            sv->queries_done++;
        }
        s.batch.clear();
        free_launch(s);
        sv->mem_used -= s.bytes;
        s.bytes = 0;
        s.busy = false;
        any = true;
    }
    if (any) sv->cv_done.notify_all();
    return any;
}

// Start new launches while slots and memory allow (caller holds the lock).
bool launch_more(blest_server* sv) {
    bool any = false;
    for (;;) {
        Slot* slot = nullptr;
        for (Slot& s : sv->slots)
            if (!s.busy) { slot = &s; break; }
        if (!slot) return any;
        // graph whose oldest waiting query is oldest, passing over long graphs while
        // long_slots launches of long graphs are in flight
        int long_inflight = 0;
        for (const Slot& s : sv->slots) long_inflight += (s.busy && s.long_launch) ? 1 : 0;
        const bool long_full = long_inflight >= sv->p.long_slots;
        int g = -1;
        for (size_t i = 0; i < sv->pending.size(); ++i) {
            if (sv->pending[i].empty() || (long_full && sv->last_levels[i] > sv->p.narrow_levels)) continue;
            if (g < 0 || sv->pending[i].front()->t_submit < sv->pending[g].front()->t_submit) g = (int)i;
        }
        if (g < 0) return any;
        const blest::HandleView& v = sv->views[g];
        std::vector<Query*> batch;
        int k = 0;
        for (Query* r : sv->pending[g]) {
            const int k2 = k + (int)r->roots.size();
            if (k2 > sv->p.max_batch_sources || sv->mem_used + launch_bytes(v, k2) > sv->p.memory_cap_bytes) break;
            if (sv->p.max_queries_per_launch > 0 && (int)batch.size() >= sv->p.max_queries_per_launch) break;
            batch.push_back(r);
            k = k2;
        }
        if (batch.empty()) return any;   // the oldest query waits until memory is returned
        const int64_t bytes = launch_bytes(v, k);
        for (size_t i = 0; i < batch.size(); ++i) sv->pending[g].pop_front();
        std::vector<int32_t> roots;
        roots.reserve((size_t)k);
        for (Query* r : batch) roots.insert(roots.end(), r->roots.begin(), r->roots.end());
        Slot& s = *slot;
        s.batch = batch;
        s.bytes = bytes;
        sv->mem_used += bytes;
        sv->mem_peak = std::max(sv->mem_peak, sv->mem_used);
        s.busy = true;
        s.long_launch = sv->last_levels[(size_t)g] > sv->p.narrow_levels;
        sv->launches++;
        sv->sources_launched += k;
        cudaError_t e = alloc_launch(s, v, k);
        blest::MsbfsLaunchCommon c;
        c.n = v.n;
        c.nss = v.nss;
        c.nvss = v.nvss;
        c.real_ptrs = v.real_ptrs;
        c.row_ids = v.row_ids;
        c.masks = v.masks;
        c.new_id = v.new_id_dev;
        c.ctrl = s.d_ctrl;
        c.sms = v.sms;
        if (sv->p.narrow_sms > 0 && sv->last_levels[(size_t)g] > sv->p.narrow_levels)
            c.sms = std::min(v.sms, sv->p.narrow_sms);
        c.blocks_per_sm = sv->p.blocks_per_sm;
        c.levels_layout = v.levels_layout;
        s.graph = g;
        int rc = 0;
        const char* err = nullptr;
        if (e == cudaSuccess) e = cudaMemsetAsync(s.d_ctrl + kStickyWord, 0, sizeof(unsigned int), s.stream);
        if (e == cudaSuccess) rc = blest::run_msbfs(s.ms, c, roots, s.d_levels, s.stream, &err);
        size_t off = 0;
        for (Query* r : batch) {
            const size_t bytes_r = sizeof(int32_t) * r->roots.size() * (size_t)v.n;
            if (e == cudaSuccess && rc == 0 && r->levels)
                e = cudaMemcpyAsync(r->levels, s.d_levels + off, bytes_r, cudaMemcpyDefault, s.stream);
            off += r->roots.size() * (size_t)v.n;
        }
        if (e == cudaSuccess && rc == 0)
            e = cudaMemcpyAsync(s.h_status, s.d_ctrl + kStickyWord, sizeof(unsigned int), cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess && rc == 0)   // Ctrl::levels of the (last) launch
            e = cudaMemcpyAsync(s.h_status + 1, s.d_ctrl + 6, sizeof(unsigned int), cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess && rc == 0) e = cudaEventRecord(s.done, s.stream);
        if (e != cudaSuccess || rc != 0) {
            // the launch could not be issued: fail its queries now
            cudaStreamSynchronize(s.stream);
            const auto now = clk::now();
            for (Query* r : batch) {
                r->status = rc ? (blest_status)rc : BLEST_ERR_CUDA;
                r->t_done = now;
                r->done = true;
                sv->queries_done++;
            }
            sv->worker_error = err ? err : cudaGetErrorString(e);
            s.batch.clear();
            free_launch(s);
            sv->mem_used -= s.bytes;
            s.bytes = 0;
            s.busy = false;
            sv->cv_done.notify_all();
        }
        any = true;
    }
}

void worker_main(blest_server* sv) {
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        const bool a = retire(sv);
        const bool b = sv->paused ? false : launch_more(sv);
        if (a || b) continue;
        bool inflight = false;
        for (const Slot& s : sv->slots) inflight |= s.busy;
        // poll in-flight launches every 20 microseconds; sleep until a submit when idle
        if (inflight) sv->cv_work.wait_for(lk, std::chrono::microseconds(20));
        else sv->cv_work.wait_for(lk, std::chrono::milliseconds(50));
    }
    // drain: wait for in-flight launches before the slots are released
    for (Slot& s : sv->slots)
        if (s.busy) cudaEventSynchronize(s.done);
    retire(sv);
}

}  // namespace

extern "C" {

blest_status blest_server_create(const blest_handle* graphs, int32_t num_graphs, const blest_server_params* params,
                                 blest_server_handle* out) {
    if (!out) return fail(BLEST_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (num_graphs < 1 || !graphs) return fail(BLEST_ERR_INVALID_ARG, "need at least one graph");
    std::unique_ptr<blest_server> sv(new blest_server());
    sv->p.memory_cap_bytes = params && params->memory_cap_bytes > 0 ? params->memory_cap_bytes : (int64_t)40 << 30;
    sv->p.max_batch_sources = params && params->max_batch_sources > 0 ? params->max_batch_sources : 64;
    sv->p.max_inflight = params && params->max_inflight > 0 ? params->max_inflight : 4;
    sv->p.blocks_per_sm = params && params->blocks_per_sm > 0 ? params->blocks_per_sm : 1;
    sv->p.max_queries_per_launch = params && params->max_queries_per_launch > 0 ? params->max_queries_per_launch : 0;
    sv->p.narrow_sms = params && params->narrow_sms > 0 ? params->narrow_sms : 0;
    sv->p.narrow_levels = params && params->narrow_levels > 0 ? params->narrow_levels : 256;
    sv->p.long_slots = params && params->long_slots > 0 ? params->long_slots : std::max(1, sv->p.max_inflight - 1);
    if (sv->p.max_batch_sources > 256) return fail(BLEST_ERR_INVALID_ARG, "max_batch_sources must be <= 256");
    if (sv->p.max_inflight > 64) return fail(BLEST_ERR_INVALID_ARG, "max_inflight must be <= 64");
    for (int32_t g = 0; g < num_graphs; ++g) {
        blest::HandleView v;
        if (!graphs[g] || !blest::handle_view(graphs[g], &v)) return fail(BLEST_ERR_INVALID_ARG, "bad graph handle");
        sv->graphs.push_back(graphs[g]);
        sv->views.push_back(v);
    }
    sv->pending.resize((size_t)num_graphs);
    sv->last_levels.assign((size_t)num_graphs, 0);
    sv->slots.resize((size_t)sv->p.max_inflight);
    cudaError_t e;
    for (Slot& s : sv->slots) {
        if ((e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaMalloc(&s.d_ctrl, 256)) != cudaSuccess || (e = cudaMemset(s.d_ctrl, 0, 256)) != cudaSuccess ||
            (e = cudaHostAlloc(&s.h_status, 2 * sizeof(unsigned int), cudaHostAllocDefault)) != cudaSuccess) {
            for (Slot& t : sv->slots) {
                if (t.stream) cudaStreamDestroy(t.stream);
                if (t.done) cudaEventDestroy(t.done);
                cudaFree(t.d_ctrl);
                if (t.h_status) cudaFreeHost(t.h_status);
            }
            return fail(e == cudaErrorMemoryAllocation ? BLEST_ERR_OOM : BLEST_ERR_CUDA, cudaGetErrorString(e));
        }
        s.h_status[0] = 0;
        s.h_status[1] = 0;
    }
    blest_server* raw = sv.get();
    int dev = 0;
    cudaGetDevice(&dev);
    raw->dev = dev;
    pool_acquire(dev, raw->p.memory_cap_bytes);
    raw->worker = std::thread([raw, dev]() {
        cudaSetDevice(dev);
        worker_main(raw);
    });
    *out = sv.release();
    return BLEST_OK;
}

blest_status blest_server_submit(blest_server_handle sv, int32_t graph, const int32_t* srcs, int32_t k,
                                 int32_t* levels, uint64_t* ticket) {
    if (!sv || !ticket) return fail(BLEST_ERR_INVALID_ARG, "NULL argument");
    if (graph < 0 || graph >= (int32_t)sv->graphs.size()) return fail(BLEST_ERR_INVALID_ARG, "graph index out of range");
    if (k < 1 || !srcs) return fail(BLEST_ERR_INVALID_ARG, "a query needs at least one source");
    if (k > sv->p.max_batch_sources) return fail(BLEST_ERR_TOO_LARGE, "query has more sources than max_batch_sources");
    const blest::HandleView& v = sv->views[graph];
    if (launch_bytes(v, k) > sv->p.memory_cap_bytes) return fail(BLEST_ERR_TOO_LARGE, "query alone exceeds the memory cap");
    std::unique_ptr<Query> q(new Query());
    q->graph = graph;
    q->roots.resize((size_t)k);
    for (int32_t i = 0; i < k; ++i) {
        if (srcs[i] < 0 || srcs[i] >= v.n) return fail(BLEST_ERR_INVALID_ARG, "source outside [0, n)");
        q->roots[i] = v.new_id_host ? v.new_id_host[srcs[i]] : srcs[i];
    }
    q->levels = levels;
    q->t_submit = clk::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) return fail(BLEST_ERR_INVALID_ARG, "server is shutting down");
        q->ticket = sv->next_ticket++;
        *ticket = q->ticket;
        sv->pending[(size_t)graph].push_back(q.get());
        sv->queries.emplace(q->ticket, std::move(q));
    }
    sv->cv_work.notify_one();
    return BLEST_OK;
}

blest_status blest_server_wait(blest_server_handle sv, uint64_t ticket, double timeout_s, double* latency_s) {
    if (!sv) return fail(BLEST_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->queries.find(ticket);
    if (it == sv->queries.end()) return fail(BLEST_ERR_INVALID_ARG, "unknown ticket");
    Query* q = it->second.get();
    const auto deadline = clk::now() + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(timeout_s));
    while (!q->done) {
        if (timeout_s >= 0 && sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !q->done)
            return fail(BLEST_ERR_TIMEOUT, "query not finished within the wait limit");
        if (timeout_s < 0) sv->cv_done.wait(lk);
    }
    if (latency_s) *latency_s = std::chrono::duration<double>(q->t_done - q->t_submit).count();
    const blest_status st = q->status;
    sv->queries.erase(it);
    if (st != BLEST_OK) return fail(st, "query failed: " + sv->worker_error);
    return BLEST_OK;
}

blest_status blest_server_pause(blest_server_handle sv, int32_t paused) {
    if (!sv) return fail(BLEST_ERR_INVALID_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->paused = paused != 0;
    }
    sv->cv_work.notify_all();
    return BLEST_OK;
}

blest_status blest_server_get_stats(blest_server_handle sv, blest_server_stats* out) {
    if (!sv || !out) return fail(BLEST_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    out->launches = sv->launches;
    out->sources_launched = sv->sources_launched;
    out->queries_done = sv->queries_done;
    out->memory_in_use = sv->mem_used;
    out->memory_peak = sv->mem_peak;
    int64_t waiting = 0;
    for (const auto& d : sv->pending) waiting += (int64_t)d.size();
    out->queries_waiting = waiting;
    return BLEST_OK;
}

void blest_server_destroy(blest_server_handle sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (Slot& s : sv->slots) {
        cudaStreamSynchronize(s.stream);
        cudaStreamDestroy(s.stream);
        cudaEventDestroy(s.done);
        cudaFree(s.d_ctrl);
        cudaFreeHost(s.h_status);
    }
    pool_release(sv->dev);
    delete sv;
}

}  // extern "C"
