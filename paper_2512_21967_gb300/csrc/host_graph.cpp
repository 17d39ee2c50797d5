// Host-side graph preprocessing (see host_graph.h).
#include "host_graph.h"

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <memory>
#include <thread>

#include "../../include/blest.h"

namespace blest {

int host_threads(int requested) {
    if (requested > 0) return std::min(requested, 256);
    unsigned hc = std::thread::hardware_concurrency();
    return hc ? (int)std::min(hc, 256u) : 1;
}

// Run fn(lo, hi) over [0, n) in chunks handed out dynamically to `threads` workers.
template <class F>
static void parallel_chunks(int threads, int64_t n, int64_t chunk, F fn) {
    if (threads <= 1 || n <= chunk) {
        for (int64_t lo = 0; lo < n; lo += chunk) fn(lo, std::min(n, lo + chunk));
        return;
    }
    std::atomic<int64_t> next(0);
    auto worker = [&]() {
        for (;;) {
            int64_t lo = next.fetch_add(chunk);
            if (lo >= n) break;
            fn(lo, std::min(n, lo + chunk));
        }
    };
    std::vector<std::thread> pool;
    int nt = (int)std::min<int64_t>(threads, (n + chunk - 1) / chunk);
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
}

// ------------------------------------------------------------------ cleaning

// Sorts ids in [0, bound): an LSD radix sort in three 10-bit passes (counts stay
// in L1) for long rows when bound <= 2^30, std::sort otherwise.
static void sort_ids(int32_t* a, int64_t len, int64_t bound, std::vector<int32_t>& tmp) {
    if (len <= 1024 || bound > ((int64_t)1 << 30)) {
        std::sort(a, a + len);
        return;
    }
    tmp.resize((size_t)len);
    int32_t* src = a;
    int32_t* dst = tmp.data();
    for (int shift = 0; shift < 30; shift += 10) {
        int64_t cnt[1025] = {0};
        for (int64_t i = 0; i < len; ++i) ++cnt[((uint32_t)src[i] >> shift & 1023u) + 1];
        for (int d = 0; d < 1024; ++d) cnt[d + 1] += cnt[d];
        for (int64_t i = 0; i < len; ++i) dst[cnt[(uint32_t)src[i] >> shift & 1023u]++] = src[i];
        std::swap(src, dst);
    }
    // after three passes (an odd count) the sorted ids are in tmp, where src points
    std::memcpy(a, src, (size_t)len * sizeof(int32_t));
}

int clean_csr(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int threads, Csr& out,
              std::string& err) {
    if (n < 0) { err = "n must be >= 0"; return BLEST_ERR_INVALID_ARG; }
    if (!row_ptr) { err = "row_ptr is NULL"; return BLEST_ERR_INVALID_ARG; }
    if (row_ptr[0] != 0) { err = "row_ptr[0] must be 0"; return BLEST_ERR_INVALID_ARG; }
    for (int64_t u = 0; u < n; ++u)
        if (row_ptr[u + 1] < row_ptr[u]) { err = "row_ptr must be non-decreasing"; return BLEST_ERR_INVALID_ARG; }
    int64_t m = row_ptr[n];
    if (m > 0 && !col_idx) { err = "col_idx is NULL"; return BLEST_ERR_INVALID_ARG; }
    std::atomic<int64_t> bad(-1);
    parallel_chunks(threads, m, 1 << 20, [&](int64_t lo, int64_t hi) {
        for (int64_t e = lo; e < hi; ++e)
            if (col_idx[e] < 0 || col_idx[e] >= n) { bad.store(e); return; }
    });
    if (bad.load() >= 0) { err = "col_idx entry out of range [0, n)"; return BLEST_ERR_INVALID_ARG; }

    out.n = n;
    out.rp.assign((size_t)n + 1, 0);
    std::unique_ptr<int32_t[]> tmp(new int32_t[(size_t)std::max<int64_t>(m, 1)]);   // every entry is written before use
    std::vector<int32_t> newdeg((size_t)n + 1, 0);
    parallel_chunks(threads, n, 4096, [&](int64_t lo, int64_t hi) {
        std::vector<int32_t> scratch;
        for (int64_t u = lo; u < hi; ++u) {
            int32_t* a = tmp.get() + row_ptr[u];
            int64_t len = row_ptr[u + 1] - row_ptr[u];
            if (len > 0) std::memcpy(a, col_idx + row_ptr[u], (size_t)len * sizeof(int32_t));
            if (!std::is_sorted(a, a + len)) sort_ids(a, len, n, scratch);
            int64_t w = 0;
            for (int64_t i = 0; i < len; ++i)
                if (a[i] != (int32_t)u && (w == 0 || a[w - 1] != a[i])) a[w++] = a[i];
            newdeg[u] = (int32_t)w;
        }
    });
    for (int64_t u = 0; u < n; ++u) out.rp[u + 1] = out.rp[u] + newdeg[u];
    out.ci.resize((size_t)out.rp[n]);
    parallel_chunks(threads, n, 4096, [&](int64_t lo, int64_t hi) {
        for (int64_t u = lo; u < hi; ++u)
            if (newdeg[u] > 0)
                std::memcpy(out.ci.data() + out.rp[u], tmp.get() + row_ptr[u], (size_t)newdeg[u] * sizeof(int32_t));
    });
    return BLEST_OK;
}

bool is_symmetric(const Csr& g, int threads, int64_t* bad_u, int64_t* bad_v) {
    // Rows are sorted and hold neither self-loops nor duplicates.  Reversal maps
    // the edges (u, v) with v > u one-to-one onto edges with v < u, so the graph
    // is symmetric iff every such upper edge has its reverse and there are as
    // many upper as lower edges.  The reverse of (u, v) lies in row v below v.
    //
    // Workers take chunks of consecutive rows u in ascending order, so within a
    // chunk the reverses sought in one row v come in ascending order too.  In a
    // long row (a hub, where a binary search misses the cache at most steps) the
    // worker keeps a cursor per chunk: placed by one binary search at the chunk's
    // first visit, then moved forward only.  Short rows are binary-searched.
    constexpr int32_t kHubDeg = 256;
    constexpr int64_t kChunk = 4096;
    std::vector<int32_t> hub_of((size_t)g.n, -1);
    int32_t nhub = 0;
    for (int32_t v = 0; v < g.n; ++v)
        if (g.rp[v + 1] - g.rp[v] >= kHubDeg) hub_of[(size_t)v] = nhub++;
    std::atomic<int64_t> found(-1);
    std::atomic<int64_t> found_v(-1);
    std::atomic<int64_t> upper(0), lower(0);
    std::atomic<int64_t> next(0);
    auto worker = [&]() {
        std::vector<int64_t> cur((size_t)nhub), tag((size_t)nhub, -1);   // cursor and its chunk
        int64_t up = 0, low = 0;
        for (;;) {
            const int64_t lo = next.fetch_add(kChunk);
            if (lo >= g.n || found.load(std::memory_order_relaxed) >= 0) break;
            const int64_t hi = std::min<int64_t>(g.n, lo + kChunk);
            for (int64_t u = lo; u < hi && found.load(std::memory_order_relaxed) < 0; ++u) {
                const int32_t* rb = g.ci.data() + g.rp[u];
                const int32_t* re = g.ci.data() + g.rp[u + 1];
                const int32_t* mid = std::upper_bound(rb, re, (int32_t)u);   // first neighbour above u
                low += mid - rb;
                up += re - mid;
                for (const int32_t* p = mid; p < re; ++p) {
                    const int32_t v = *p;
                    const int32_t* b = g.ci.data() + g.rp[v];
                    const int32_t* en = g.ci.data() + g.rp[v + 1];
                    bool ok;
                    const int32_t h = hub_of[(size_t)v];
                    if (h >= 0) {
                        int64_t c = cur[(size_t)h];
                        if (tag[(size_t)h] != lo) {
                            c = std::lower_bound(b, en, (int32_t)u) - b;
                            tag[(size_t)h] = lo;
                        }
                        while (b + c < en && b[c] < (int32_t)u) ++c;
                        cur[(size_t)h] = c;
                        ok = b + c < en && b[c] == (int32_t)u;
                    } else {
                        ok = std::binary_search(b, en, (int32_t)u);
                    }
                    if (!ok) { found.store(u); found_v.store(v); break; }
                }
            }
        }
        upper += up;
        lower += low;
    };
    {
        const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(threads, (g.n + kChunk - 1) / kChunk));
        std::vector<std::thread> pool;
        for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
        worker();
        for (auto& th : pool) th.join();
    }
    if (found.load() < 0 && upper.load() != lower.load()) {
        // some lower edge (u, v) has no reverse: find one for the message
        parallel_chunks(threads, g.n, 4096, [&](int64_t lo, int64_t hi) {
            for (int64_t u = lo; u < hi && found.load(std::memory_order_relaxed) < 0; ++u)
                for (int64_t e = g.rp[u]; e < g.rp[u + 1]; ++e) {
                    const int32_t v = g.ci[e];
                    if (v >= u) break;
                    const int32_t* b = g.ci.data() + g.rp[v];
                    const int32_t* en = g.ci.data() + g.rp[v + 1];
                    if (!std::binary_search(b, en, (int32_t)u)) { found.store(u); found_v.store(v); break; }
                }
        });
    }
    if (found.load() >= 0) {
        if (bad_u) *bad_u = found.load();
        if (bad_v) *bad_v = found_v.load();
        return false;
    }
    return true;
}

void relabel_csr(const Csr& g, const std::vector<int32_t>& new_id, int threads, Csr& out) {
    int32_t n = g.n;
    std::vector<int32_t> old_of((size_t)n);
    for (int32_t v = 0; v < n; ++v) old_of[new_id[v]] = v;
    out.n = n;
    out.rp.assign((size_t)n + 1, 0);
    for (int32_t w = 0; w < n; ++w) {
        int32_t v = old_of[w];
        out.rp[w + 1] = out.rp[w] + (g.rp[v + 1] - g.rp[v]);
    }
    out.ci.resize((size_t)out.rp[n]);
    parallel_chunks(threads, n, 4096, [&](int64_t lo, int64_t hi) {
        std::vector<int32_t> tmp;
        for (int64_t w = lo; w < hi; ++w) {
            int32_t v = old_of[w];
            int32_t* dst = out.ci.data() + out.rp[w];
            int64_t len = g.rp[v + 1] - g.rp[v];
            for (int64_t i = 0; i < len; ++i) dst[i] = new_id[g.ci[g.rp[v] + i]];
            sort_ids(dst, len, n, tmp);
        }
    });
}

// -------------------------------------------------------------------- RCM
// Section 3.2.1 uses RCM as a bandwidth-reducing order.  Each component (in
// order of its smallest id) starts at a George-Liu pseudo-peripheral vertex;
// unvisited neighbours are queued in ascending (degree, id); the whole
// Cuthill-McKee sequence is reversed at the end.

namespace {
// Spin barrier for a fixed set of host threads (sense by generation count).
class SpinBarrier {
  public:
    explicit SpinBarrier(int n) : n_(n) {}
    void wait() {
        const unsigned gen = gen_.load(std::memory_order_acquire);
        if (arrived_.fetch_add(1, std::memory_order_acq_rel) + 1 == n_) {
            arrived_.store(0, std::memory_order_relaxed);
            gen_.fetch_add(1, std::memory_order_acq_rel);
            return;
        }
        for (unsigned spins = 0; gen_.load(std::memory_order_acquire) == gen; ++spins)
            if (spins > 1024) std::this_thread::yield();
    }

  private:
    const int n_;
    std::atomic<int> arrived_{0};
    std::atomic<unsigned> gen_{0};
};

// BFS that only needs the set of vertices on each level (the eccentricity and
// the last level), not a visit order: levels are expanded sequentially while the
// frontier is small and by `threads` host threads, each claiming vertices with a
// compare-and-swap on their stamp, once a frontier holds kParallelFrontier
// vertices.  queue[0..count) holds the vertices level by level.
struct LevelBfs {
    static constexpr int64_t kParallelFrontier = 1024;
    struct Mark {
        int32_t stamp, level;
    };
    std::vector<Mark> mark;
    std::vector<int32_t> queue;
    int32_t cur = 0;
    int threads = 1;
    LevelBfs(int32_t n, int t) : mark((size_t)n, Mark{0, 0}), queue((size_t)std::max(n, 1)), threads(t) {}
    int32_t level(int32_t v) const { return mark[(size_t)v].level; }

    // returns the eccentricity of root
    int32_t run(const Csr& g, int32_t root, int64_t& count) {
        ++cur;
        int64_t head = 0, tail = 0, lvl_end = 1;
        int32_t lvl = 0;
        mark[root] = Mark{cur, 0};
        queue[tail++] = root;
        while (head < tail) {
            if (head == lvl_end) {   // a level boundary
                ++lvl;
                lvl_end = tail;
                if (threads > 1 && lvl_end - head >= kParallelFrontier) {
                    tail = parallel_levels(g, head, tail, lvl);
                    break;
                }
            }
            const int32_t u = queue[head++];
            for (int32_t e = g.rp[u]; e < g.rp[u + 1]; ++e) {
                const int32_t v = g.ci[e];
                if (mark[v].stamp != cur) {
                    mark[v] = Mark{cur, lvl + 1};
                    queue[tail++] = v;
                }
            }
        }
        count = tail;
        return mark[queue[tail - 1]].level;
    }

    // Expands the frontier queue[lo, hi) (level lvl) and every later level with
    // all threads; returns the new tail.
    int64_t parallel_levels(const Csr& g, int64_t lo, int64_t hi, int32_t lvl) {
        const int T = threads;
        std::vector<std::vector<int32_t>> found((size_t)T);
        std::vector<int64_t> sizes((size_t)T, 0);
        std::atomic<int64_t> next(0);
        int64_t end = hi;
        SpinBarrier bar(T);
        auto worker = [&](int t) {
            int64_t fs = lo, fe = hi;   // the current frontier (each thread keeps its own copy)
            int32_t l = lvl;
            std::vector<int32_t>& out = found[(size_t)t];
            for (;;) {
                out.clear();
                for (;;) {
                    const int64_t c = fs + next.fetch_add(256, std::memory_order_relaxed);
                    if (c >= fe) break;
                    const int64_t c_end = std::min<int64_t>(c + 256, fe);
                    for (int64_t i = c; i < c_end; ++i) {
                        const int32_t u = queue[(size_t)i];
                        for (int32_t e = g.rp[u]; e < g.rp[u + 1]; ++e) {
                            const int32_t v = g.ci[e];
                            int32_t seen = __atomic_load_n(&mark[v].stamp, __ATOMIC_RELAXED);
                            if (seen == cur) continue;
                            if (__atomic_compare_exchange_n(&mark[v].stamp, &seen, cur, false, __ATOMIC_RELAXED,
                                                            __ATOMIC_RELAXED)) {
                                mark[v].level = l + 1;
                                out.push_back(v);
                            }
                        }
                    }
                }
                sizes[(size_t)t] = (int64_t)out.size();
                bar.wait();   // every thread's share of the next level is in `found`
                int64_t off = fe, total = 0;
                for (int i = 0; i < T; ++i) {
                    if (i < t) off += sizes[(size_t)i];
                    total += sizes[(size_t)i];
                }
                if (!out.empty()) std::memcpy(&queue[(size_t)off], out.data(), out.size() * sizeof(int32_t));
                if (t == 0) next.store(0, std::memory_order_relaxed);
                bar.wait();   // the next level is in the queue and the chunk counter is reset
                if (total == 0) {
                    if (t == 0) end = fe;
                    return;
                }
                fs = fe;
                fe += total;
                ++l;
            }
        };
        std::vector<std::thread> pool;
        for (int t = 1; t < T; ++t) pool.emplace_back(worker, t);
        worker(0);
        for (auto& th : pool) th.join();
        return end;
    }
};
}  // namespace

// One level of a FIFO-order BFS: appends to queue[tail..), for i = fs .. fe-1 in
// order, the neighbours of queue[i] that are not yet seen and not taken by an
// earlier position, each group in the order arrange(u, first, last) leaves it,
// and marks them seen.  Returns the new tail.
template <class Arrange>
static int64_t expand_level_fifo(const Csr& g, int32_t* queue, int64_t fs, int64_t fe, int64_t tail,
                                 std::vector<uint8_t>& seen, Arrange arrange) {
    for (int64_t i = fs; i < fe; ++i) {
        const int32_t u = queue[i];
        const int64_t first = tail;
        for (int32_t e = g.rp[u]; e < g.rp[u + 1]; ++e) {
            const int32_t v = g.ci[e];
            if (!seen[(size_t)v]) { seen[(size_t)v] = 1; queue[tail++] = v; }
        }
        arrange(u, queue + first, queue + tail);
    }
    return tail;
}

// Every remaining level of one component's FIFO-order BFS, queue[fs, tail) being
// the current frontier: the same result as expand_level_fifo level after level.
// Levels run sequentially until one holds kPoolLevel positions; from then on
// `threads` host threads stay alive for the rest of the component and meet at
// spin barriers, so that a high-diameter graph's thousands of mid-sized levels
// do not each pay thread launches.  A pooled level of kPoolLevel positions or
// more is expanded by all threads: every unseen neighbour belongs to the
// smallest position that reaches it (an atomic minimum in owner[], which holds
// INT32_MAX for every vertex not yet owned), and each position writes its group
// at an offset from a prefix sum of group sizes; smaller levels run on thread 0.
// Returns the new tail.
template <class Arrange>
static int64_t fifo_component(const Csr& g, int32_t* queue, int64_t fs, int64_t tail, std::vector<uint8_t>& seen,
                              std::vector<int32_t>& owner, int threads, Arrange arrange) {
    constexpr int64_t kPoolLevel = 1024;
    constexpr int64_t kChunk = 256;
    while (fs < tail && (threads <= 1 || tail - fs < kPoolLevel)) {
        const int64_t fe = tail;
        tail = expand_level_fifo(g, queue, fs, fe, tail, seen, arrange);
        fs = fe;
    }
    if (fs >= tail) return tail;
    const int T = threads;
    SpinBarrier bar(T);
    std::atomic<int64_t> next_own(0), next_count(0), next_place(0), next_seen(0);
    std::vector<int64_t> off;                // group offsets of the current level's positions
    int64_t lvl_fs = fs, lvl_fe = tail;      // the current level; written by thread 0 between barriers
    int64_t new_tail = tail;
    bool done = false;
    auto worker = [&](int t) {
        for (;;) {
            const int64_t s = lvl_fs, e = lvl_fe, L = e - s;
            if (L < kPoolLevel) {
                if (t == 0) new_tail = expand_level_fifo(g, queue, s, e, e, seen, arrange);
            } else {
                for (;;) {   // owners
                    const int64_t c = s + next_own.fetch_add(kChunk, std::memory_order_relaxed);
                    if (c >= e) break;
                    for (int64_t i = c, ce = std::min(c + kChunk, e); i < ce; ++i) {
                        const int32_t u = queue[i];
                        for (int32_t x = g.rp[u]; x < g.rp[u + 1]; ++x) {
                            const int32_t v = g.ci[x];
                            if (seen[(size_t)v]) continue;
                            int32_t cur = __atomic_load_n(&owner[(size_t)v], __ATOMIC_RELAXED);
                            while ((int32_t)i < cur &&
                                   !__atomic_compare_exchange_n(&owner[(size_t)v], &cur, (int32_t)i, true,
                                                                __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
                            }
                        }
                    }
                }
                bar.wait();
                for (;;) {   // group sizes
                    const int64_t c = s + next_count.fetch_add(kChunk, std::memory_order_relaxed);
                    if (c >= e) break;
                    for (int64_t i = c, ce = std::min(c + kChunk, e); i < ce; ++i) {
                        const int32_t u = queue[i];
                        int64_t k = 0;
                        for (int32_t x = g.rp[u]; x < g.rp[u + 1]; ++x) {
                            const int32_t v = g.ci[x];
                            k += !seen[(size_t)v] && owner[(size_t)v] == (int32_t)i;
                        }
                        off[(size_t)(i - s) + 1] = k;
                    }
                }
                bar.wait();
                if (t == 0) {
                    off[0] = 0;
                    for (int64_t k = 1; k <= L; ++k) off[(size_t)k] += off[(size_t)k - 1];
                    new_tail = e + off[(size_t)L];
                }
                bar.wait();
                for (;;) {   // groups, each arranged
                    const int64_t c = s + next_place.fetch_add(kChunk, std::memory_order_relaxed);
                    if (c >= e) break;
                    for (int64_t i = c, ce = std::min(c + kChunk, e); i < ce; ++i) {
                        const int32_t u = queue[i];
                        int32_t* first = queue + e + off[(size_t)(i - s)];
                        int32_t* w = first;
                        for (int32_t x = g.rp[u]; x < g.rp[u + 1]; ++x) {
                            const int32_t v = g.ci[x];
                            if (!seen[(size_t)v] && owner[(size_t)v] == (int32_t)i) *w++ = v;
                        }
                        arrange(u, first, w);
                    }
                }
                bar.wait();
                for (;;) {   // the new level is seen
                    const int64_t c = e + next_seen.fetch_add(kChunk, std::memory_order_relaxed);
                    if (c >= new_tail) break;
                    for (int64_t k = c, ce = std::min(c + kChunk, new_tail); k < ce; ++k)
                        seen[(size_t)queue[k]] = 1;
                }
            }
            bar.wait();
            if (t == 0) {   // the next level
                next_own.store(0, std::memory_order_relaxed);
                next_count.store(0, std::memory_order_relaxed);
                next_place.store(0, std::memory_order_relaxed);
                next_seen.store(0, std::memory_order_relaxed);
                lvl_fs = e;
                lvl_fe = new_tail;
                done = new_tail == e;
                if ((int64_t)off.size() < new_tail - e + 1) off.resize((size_t)(new_tail - e + 1));
            }
            bar.wait();
            if (done) return;
        }
    };
    if ((int64_t)off.size() < tail - fs + 1) off.resize((size_t)(tail - fs + 1));
    std::vector<std::thread> pool;
    for (int t = 1; t < T; ++t) pool.emplace_back(worker, t);
    worker(0);
    for (auto& th : pool) th.join();
    return lvl_fe;
}

static int32_t pseudo_peripheral(const Csr& g, LevelBfs& bfs, int32_t start) {
    int32_t x = start;
    int64_t cnt = 0;
    int32_t ex = bfs.run(g, x, cnt);
    for (;;) {
        int32_t y = -1;
        for (int64_t i = 0; i < cnt; ++i) {
            int32_t v = bfs.queue[i];
            if (bfs.level(v) != ex) continue;
            if (y < 0) { y = v; continue; }
            int32_t dv = g.rp[v + 1] - g.rp[v], dy = g.rp[y + 1] - g.rp[y];
            if (dv < dy || (dv == dy && v < y)) y = v;
        }
        int64_t cy = 0;
        int32_t ey = bfs.run(g, y, cy);
        if (ey > ex) {
            x = y; ex = ey; cnt = cy;
        } else {
            return x;
        }
    }
}

void order_rcm(const Csr& g, std::vector<int32_t>& new_id, int threads) {
    int32_t n = g.n;
    new_id.assign((size_t)n, 0);
    if (n == 0) return;
    LevelBfs bfs(n, threads);
    std::vector<uint8_t> seen((size_t)n, 0);
    std::vector<int32_t> order((size_t)n), owner((size_t)n, INT32_MAX);
    int64_t tail = 0;
    // each vertex's unvisited neighbours join the queue by ascending (degree, id)
    auto by_degree = [&](int32_t, int32_t* first, int32_t* last) {
        std::sort(first, last, [&](int32_t a, int32_t b) {
            int32_t da = g.rp[a + 1] - g.rp[a], db = g.rp[b + 1] - g.rp[b];
            return da != db ? da < db : a < b;
        });
    };
    for (int32_t v0 = 0; v0 < n; ++v0) {
        if (seen[v0]) continue;
        if (g.rp[v0 + 1] == g.rp[v0]) {   // an isolated vertex is its own component and its own order
            seen[v0] = 1;
            order[(size_t)tail++] = v0;
            continue;
        }
        int32_t r = pseudo_peripheral(g, bfs, v0);
        seen[r] = 1;
        const int64_t fs = tail;
        order[(size_t)tail++] = r;
        // level by level, in the FIFO order of the sequential method
        tail = fifo_component(g, order.data(), fs, tail, seen, owner, threads, by_degree);
    }
    for (int64_t pos = 0; pos < n; ++pos) new_id[order[pos]] = (int32_t)(n - 1 - pos);
}

// ------------------------------------------------------------ hub pre-pass
// Stand-in for the Gorder pre-pass of Section 3.2: BFS visit order, every
// component rooted at the highest-degree unvisited vertex (smallest id on
// ties), neighbours scanned in ascending id.  Neighbours of the same hub land
// in the same window of Algorithm 1.

void order_hub_prepass(const Csr& g, std::vector<int32_t>& new_id, int threads) {
    int32_t n = g.n;
    new_id.assign((size_t)n, 0);
    // roots by descending degree, ascending id within a degree (a counting sort)
    int32_t dmax = 0;
    for (int32_t v = 0; v < n; ++v) dmax = std::max(dmax, g.rp[v + 1] - g.rp[v]);
    std::vector<int64_t> start((size_t)dmax + 2, 0);
    for (int32_t v = 0; v < n; ++v) ++start[(size_t)(dmax - (g.rp[v + 1] - g.rp[v])) + 1];
    for (size_t d = 1; d < start.size(); ++d) start[d] += start[d - 1];
    std::vector<int32_t> cand((size_t)n);
    for (int32_t v = 0; v < n; ++v) cand[(size_t)start[(size_t)(dmax - (g.rp[v + 1] - g.rp[v]))]++] = v;
    std::vector<uint8_t> seen((size_t)n, 0);
    std::vector<int32_t> order((size_t)n), owner((size_t)n, INT32_MAX);
    int64_t tail = 0;
    auto as_listed = [](int32_t, int32_t*, int32_t*) {};   // neighbours in ascending id, as stored
    for (int32_t r : cand) {
        if (seen[r]) continue;
        seen[r] = 1;
        const int64_t fs = tail;
        order[(size_t)tail++] = r;
        tail = fifo_component(g, order.data(), fs, tail, seen, owner, threads, as_listed);
    }
    for (int32_t pos = 0; pos < n; ++pos) new_id[order[pos]] = pos;
}

// --------------------------------------------------------------- Gorder
// The pre-pass Section 3.2 names (Wei, Yu, Lu, Lin, SIGMOD 2016), restated from
// its published definition: place next the unplaced vertex with the largest
// score summed over the last w placed vertices, S(u, v) = 2 [u ~ v] (edges in
// both directions of a symmetric graph) + the common neighbours of u and v of
// degree <= hub_cap.  The first vertex has the largest degree; ties go to the
// smallest id.  Scores change by +-1 steps when a vertex enters or leaves the
// window, so they are updated incrementally (through the vertex's neighbours
// and, for neighbours of degree <= hub_cap, their neighbours), and a max
// segment tree over vertex ids (key, then smaller id) finds the next vertex.
void order_gorder(const Csr& g, int w, int32_t hub_cap, std::vector<int32_t>& new_id) {
    const int32_t n = g.n;
    new_id.assign((size_t)n, 0);
    if (n == 0) return;
    int32_t size = 1;
    while (size < n) size <<= 1;
    std::vector<int64_t> key((size_t)n, 0);
    std::vector<uint8_t> placed((size_t)n, 0);
    std::vector<int32_t> tree(2 * (size_t)size, -1);   // leaf = vertex id or -1 (none)
    auto better = [&](int32_t a, int32_t b) {          // a beats b
        if (a < 0) return false;
        if (b < 0) return true;
        return key[a] != key[b] ? key[a] > key[b] : a < b;
    };
    // point update after v's key or placement changed; a node whose winner stays
    // the same and is not v leaves every ancestor's comparison as it was
    auto fix = [&](int32_t v) {
        size_t i = (size_t)size + (size_t)v;
        tree[i] = placed[v] ? -1 : v;
        for (i >>= 1; i >= 1; i >>= 1) {
            const int32_t l = tree[2 * i], r = tree[2 * i + 1];
            const int32_t win = better(l, r) ? l : (r >= 0 ? r : l);
            if (win == tree[i] && win != v) break;
            tree[i] = win;
        }
    };
    for (int32_t v = 0; v < n; ++v) { key[v] = g.rp[v + 1] - g.rp[v]; tree[(size_t)size + v] = v; }
    for (size_t i = (size_t)size - 1; i >= 1; --i) {
        const int32_t l = tree[2 * i], r = tree[2 * i + 1];
        tree[i] = better(l, r) ? l : (r >= 0 ? r : l);
    }
    // the first vertex is chosen on degree; after it every key starts at 0
    const int32_t first = tree[1];
    std::fill(key.begin(), key.end(), 0);
    for (int32_t v = 0; v < n; ++v) tree[(size_t)size + v] = v;
    for (size_t i = (size_t)size - 1; i >= 1; --i) {
        const int32_t l = tree[2 * i], r = tree[2 * i + 1];
        tree[i] = better(l, r) ? l : (r >= 0 ? r : l);
    }
    std::vector<int32_t> order;
    order.reserve((size_t)n);
    std::vector<int32_t> touched;
    std::vector<int32_t> seen_at((size_t)n, -1);   // the step that last listed a vertex in touched
    int32_t step = 0;
    auto touch = [&](int32_t u) {
        if (seen_at[(size_t)u] != step) { seen_at[(size_t)u] = step; touched.push_back(u); }
    };
    auto contribute = [&](int32_t v, int64_t sign) {
        for (int32_t e = g.rp[v]; e < g.rp[v + 1]; ++e) {
            const int32_t x = g.ci[e];
            if (!placed[x]) { key[x] += 2 * sign; touch(x); }
            if (g.rp[x + 1] - g.rp[x] > hub_cap) continue;
            for (int32_t f = g.rp[x]; f < g.rp[x + 1]; ++f) {
                const int32_t u = g.ci[f];
                if (u != v && !placed[u]) { key[u] += sign; touch(u); }
            }
        }
    };
    auto place = [&](int32_t v) {
        placed[v] = 1;
        fix(v);
        order.push_back(v);
    };
    place(first);
    while ((int32_t)order.size() < n) {
        touched.clear();
        ++step;
        contribute(order.back(), +1);
        if ((int)order.size() > w) contribute(order[order.size() - 1 - (size_t)w], -1);
        for (int32_t u : touched) fix(u);
        place(tree[1]);
    }
    for (int32_t pos = 0; pos < n; ++pos) new_id[order[pos]] = pos;
}

// ------------------------------------------------------- JaccardWithWindows
// Algorithm 1.  Windows [s_k, e_k) of at most w ids are independent and run in
// parallel.  Inside a window: M_k = ceil(L_k / sigma) clusters; each starts at
// the smallest remaining id (pop(Q)), then sigma-1 times adds the remaining
// vertex j maximising J = |N(j) & U| / |N(j) | U| (exact rational comparison,
// smallest id on ties), U growing by N(j).
//
// The counts c[j] = |N(j) & U| are kept incrementally: when a vertex x joins U,
// every window member adjacent to x gets c[j] + 1 (a window-local reverse
// index x -> {j in window : x in N(j)} makes that a list walk).  Members with
// c[j] = 0 all have J = 0, so when no member has c[j] > 0 the smallest
// remaining id is chosen, as the argmax tie rule says.

namespace {
template <class Pos>   // type of a window position in the reverse lists (uint16_t when windows fit)
struct JaccardWorker {
    const Csr& g;
    const int32_t* row_at;   // window position -> row of g (NULL: the identity)
    int sigma;
    std::vector<int32_t> c;        // scratch of build_index
    // per window row: (cluster stamp << 32) | |N(j) & U|, one word per row so that a
    // list walk reads and writes one array; the count is current iff the stamp is
    std::vector<uint64_t> cs;
    std::vector<int32_t> wdeg;   // degree of each window row (read at every pick)
    std::vector<uint8_t> inq;
    std::vector<int32_t> touched;
    // Reverse index of the window: neighbour x -> the window rows that hold x.
    // An open-addressing table keyed by x, built once per window, gives each x
    // its list in revj (hoff, hlen); rows already placed are dropped from a list
    // as it is walked.  Every neighbour of a window row has a slot, so the slot
    // also records (ustamp) the cluster whose U holds x: no per-vertex array per
    // thread.
    std::vector<int32_t> hkey, hoff, hlen, ustamp;
    std::vector<Pos> revj;
    // eslot[eoff[jl] + k]: the slot of the k-th neighbour of window row jl, found
    // once while the table is built
    std::vector<int32_t> eslot;
    std::vector<int64_t> eoff;
    int hshift = 60;
    int32_t stamp = 0;

    JaccardWorker(const Csr& gr, const int32_t* at, int s) : g(gr), row_at(at), sigma(s) {}

    int32_t row(int32_t pos) const { return row_at ? row_at[pos] : pos; }
    int32_t deg(int32_t pos) const { const int32_t r = row(pos); return g.rp[r + 1] - g.rp[r]; }

    // Fibonacci hashing: the high bits of x times 2^64 / golden ratio
    size_t slot0(int32_t x) const { return (size_t)(((uint64_t)(uint32_t)x * 0x9E3779B97F4A7C15ull) >> hshift); }

    void build_index(int32_t s_k, int32_t L) {
        int64_t nnz = 0;
        for (int32_t jl = 0; jl < L; ++jl) nnz += deg(s_k + jl);
        const int64_t distinct_max = std::min<int64_t>(nnz, g.n);
        size_t cap = 16;
        hshift = 60;
        while ((int64_t)cap < 2 * distinct_max) { cap <<= 1; --hshift; }   // load factor <= 1/2
        const size_t mask = cap - 1;
        hkey.assign(cap, -1);
        hlen.assign(cap, 0);
        ustamp.assign(cap, 0);
        hoff.resize(cap);
        eslot.resize((size_t)nnz);
        eoff.resize((size_t)L + 1);
        int64_t k = 0;
        for (int32_t jl = 0; jl < L; ++jl) {
            eoff[(size_t)jl] = k;
            const int32_t r = row(s_k + jl);
            for (int32_t e = g.rp[r]; e < g.rp[r + 1]; ++e) {
                const int32_t x = g.ci[e];
                size_t h = slot0(x);
                while (hkey[h] >= 0 && hkey[h] != x) h = (h + 1) & mask;
                hkey[h] = x;
                ++hlen[h];
                eslot[(size_t)k++] = (int32_t)h;
            }
        }
        eoff[(size_t)L] = k;
        int32_t run = 0;
        for (size_t h = 0; h < cap; ++h) { hoff[h] = run; run += hlen[h]; }
        revj.resize((size_t)nnz);
        std::vector<int32_t>& fill = c;   // scratch: per-slot fill position
        fill.assign(cap, 0);
        for (int32_t jl = 0; jl < L; ++jl)
            for (int64_t i = eoff[(size_t)jl]; i < eoff[(size_t)jl + 1]; ++i) {
                const size_t h = (size_t)eslot[(size_t)i];
                revj[(size_t)(hoff[h] + fill[h]++)] = (Pos)jl;   // rows in ascending order per x
            }
    }

    int32_t s_k_ = 0;   // first position of the current window

    void window(int32_t s_k, int32_t e_k, int32_t* new_id) {
        int32_t L = e_k - s_k;
        s_k_ = s_k;
        build_index(s_k, L);
        wdeg.resize((size_t)L);
        for (int32_t jl = 0; jl < L; ++jl) wdeg[(size_t)jl] = deg(s_k + jl);
        cs.assign((size_t)L, 0);
        inq.assign((size_t)L, 1);

        int32_t qptr = 0, remaining = L;
        int32_t M = (L + sigma - 1) / sigma;
        for (int32_t ell = 0; ell < M; ++ell) {
            while (!inq[qptr]) ++qptr;
            int32_t js = qptr;
            inq[js] = 0; --remaining;
            new_id[s_k + js] = s_k + ell * sigma;
            ++stamp;
            if (stamp == 0x7fffffff) {  // stamp wrap: reset the marks
                std::fill(ustamp.begin(), ustamp.end(), 0);
                std::fill(cs.begin(), cs.end(), 0);
                stamp = 1;
            }
            int64_t usize = 0;
            touched.clear();
            add_to_u(s_k + js, usize);
            for (int r = 1; r < sigma; ++r) {
                if (remaining == 0) break;
                int32_t best = -1;
                int64_t bnum = 0, bden = 1;
                for (int32_t jl : touched) {
                    if (!inq[jl]) continue;
                    int64_t num = (int64_t)(uint32_t)cs[(size_t)jl];
                    int64_t den = (int64_t)wdeg[(size_t)jl] + usize - num;
                    // num > 0 here, so den >= 1
                    bool better = best < 0 || num * bden > bnum * den || (num * bden == bnum * den && jl < best);
                    if (better) { best = jl; bnum = num; bden = den; }
                }
                if (best < 0) {
                    while (!inq[qptr]) ++qptr;
                    best = qptr;
                }
                inq[best] = 0; --remaining;
                new_id[s_k + best] = s_k + ell * sigma + r;
                add_to_u(s_k + best, usize);
            }
        }
    }

    // U gains j's neighbours; every unplaced row sharing a new one gets c += 1.
    // The pick above is the best ratio with ties to the smallest row, so it does
    // not depend on the order in which rows are touched or listed.
    void add_to_u(int32_t pos, int64_t& usize) {
        const int32_t jl0 = pos - s_k_;
        for (int64_t i = eoff[(size_t)jl0]; i < eoff[(size_t)jl0 + 1]; ++i) {
            const size_t h = (size_t)eslot[(size_t)i];
            if (ustamp[h] == stamp) continue;
            ustamp[h] = stamp;
            ++usize;
            int32_t w = hoff[h];
            for (int32_t i = hoff[h], end = hoff[h] + hlen[h]; i < end; ++i) {
                const int32_t jl = revj[i];
                if (!inq[jl]) continue;   // placed rows leave the list
                revj[w++] = (Pos)jl;
                const uint64_t x = cs[jl];
                if ((uint32_t)(x >> 32) != (uint32_t)stamp) {
                    cs[jl] = ((uint64_t)(uint32_t)stamp << 32) | 1u;
                    touched.push_back(jl);
                } else {
                    cs[jl] = x + 1u;
                }
            }
            hlen[h] = w - hoff[h];
        }
    }
};
}  // namespace

void order_jaccard_windows(const Csr& g, int sigma, int32_t window, int threads, std::vector<int32_t>& new_id,
                           const int32_t* row_at) {
    int32_t n = g.n;
    new_id.assign((size_t)n, 0);
    if (n == 0) return;
    int64_t nwin = ((int64_t)n + window - 1) / window;
    int nt = (int)std::min<int64_t>(threads, nwin);
    if (nt < 1) nt = 1;
    std::atomic<int64_t> next(0);
    auto run = [&](auto& wk) {
        for (;;) {
            int64_t k = next.fetch_add(1);
            if (k >= nwin) break;
            int32_t s_k = (int32_t)(k * window);
            int32_t e_k = (int32_t)std::min<int64_t>((int64_t)s_k + window, n);
            wk.window(s_k, e_k, new_id.data());
        }
    };
    auto work = [&]() {
        if (window <= 65536) {   // positions fit 16 bits: half the bytes in every list walk
            JaccardWorker<uint16_t> wk(g, row_at, sigma);
            run(wk);
        } else {
            JaccardWorker<int32_t> wk(g, row_at, sigma);
            run(wk);
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (auto& th : pool) th.join();
}

void order_compress(const Csr& g, int sigma, int32_t window, int threads, std::vector<int32_t>& new_id,
                    int prepass) {
    std::vector<int32_t> pre;
    if (prepass == 1) order_gorder(g, 5, 64, pre);
    else order_hub_prepass(g, pre, threads);
    // Algorithm 1 over the pre-pass order, reading g's rows through the
    // permutation: neighbours only need to compare equal, and ties go to the
    // smaller window position, so no relabelled copy of g is needed
    std::vector<int32_t> at((size_t)g.n);
    for (int32_t v = 0; v < g.n; ++v) at[(size_t)pre[v]] = v;
    std::vector<int32_t> jw;
    order_jaccard_windows(g, sigma, window, threads, jw, at.data());
    new_id.resize((size_t)g.n);
    for (int32_t v = 0; v < g.n; ++v) new_id[v] = jw[pre[v]];
}

// ------------------------------------------------------------ classifier

bool is_social_like(const Csr& g) {
    int32_t n = g.n;
    if (n == 0) return false;
    std::vector<int64_t> deg((size_t)n);
    int64_t total = 0;
    for (int32_t v = 0; v < n; ++v) { deg[v] = g.rp[v + 1] - g.rp[v]; total += deg[v]; }
    if (total == 0) return false;
    std::vector<int64_t> sorted = deg;
    std::sort(sorted.begin(), sorted.end(), std::greater<int64_t>());
    int64_t k1 = std::max<int64_t>(1, (n + 99) / 100), k10 = std::max<int64_t>(1, (n + 9) / 10);
    int64_t s1 = 0, s10 = 0;
    for (int64_t i = 0; i < k10; ++i) { if (i < k1) s1 += sorted[i]; s10 += sorted[i]; }
    // "more than 5% / 40%" as exact integer comparisons
    bool heavy = 20 * s1 > total && 5 * s10 > 2 * total;
    if (heavy) return true;
    // log-log degree histogram, least-squares line over degrees >= 1
    int64_t dmax = sorted[0];
    std::vector<int64_t> hist((size_t)dmax + 1, 0);
    for (int64_t d : deg) hist[d]++;
    double sx = 0, sy = 0, sxx = 0, sxy = 0, syy = 0;
    int pts = 0;
    for (int64_t d = 1; d <= dmax; ++d) {
        if (!hist[d]) continue;
        double x = std::log((double)d), y = std::log((double)hist[d]);
        sx += x; sy += y; sxx += x * x; sxy += x * y; syy += y * y; ++pts;
    }
    if (pts < 5) return false;
    double vx = sxx - sx * sx / pts, vy = syy - sy * sy / pts, cxy = sxy - sx * sy / pts;
    if (vx <= 0 || vy <= 0) return false;
    double slope = cxy / vx;
    double r2 = cxy * cxy / (vx * vy);
    return slope >= -3.5 && slope <= -1.5 && r2 >= 0.8;
}

}  // namespace blest
