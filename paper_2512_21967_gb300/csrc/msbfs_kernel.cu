// Multi-source BFS as a Boolean SpMM over BVSS (Section 2: k frontiers stacked
// column-wise form an n x k frontier matrix).  One persistent cooperative
// launch runs up to 256 sources; each vertex carries W = ceil(k / 64) 64-bit
// words of frontier and of visited bits.  Per level:
//   stage 1: warps take queued virtual slice sets round-robin, with the next
//     item's tile and frontier words (and the entry after it) loaded while the
//     current one is pulled; tiles stream past L1 with an evict-first L2 policy.
//     The 8 x k frontier tile of the slice set (8 W words) is loaded once per VSS
//     by 8 W lanes and broadcast by shuffles; each lane ORs, for each of its 4
//     slices, the k-bit words of the columns its mask selects --
//     y_u |= OR_{j in mask} X[8s + j] -- and marks the result in V_next[u] with
//     returnless 64-bit atomicOrs (the lazy marking of Algorithm 3, k bits at a time).
//   stage 2: a coalesced sweep over vertices: diff = V_next ^ V_curr becomes
//     the next frontier, newly set bits give levels, and the slice sets of
//     vertices with any new bit are enqueued with one atomicAdd per warp.
// Two layouts keep the levels during the traversal (LV):
//   LV 0, vertex-major: a vertex's k levels are contiguous; the sweep writes a
//     vertex's new levels with one warp store per 32 sources, and the output
//     kernel transposes them to the source-major output in original ids;
//   LV 1, bit planes: bit i of plane p's word w of vertex u is bit p of u's level
//     from source 64 w + i; a sweep ORs each vertex's new-bit word into the planes
//     of the bits set in the level number (a coalesced read-modify-write per vertex
//     and plane), and the output kernel rebuilds the levels 8 sources at a time
//     with 8 x 8 bit transposes.
// Planes cost popc(level) updates per distinct level at which a vertex gains bits:
// few on low-diameter graphs (most sources reach a vertex within a few levels),
// many on high-diameter ones, where the vertex-major layout is cheaper.
// Two back-ends compute the pull.  PULL 0 (default) ORs the selected frontier
// words on the CUDA cores.  PULL 1 runs the same product as b1 AND+POPC
// tensor-core MMAs (m16n8k128): VSS slots along M, sources along N, the slice
// set's 8 columns along K, so a VSS of k sources takes k MMAs (for k <= 64;
// 64 per word of 64 sources) and its counts are turned back into hit bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device_common.cuh"
#include "msbfs_launch.h"

namespace blest {

namespace {

constexpr int kMsBlock = 512;

struct MsArgs {
    int32_t n;
    int32_t k;
    unsigned int qcap;
    const int32_t* __restrict__ real_ptrs;
    const int4* __restrict__ row_ids4;
    const uint32_t* __restrict__ masks;
    const int32_t* __restrict__ new_id;
    unsigned long long* vcur;
    unsigned long long* vnext;
    unsigned long long* front;
    unsigned long long* Q[3];
    int32_t* lint;                // LV 0: n x kst, lint[u * kst + i] = level of BVSS vertex u from source i
    int32_t kst;                  // row stride of lint: k rounded up to a multiple of 8
    unsigned long long* planes;   // LV 1: nplanes x (n x W) words: plane p holds bit p of every level
    int32_t nplanes;              // msbfs_planes(n): enough bits for level n - 1
    int32_t vfilter;              // 1: test V_curr before each mark; 2: test V_next; 0: mark every hit word
    int32_t* out;        // k x n, source-major, original ids
    uint32_t* dirty;     // one bit per slice set touched by a mark in a sparse level (cleared by the sweep)
    const int32_t* roots;
    Ctrl* ctrl;
    int32_t* level_sizes;
    int32_t level_cap;
    uint64_t timeout_ns;
    unsigned int phantom;
};

// LV 0: levels of the new bits, vertex-major.  Lane j holds the new-bit word d
// (sources 64 w .. 64 w + 63) of vertex u0 + stride * j; for each such vertex with
// a new bit the warp writes that vertex's entries with two stores of 32
// consecutive sources, so a store touches one row instead of 32.
__device__ __forceinline__ void ms_write_levels(const MsArgs& a, unsigned long long d, int u0, int stride, int w,
                                                int lvl, int lane) {
    unsigned int todo = __ballot_sync(0xffffffffu, d != 0ull);
    while (todo) {
        const int j = __ffs(todo) - 1;
        todo &= todo - 1u;
        const unsigned long long dj = __shfl_sync(0xffffffffu, d, j);
        int32_t* row = a.lint + (size_t)(u0 + stride * j) * (size_t)a.kst + (size_t)(64 * w);
        if ((dj >> lane) & 1ull) row[lane] = lvl;
        if ((dj >> (32 + lane)) & 1ull) row[32 + lane] = lvl;
    }
}

// LV 1: level lvl for the new bits d of word w of vertex u: d is ORed into every
// plane p with bit p set in lvl.  Only the calling lane writes u's words in a
// sweep, so a plain read-modify-write suffices (measured faster than returnless
// atomic ORs); plane p was cleared during stage 1 of level 2^p, its first use.
template <int W>
__device__ __forceinline__ void ms_write_planes(const MsArgs& a, unsigned long long d, int u, int w, int lvl) {
    if (!d) return;
    const size_t stride = (size_t)a.n * W;
    unsigned long long* q = a.planes + (size_t)u * W + w;
    for (int p = 0; (lvl >> p) != 0; ++p)
        if ((lvl >> p) & 1) q[(size_t)p * stride] |= d;
}

template <int W, int LV>
__device__ __forceinline__ void ms_sweep(const MsArgs& a, int lvl, unsigned long long* Qout, unsigned long long* qcount) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int nchunks = (a.n + kWarp - 1) / kWarp;
    // one row per lane, 32 consecutive rows per warp step (they share bitmap
    // lines); consecutive chunks go to consecutive thread blocks so that the hub
    // rows at the lowest ids, whose slice sets carry most queue entries, are
    // spread over the SMs
    for (int c = (int)blockIdx.x + (int)(threadIdx.x >> 5) * (int)gridDim.x; c < nchunks; c += nwarps) {
        const int u = c * kWarp + lane;
        bool any = false;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            unsigned long long d = 0ull;
            if (u < a.n) {
                const size_t idx = (size_t)u * W + w;
                const unsigned long long nx = ld_cg(&a.vnext[idx]);
                const unsigned long long cu = ld_cg(&a.vcur[idx]);
                d = nx ^ cu;
                a.front[idx] = d;
                if (d) {
                    a.vcur[idx] = nx;
                    any = true;
                }
            }
            if (LV == 1) ms_write_planes<W>(a, d, u, w, lvl);
            else ms_write_levels(a, d, c * kWarp, 1, w, lvl, lane);
        }
        const unsigned int ball = __ballot_sync(0xffffffffu, any);
        int st = 0, ln = 0;
        uint32_t pay = 0;
        if ((lane & 7) == 0 && ((ball >> lane) & 0xFFu)) {
            const int s = u >> 3;
            st = __ldg(&a.real_ptrs[s]);
            ln = __ldg(&a.real_ptrs[s + 1]) - st;
            pay = (uint32_t)s;
        }
        warp_enqueue_coalesced(a.qcap, a.ctrl, Qout, qcount, st, ln, pay, lane);
    }
}

// Sparse finalisation: only the slice sets marked dirty in stage 1 are swept.
// Warp w takes dirty words t = w, w + nwarps, ...; lane b handles slice set
// 32 t + b when its bit is set: the 8 vertices' words get diff = V_next ^ V_curr
// (written to the frontier, zero included, so every vertex of a queued slice set
// has a current frontier word), levels, and the enqueue.  Slice sets outside
// the dirty set keep stale frontier words, but they are not queued, so stage 1
// never reads them.
template <int W, int LV>
__device__ __forceinline__ void ms_sweep_sparse(const MsArgs& a, int lvl, unsigned long long* Qout,
                                                unsigned long long* qcount) {
    const int lane = threadIdx.x & 31;
    const int wpb = (int)(blockDim.x >> 5);
    const int nss = (a.n + 7) >> 3;
    const int dwords = (nss + 31) >> 5;
    // block-strided over dirty words so that every warp of a block runs the same iterations
    for (int t0 = (int)blockIdx.x * wpb; t0 < dwords; t0 += (int)gridDim.x * wpb) {
        const int t = t0 + (int)(threadIdx.x >> 5);
        const uint32_t dw = t < dwords ? ld_cg(&a.dirty[t]) : 0u;
        if (lane == 0 && dw) a.dirty[t] = 0u;
        const int s = 32 * t + lane;
        const bool mine = (dw >> lane) & 1u;
        bool any = false;
        if (dw) {   // warp-uniform; every lane runs the loop for the level writes
            for (int j = 0; j < 8; ++j) {
                const int u = 8 * s + j;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    unsigned long long d = 0ull;
                    if (mine && u < a.n) {
                        const size_t idx = (size_t)u * W + w;
                        const unsigned long long nx = ld_cg(&a.vnext[idx]);
                        const unsigned long long cu = ld_cg(&a.vcur[idx]);
                        d = nx ^ cu;
                        a.front[idx] = d;
                        if (d) {
                            a.vcur[idx] = nx;
                            any = true;
                        }
                    }
                    if (LV == 1) ms_write_planes<W>(a, d, u, w, lvl);
                    else ms_write_levels(a, d, 8 * 32 * t + j, 8, w, lvl, lane);
                }
            }
        }
        int st = 0, ln = 0;
        uint32_t pay = 0;
        if (any) {
            st = __ldg(&a.real_ptrs[s]);
            ln = __ldg(&a.real_ptrs[s + 1]) - st;
            pay = (uint32_t)s;
        }
        warp_enqueue_coalesced(a.qcap, a.ctrl, Qout, qcount, st, ln, pay, lane);
    }
}

// One queued VSS as stage 1 needs it: its tile (four row ids and the mask word
// of this lane) and the 8 x k frontier tile of its slice set (lane j*W + w holds
// word w of column 8s + j).
template <int W>
struct MsTile {
    int4 r;
    uint32_t m;
    unsigned long long fw;
};

constexpr unsigned long long kNoEntry = ~0ull;

template <int W>
__device__ __forceinline__ MsTile<W> ms_load_tile(const MsArgs& a, unsigned long long ent, int lane, uint64_t pol) {
    MsTile<W> t;
    t.r = make_int4(0, 0, 0, 0);
    t.m = 0u;
    t.fw = 0ull;
    if (ent == kNoEntry) return t;   // warp-uniform
    const uint32_t nu = (uint32_t)ent;
    const int s = (int)(ent >> 32);
    if (lane < 8 * W) {
        const int col = 8 * s + lane / W;
        if (col < a.n) t.fw = ld_cg(&a.front[(size_t)col * W + (lane % W)]);
    }
    // read once per level: streamed past L1 with an evict-first L2 policy so that
    // the bitmaps and the frontier stay resident in L2
    const size_t tile = (size_t)nu * kWarp + lane;
    t.r = ld_stream_v4(&a.row_ids4[tile], pol);
    t.m = ld_stream_u32(&a.masks[tile], pol);
    return t;
}

// The tensor-core product of one VSS and one 64-source word w of its slice set's
// frontier tile: y[q] = the sources (bits) reaching this lane's sub-slot q.
//   M (16 rows per MMA, 8 MMA row tiles): slot (tile m, row r) is sub-slot
//     2 (m / 4) + r / 8 of lane 4 (r % 8) + m % 4, so an MMA group's rows are the
//     sub-slots of its own 4 lanes and the results come back to their owners;
//   N (8 per MMA, 8 column tiles): source 64 w + 8 n + c;
//   K (bits 0..7 of the 128; the rest zero): the slice set's 8 columns.
// D[r][c] = popc(mask byte of slot r & column bits of source c) > 0 is the hit.
// Fragments (m16n8k128, b1): lane 4 g + t holds A rows g and g + 8 and B column
// g, each over K bits 32 t .. 32 t + 31 (so only t = 0 carries data), and D
// rows g and g + 8 at columns 2 t, 2 t + 1.
template <int W>
__device__ __forceinline__ void ms_mma_word(const MsTile<W>& t, int lane, int w, unsigned long long (&y)[4][W]) {
    const int g = lane >> 2, tq = lane & 3;
    // column bits of sources 64 w + 8 n + g, byte n: a transpose of the 8 x 64 tile
    unsigned long long bt = 0ull;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const unsigned long long x = __shfl_sync(0xffffffffu, t.fw, j * W + w);
        bt |= ((x >> g) & 0x0101010101010101ull) << j;
    }
    uint32_t mw[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) mw[i] = __shfl_sync(0xffffffffu, t.m, 4 * g + i);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const uint32_t a0 = tq == 0 ? (mw[m & 3] >> (8 * (2 * (m >> 2)))) & 0xFFu : 0u;
        const uint32_t a1 = tq == 0 ? (mw[m & 3] >> (8 * (2 * (m >> 2) + 1))) & 0xFFu : 0u;
        unsigned long long pg = 0ull, pg8 = 0ull;   // this lane's columns of rows g and g + 8
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const uint32_t b0 = tq == 0 ? (uint32_t)(bt >> (8 * n)) & 0xFFu : 0u;
            int d0, d1, d2, d3;
            asm volatile(
                "mma.sync.aligned.m16n8k128.row.col.s32.b1.b1.s32.and.popc {%0,%1,%2,%3}, {%4,%5}, {%6}, "
                "{%7,%7,%7,%7};\n"
                : "=r"(d0), "=r"(d1), "=r"(d2), "=r"(d3)
                : "r"(a0), "r"(a1), "r"(b0), "r"(0));
            const int sh = 8 * n + 2 * tq;
            pg |= (unsigned long long)((d0 > 0 ? 1u : 0u) | (d1 > 0 ? 2u : 0u)) << sh;
            pg8 |= (unsigned long long)((d2 > 0 ? 1u : 0u) | (d3 > 0 ? 2u : 0u)) << sh;
        }
        // the 4 lanes of the group hold 16 of the 64 columns each
        pg |= __shfl_xor_sync(0xffffffffu, pg, 1);
        pg |= __shfl_xor_sync(0xffffffffu, pg, 2);
        pg8 |= __shfl_xor_sync(0xffffffffu, pg8, 1);
        pg8 |= __shfl_xor_sync(0xffffffffu, pg8, 2);
        if (tq == (m & 3)) {   // the owner of slots (m, g) and (m, g + 8)
            y[2 * (m >> 2)][w] = pg;
            y[2 * (m >> 2) + 1][w] = pg8;
        }
    }
}

// y_u |= OR over the columns j of u's mask of the frontier word X[8s + j], then
// the returnless marks of the fresh bits in V_next (Algorithm 3, k bits at a time).
template <int W, int PULL>
__device__ __forceinline__ void ms_pull_tile(const MsArgs& a, const MsTile<W>& t, int lane, bool sparse) {
    const unsigned int nzb = __ballot_sync(0xffffffffu, t.fw != 0ull);
    uint32_t alpha = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if ((nzb >> (j * W)) & ((1u << W) - 1u)) alpha |= 1u << j;
    if (!alpha) return;   // warp-uniform: no column of this slice set is in the frontier
    unsigned long long y[4][W];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < W; ++w) y[q][w] = 0ull;
    if (PULL == 1) {
#pragma unroll
        for (int w = 0; w < W; ++w) ms_mma_word<W>(t, lane, w, y);
    } else {
        const uint32_t m = t.m & (alpha * 0x01010101u);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (!((alpha >> j) & 1u)) continue;   // warp-uniform
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const unsigned long long v = __shfl_sync(0xffffffffu, t.fw, j * W + w);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if ((m >> (8 * q + j)) & 1u) y[q][w] |= v;
            }
        }
    }
    const int r4[4] = {t.r.x, t.r.y, t.r.z, t.r.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < W; ++w) {
            if (!y[q][w]) continue;
            // sources that already reached the row need no mark; V_curr only gains
            // bits during a traversal, so a stale word can only let a mark through.
            // Without the test every hit word is marked: V_next keeps containing V_curr,
            // so the sweep's diff is the same, and the gather (a dependent load) is gone.
            // V_next contains V_curr, so testing it also skips sources already marked at
            // this level (a stale word again only lets a mark through).
            const size_t vi = (size_t)r4[q] * W + w;
            const unsigned long long fresh =
                a.vfilter == 0 ? y[q][w] : y[q][w] & ~(a.vfilter == 2 ? a.vnext[vi] : a.vcur[vi]);
            if (fresh) {
                atomicOr(&a.vnext[(size_t)r4[q] * W + w], fresh);
                if (sparse) atomicOr(&a.dirty[r4[q] >> 8], 1u << ((r4[q] >> 3) & 31));
            }
        }
}

template <int W, int PULL, int LV>
__device__ __forceinline__ void ms_body(const MsArgs& a) {
    const int lane = threadIdx.x & 31;
    const int gtid = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int nthreads = (int)(gridDim.x * blockDim.x);
    const int gwarp = gtid >> 5;
    const int nwarps = nthreads >> 5;
    unsigned int bar = 0;   // barriers passed; the next one is number bar
    Ctrl* ctrl = a.ctrl;
    const uint64_t pol = l2_evict_first_policy();

    for (int i = gtid; i < a.k; i += nthreads) {
        const int r = a.roots[i];
        atomicOr(&a.vnext[(size_t)r * W + (i >> 6)], 1ull << (i & 63));
    }
    if (!grid_barrier(ctrl, gridDim.x, a.phantom, bar, a.timeout_ns)) return;
    ms_sweep<W, LV>(a, 0, a.Q[1], ring_word(ctrl, bar));
    unsigned int qn = 0;
    if (!grid_barrier(ctrl, gridDim.x, a.phantom, bar, a.timeout_ns, &qn)) return;

    int lvl = 1;
    for (;; ++lvl) {
        if (qn > a.qcap) qn = a.qcap;   // only after an overflow, which already raised an error
        // few queued VSSs: track the touched slice sets and sweep only those
        const bool sparse = (unsigned long long)qn * 128ull <= (unsigned long long)a.n;
        if (gtid == 0 && a.level_sizes && lvl - 1 < a.level_cap) a.level_sizes[lvl - 1] = (int32_t)qn;
        const unsigned long long* Qin = a.Q[lvl % 3];
        unsigned long long* Qout = a.Q[(lvl + 1) % 3];
        unsigned long long* qcount_next = ring_word(ctrl, bar + 1u);   // the barrier after the sweep
        if (LV == 1 && (lvl & (lvl - 1)) == 0) {
            // lvl = 2^p: this level's sweep is the first to write plane p, so it is
            // cleared now (stage 1 does not touch the planes; the barrier orders it)
            const int p = __ffs(lvl) - 1;
            if (p < a.nplanes) {
                unsigned long long* pl = a.planes + (size_t)p * (size_t)a.n * W;
                for (size_t i = (size_t)gtid; i < (size_t)a.n * W; i += (size_t)nthreads) pl[i] = 0ull;
            }
        }
        // software pipeline over this warp's items p, p + nwarps, ...: the entry two
        // items ahead and the tile and frontier words one item ahead are in flight
        // while the current item is pulled
        const unsigned int nw = (unsigned int)nwarps;
        unsigned int p = (unsigned int)gwarp;
        unsigned long long e_next = p + nw < qn ? ld_cg(&Qin[p + nw]) : kNoEntry;
        MsTile<W> t = ms_load_tile<W>(a, p < qn ? ld_cg(&Qin[p]) : kNoEntry, lane, pol);
        for (; p < qn; p += nw) {
            const unsigned long long e_after = p + 2u * nw < qn ? ld_cg(&Qin[p + 2u * nw]) : kNoEntry;
            const MsTile<W> t_next = ms_load_tile<W>(a, e_next, lane, pol);
            ms_pull_tile<W, PULL>(a, t, lane, sparse);
            t = t_next;
            e_next = e_after;
        }
        if (!grid_barrier(ctrl, gridDim.x, a.phantom, bar, a.timeout_ns)) return;
        if (sparse) ms_sweep_sparse<W, LV>(a, lvl, Qout, qcount_next);
        else ms_sweep<W, LV>(a, lvl, Qout, qcount_next);
        unsigned int qnext = 0;
        if (!grid_barrier(ctrl, gridDim.x, a.phantom, bar, a.timeout_ns, &qnext)) return;
        if (qnext == 0) break;
        qn = qnext;
    }
    if (gtid == 0) ctrl->levels = (unsigned int)lvl;
}

// Output kernels: out[i*n + v] = level of v from source i (original ids), -1 if
// unreached, as a separate launch after the traversal (ctrl->levels holds its
// level count) so that the traversal kernel keeps its register budget.  Lane j
// takes vertex v = 32 b + j and stores the levels source by source, 32
// consecutive vertices per store.

// LV 0: the vertex's levels are read 4 sources (16 bytes) at a time.
template <int W>
__global__ void __launch_bounds__(kMsBlock) msbfs_output_rows_kernel(MsArgs a) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int nvb = (a.n + kWarp - 1) / kWarp;
    for (int b = gwarp; b < nvb; b += nwarps) {
        const int v = b * kWarp + lane;
        if (v >= a.n) continue;
        const int u = a.new_id ? __ldg(&a.new_id[v]) : v;
        const int4* row = reinterpret_cast<const int4*>(a.lint + (size_t)u * (size_t)a.kst);
        int32_t* o = a.out + v;
#pragma unroll 1
        for (int w = 0; w < W; ++w) {
            const unsigned long long vis = ld_cg(&a.vcur[(size_t)u * W + w]);
            const int i_end = min(64 * w + 64, a.k);
#pragma unroll 1
            for (int i0 = 64 * w; i0 < i_end; i0 += 4) {
                const uint32_t bits = (uint32_t)(vis >> (i0 - 64 * w)) & 0xFu;
                // positions of sources that never reached u are never written, so never used
                const int4 lv = bits ? ld_cg(&row[i0 >> 2]) : make_int4(-1, -1, -1, -1);
                o[(size_t)i0 * (size_t)a.n] = bits & 1u ? lv.x : -1;
                if (i0 + 1 < i_end) o[(size_t)(i0 + 1) * (size_t)a.n] = bits & 2u ? lv.y : -1;
                if (i0 + 2 < i_end) o[(size_t)(i0 + 2) * (size_t)a.n] = bits & 4u ? lv.z : -1;
                if (i0 + 3 < i_end) o[(size_t)(i0 + 3) * (size_t)a.n] = bits & 8u ? lv.w : -1;
            }
        }
    }
}

// LV 1: the vertex's plane words (the planes that can hold a bit of a level <= the
// level count: the ones the traversal cleared) are read once, and the levels are
// rebuilt 8 sources at a time.
template <int W>
__global__ void __launch_bounds__(kMsBlock) msbfs_output_kernel(MsArgs a) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int lvl = (int)ld_cg(&a.ctrl->levels);
    const int np = min(32 - __clz(lvl), a.nplanes);
    const size_t pstride = (size_t)a.n * W;
    const int nvb = (a.n + kWarp - 1) / kWarp;
    for (int b = gwarp; b < nvb; b += nwarps) {
        const int v = b * kWarp + lane;
        if (v >= a.n) continue;
        const int u = a.new_id ? __ldg(&a.new_id[v]) : v;
        int32_t* o = a.out + v;
#pragma unroll 1
        for (int w = 0; w < W; ++w) {
            const size_t idx = (size_t)u * W + w;
            const unsigned long long vis = ld_cg(&a.vcur[idx]);
            const int i_end = min(64 * w + 64, a.k);
            if (np <= 8) {
                uint64_t pw[8];
#pragma unroll
                for (int p = 0; p < 8; ++p) pw[p] = p < np ? ld_cg(&a.planes[(size_t)p * pstride + idx]) : 0ull;
#pragma unroll 1
                for (int i0 = 64 * w; i0 < i_end; i0 += 8) {
                    const int c = (i0 - 64 * w) >> 3;
                    const unsigned long long lv8 = levels_of_8(pw, c);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int i = i0 + j;
                        if (i < i_end)
                            o[(size_t)i * (size_t)a.n] =
                                (vis >> (8 * c + j)) & 1ull ? (int32_t)((lv8 >> (8 * j)) & 0xFFull) : -1;
                    }
                }
            } else {
                // levels of 256 and more (high-diameter graphs): planes 0..15 in registers, two
                // transposes per 8 sources; planes 16.. (levels of 65536 and more) read per source
                uint64_t pw[16];
#pragma unroll
                for (int p = 0; p < 16; ++p) pw[p] = p < np ? ld_cg(&a.planes[(size_t)p * pstride + idx]) : 0ull;
#pragma unroll 1
                for (int i0 = 64 * w; i0 < i_end; i0 += 8) {
                    const int c = (i0 - 64 * w) >> 3;
                    uint64_t lo, hi;
                    levels_of_8x16(pw, c, lo, hi);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int i = i0 + j;
                        if (i >= i_end) continue;
                        const int bit = 8 * c + j;
                        int32_t lv = -1;
                        if ((vis >> bit) & 1ull) {
                            lv = (int32_t)((lo >> (8 * j)) & 0xFFull) | ((int32_t)((hi >> (8 * j)) & 0xFFull) << 8);
                            for (int p = 16; p < np; ++p)
                                lv |= (int32_t)((ld_cg(&a.planes[(size_t)p * pstride + idx]) >> bit) & 1ull) << p;
                        }
                        o[(size_t)i * (size_t)a.n] = lv;
                    }
                }
            }
        }
    }
}

template <int W, int PULL, int LV>
__global__ void __launch_bounds__(kMsBlock) msbfs_kernel(MsArgs a) {
    ms_body<W, PULL, LV>(a);
    fold_status(a.ctrl);
}

// One word of sources (W = 1) on the CUDA cores, held to 3 resident blocks per SM:
// as many warps in flight as the register file allows at that width.
template <int LV>
__global__ void __launch_bounds__(kMsBlock, 3) msbfs_kernel_w1(MsArgs a) {
    ms_body<1, 0, LV>(a);
    fold_status(a.ctrl);
}

template <int LV>
void* ms_kernel_ptr(int W, int pull) {
    if (pull == 1)
        return W == 1 ? (void*)&msbfs_kernel<1, 1, LV> : (W == 2 ? (void*)&msbfs_kernel<2, 1, LV>
                                                                  : (void*)&msbfs_kernel<4, 1, LV>);
    return W == 1 ? (void*)&msbfs_kernel_w1<LV> : (W == 2 ? (void*)&msbfs_kernel<2, 0, LV>
                                                           : (void*)&msbfs_kernel<4, 0, LV>);
}

void* ms_output_ptr(int W, int lv) {
    if (lv == 1)
        return W == 1 ? (void*)&msbfs_output_kernel<1> : (W == 2 ? (void*)&msbfs_output_kernel<2>
                                                                 : (void*)&msbfs_output_kernel<4>);
    return W == 1 ? (void*)&msbfs_output_rows_kernel<1> : (W == 2 ? (void*)&msbfs_output_rows_kernel<2>
                                                                   : (void*)&msbfs_output_rows_kernel<4>);
}

template <class T>
cudaError_t grow(T*& p, int64_t& cap, int64_t need, bool caller_owned, int copies = 1) {
    if (need <= cap) return cudaSuccess;
    if (caller_owned) return cudaErrorInvalidValue;   // never free or replace the caller's memory
    cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, sizeof(T) * (size_t)need * copies);
    if (e == cudaSuccess) cap = need;
    return e;
}

}  // namespace

void free_msbfs_state(MsbfsState& s) {
    cudaFree(s.vcur);
    cudaFree(s.vnext);
    cudaFree(s.front);
    cudaFree(s.Q);
    cudaFree(s.lint);
    cudaFree(s.planes);
    cudaFree(s.roots);
    cudaFree(s.dirty);
    s = MsbfsState();
}

int run_msbfs(MsbfsState& s, const MsbfsLaunchCommon& c, const std::vector<int32_t>& roots, int32_t* d_out,
              cudaStream_t st, const char** err) {
    const int64_t k_all = (int64_t)roots.size();
    if (k_all == 0 || c.n == 0) return 0;
    cudaError_t e = cudaSuccess;
    const bool own = s.caller_owned;
    const int chunk = c.chunk == 64 || c.chunk == 128 ? c.chunk : kMsbfsChunk;
    for (int64_t i0 = 0; i0 < k_all; i0 += chunk) {
        const int k = (int)std::min<int64_t>(chunk, k_all - i0);
        const int W = msbfs_words(k, chunk);
        const int64_t words = (int64_t)c.n * W;
        int64_t cap_v = s.words_cap, cap_n = s.words_cap, cap_f = s.words_cap;
        if ((e = grow(s.vcur, cap_v, words, own)) != cudaSuccess) break;
        if ((e = grow(s.vnext, cap_n, words, own)) != cudaSuccess) break;
        if ((e = grow(s.front, cap_f, words, own)) != cudaSuccess) break;
        s.words_cap = std::min(cap_v, std::min(cap_n, cap_f));
        if ((e = grow(s.Q, s.qcap, std::max<int64_t>(c.nvss, 1), own, 3)) != cudaSuccess) break;
        const int lv = c.levels_layout == 1 ? 1 : 0;
        const int32_t kst = (k + 7) & ~7;
        if (lv == 1) {
            if ((e = grow(s.planes, s.planes_cap, msbfs_plane_words(c.n, k, chunk), own)) != cudaSuccess) break;
        } else {
            if ((e = grow(s.lint, s.lint_cap, msbfs_level_entries(c.n, k, chunk), own)) != cudaSuccess) break;
        }
        if ((e = grow(s.roots, s.roots_cap, k, own)) != cudaSuccess) break;
        const int64_t dwords = ((int64_t)c.nss + 31) / 32;
        if ((e = grow(s.dirty, s.dirty_cap, dwords, own)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(s.roots, roots.data() + i0, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        cudaMemsetAsync(c.ctrl, 0, kCtrlClearBytes, st);
        cudaMemsetAsync(s.vcur, 0, sizeof(unsigned long long) * (size_t)words, st);
        cudaMemsetAsync(s.vnext, 0, sizeof(unsigned long long) * (size_t)words, st);
        cudaMemsetAsync(s.dirty, 0, sizeof(uint32_t) * (size_t)dwords, st);
        MsArgs a;
        a.n = c.n;
        a.k = k;
        a.qcap = (unsigned int)std::max<int64_t>(c.nvss, 1);
        a.real_ptrs = c.real_ptrs;
        a.row_ids4 = reinterpret_cast<const int4*>(c.row_ids);
        a.masks = c.masks;
        a.new_id = c.new_id;
        a.vcur = s.vcur;
        a.vnext = s.vnext;
        a.front = s.front;
        for (int i = 0; i < 3; ++i) a.Q[i] = s.Q + (size_t)i * (size_t)s.qcap;
        int32_t* out = d_out + (size_t)i0 * (size_t)c.n;
        a.lint = s.lint;
        a.kst = kst;
        a.planes = s.planes;
        a.nplanes = msbfs_planes(c.n);
        a.vfilter = c.visited_filter;
        a.out = out;
        a.roots = s.roots;
        a.dirty = s.dirty;
        a.ctrl = reinterpret_cast<Ctrl*>(c.ctrl);
        a.level_sizes = c.level_sizes;
        a.level_cap = c.level_cap;
        a.timeout_ns = c.timeout_ns;
        a.phantom = c.phantom;
        void* kfn = lv == 1 ? ms_kernel_ptr<1>(W, c.pull) : ms_kernel_ptr<0>(W, c.pull);
        int nb = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, kMsBlock, 0)) != cudaSuccess) break;
        if (nb <= 0) { *err = "msbfs kernel cannot be resident"; return 5; }
        if (c.blocks_per_sm > 0) nb = std::min(nb, c.blocks_per_sm);
        void* args[] = {&a};
        if ((e = cudaLaunchCooperativeKernel(kfn, dim3((unsigned)(nb * c.sms)), dim3(kMsBlock), args, 0, st)) != cudaSuccess) break;
        // the source-major output in original ids, from the level planes
        const int64_t warps_needed = ((int64_t)c.n + kWarp - 1) / kWarp;
        const int64_t blocks = std::min<int64_t>((warps_needed + kMsBlock / kWarp - 1) / (kMsBlock / kWarp),
                                                 (int64_t)c.sms * 8);
        void* ofn = ms_output_ptr(W, lv);
        if ((e = cudaLaunchKernel(ofn, dim3((unsigned)std::max<int64_t>(blocks, 1)), dim3(kMsBlock), args, 0, st)) != cudaSuccess)
            break;
    }
    if (e != cudaSuccess) {
        *err = own && e == cudaErrorInvalidValue ? "caller-owned multi-source state is smaller than the launch"
                                                 : cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? 4 : 5;
    }
    return 0;
}

}  // namespace blest
