// Fused persistent BFS over BVSS (Sections 4.1-4.3): one cooperative launch runs
// every level of a traversal.  Per level:
//   stage 1 (pull): warps take queued virtual slice sets round-robin (Section
//     3.1.1); each lane loads its 4 row ids (one 128-bit load) and its 4 packed
//     8-bit masks (one 32-bit load) and tests mask & alpha != 0 per sub-slot --
//     Eq. 1's threshold of the AND/POPC product -- on the CUDA cores or with the
//     two m8n8k128 b1 MMAs of Figure 2c.
//   update, eager (Algorithm 2): at each hit on an unvisited row, write its level
//     and set its frontier bit with a returning atomicOr; the first bit set in a
//     slice set's byte enqueues that slice set's VSS range.
//   update, lazy (Algorithm 3): at each hit, a returnless atomicOr marks the row
//     in V_next; after a grid barrier a coalesced sweep over the n/32 words sets
//     levels of the newly marked rows and enqueues their slice sets with one
//     warp-aggregated atomicAdd per warp.
//   termination (Section 4.3): after a grid barrier every block reads the size
//     of the next queue; zero ends the traversal.
// Differences from the printed algorithms (kept equivalent in result):
//   * lazy queue entries carry the slice set's new frontier byte alpha next to
//     the VSS id, so stage 1 needs neither virtualToReal nor a frontier-bitmap
//     load; eager entries carry the slice set id;
//   * an eager slice set is enqueued once per level (first bit of its byte),
//     not once per newly reached row;
//   * queue counters rotate over four slots and eager frontier bitmaps over
//     three, so a level needs one barrier (eager) or two (lazy), not three;
//   * level 0 (the sources) goes through the same sweep as a lazy level, which
//     handles any number of sources (multi-root and batched-graph traversal).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "bfs_launch.h"
#include "device_common.cuh"

namespace blest {

constexpr int kBfsBlock = 512;

struct BfsArgs {
    int32_t n, nwords;
    unsigned int qcap;
    const int32_t* __restrict__ real_ptrs;
    const int4* __restrict__ row_ids4;
    const uint32_t* __restrict__ masks;
    const int32_t* __restrict__ new_id;  // NULL: identity, L is the output
    int32_t* L;
    uint32_t* vcur;
    uint32_t* vnext;
    uint32_t* F[3];
    unsigned long long* Q[3];
    Ctrl* ctrl;
    int32_t* level_sizes;
    int32_t level_cap;
    const int32_t* roots;                 // device list (used when nroots > kInlineRoots)
    int32_t nroots;
    int32_t inline_roots[kInlineRoots];
    int32_t* out;                         // output in original ids (unused when new_id is NULL)
    uint64_t timeout_ns;
    unsigned int phantom;
    int filter;                           // 1 = skip rows already set in the V bitmap
};

// ------------------------------------------------------------------- pull

template <int PULL>
__device__ __forceinline__ unsigned int pull_hits(uint32_t mask, uint32_t alpha, int lane) {
    if (PULL == 0) {
        const uint32_t hit = mask & (alpha * 0x01010101u);
        return (unsigned int)((hit & 0xFFu) != 0) | ((unsigned int)((hit & 0xFF00u) != 0) << 1) |
               ((unsigned int)((hit & 0xFF0000u) != 0) << 2) | ((unsigned int)((hit & 0xFF000000u) != 0) << 3);
    } else {
        // Figure 2c: fragA = two packed masks in the low 16 bits; fragB = alpha
        // in lanes t mod 9 == 0 (selects the first mask of lane t's row/column
        // pair) and alpha << 8 in lanes t mod 9 == 4 (the second); each lane's
        // two accumulators are the popcounts of its own two slices.
        const int sel = lane % 9;
        const uint32_t fragB = sel == 0 ? alpha : (sel == 4 ? (alpha << 8) : 0u);
        const uint32_t a_lo = mask & 0xFFFFu, a_hi = mask >> 16;
        int c0, c1, c2, c3;
        asm volatile(
            "mma.sync.aligned.m8n8k128.row.col.s32.b1.b1.s32.and.popc {%0,%1}, {%2}, {%3}, {%4,%5};\n"
            : "=r"(c0), "=r"(c1)
            : "r"(a_lo), "r"(fragB), "r"(0), "r"(0));
        asm volatile(
            "mma.sync.aligned.m8n8k128.row.col.s32.b1.b1.s32.and.popc {%0,%1}, {%2}, {%3}, {%4,%5};\n"
            : "=r"(c2), "=r"(c3)
            : "r"(a_hi), "r"(fragB), "r"(0), "r"(0));
        return (unsigned int)(c0 > 0) | ((unsigned int)(c1 > 0) << 1) | ((unsigned int)(c2 > 0) << 2) |
               ((unsigned int)(c3 > 0) << 3);
    }
}

// Finalisation sweep (Algorithm 3, stage 2), also used for level 0: every word
// t with diff = V_next ^ V_curr != 0 gets V_curr = V_next, its new rows get
// level lvl, and each slice set (byte) of diff is enqueued with payload alpha
// (lazy) or its id (eager, which also stores diff into the frontier bitmap).
template <int UPDATE>
__device__ __forceinline__ void sweep(const BfsArgs& a, int lvl, unsigned long long* Qout, unsigned int* qcount,
                                      uint32_t* Fout) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int t0 = gwarp * kWarp; t0 < a.nwords; t0 += nwarps * kWarp) {
        const int t = t0 + lane;
        uint32_t diff = 0;
        if (t < a.nwords) {
            const uint32_t nx = ld_cg(&a.vnext[t]);
            const uint32_t cu = ld_cg(&a.vcur[t]);
            diff = nx ^ cu;
            if (diff) {
                a.vcur[t] = nx;
                if (UPDATE == 1) Fout[t] = diff;
            }
        }
        uint32_t d = diff;
        while (d) {
            const int b = __ffs(d) - 1;
            a.L[t * kWarp + b] = lvl;
            d &= d - 1;
        }
        int st[4], ln[4];
        uint32_t pay[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t byte = (diff >> (8 * q)) & 0xFFu;
            st[q] = 0; ln[q] = 0; pay[q] = 0;
            if (byte) {
                const int s = 4 * t + q;
                st[q] = __ldg(&a.real_ptrs[s]);
                ln[q] = __ldg(&a.real_ptrs[s + 1]) - st[q];
                pay[q] = UPDATE == 2 ? byte : (uint32_t)s;
            }
        }
        warp_enqueue<4>(a.qcap, a.ctrl, Qout, qcount, st, ln, pay, lane);
    }
}

// -------------------------------------------------------------------- kernel

template <int UPDATE, int PULL, int UNROLL>
__device__ __forceinline__ void bfs_body(const BfsArgs& a) {
    const int lane = threadIdx.x & 31;
    const int gtid = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int nthreads = (int)(gridDim.x * blockDim.x);
    const int gwarp = gtid >> 5;
    const int nwarps = nthreads >> 5;
    const unsigned int nblocks = gridDim.x;
    unsigned int gen = 0;
    Ctrl* ctrl = a.ctrl;

    // level 0: mark the sources (V_curr, V_next, L were cleared before launch)
    for (int i = gtid; i < a.nroots; i += nthreads) {
        const int r = a.nroots <= kInlineRoots ? a.inline_roots[i] : a.roots[i];
        atomicOr(&a.vnext[r >> 5], 1u << (r & 31));
    }
    if (!grid_barrier(ctrl, nblocks, a.phantom, gen, a.timeout_ns)) return;
    sweep<UPDATE>(a, 0, a.Q[1], &ctrl->qcount[1], a.F[1]);
    unsigned int qn = 0, qprev = 0;
    if (!grid_barrier(ctrl, nblocks, a.phantom, gen, a.timeout_ns, &ctrl->qcount[1], &qn)) return;

    int lvl = 1;
    for (;; ++lvl) {
        if (qn > a.qcap) qn = a.qcap;   // only after an overflow, which already raised an error
        if (gtid == 0) {
            ctrl->qcount[(lvl + 2) & 3] = 0;
            if (a.level_sizes && lvl - 1 < a.level_cap) a.level_sizes[lvl - 1] = (int32_t)qn;
        }
        const unsigned long long* Qin = a.Q[lvl % 3];
        if (UPDATE == 1) {
            // clear the frontier bytes of level lvl-1 (read last level, rewritten at lvl+1)
            const unsigned long long* Qp = a.Q[(lvl + 2) % 3];
            unsigned char* Fold = reinterpret_cast<unsigned char*>(a.F[(lvl + 2) % 3]);
            for (unsigned int i = (unsigned int)gtid; i < qprev; i += (unsigned int)nthreads)
                Fold[(uint32_t)(ld_cg(&Qp[i]) >> 32)] = 0;
        }
        const uint32_t* Fcur = a.F[lvl % 3];
        uint32_t* Fnext = a.F[(lvl + 1) % 3];
        unsigned long long* Qout = a.Q[(lvl + 1) % 3];
        unsigned int* qcount_next = &ctrl->qcount[(lvl + 1) & 3];

        // stage 1: pull the queued virtual slice sets, round-robin over warps
        for (unsigned int base = (unsigned int)gwarp; base < qn; base += (unsigned int)nwarps * UNROLL) {
            unsigned long long ent[UNROLL];
            int4 rows[UNROLL];
            uint32_t msk[UNROLL];
#pragma unroll
            for (int i = 0; i < UNROLL; ++i) {
                const unsigned int p = base + (unsigned int)i * (unsigned int)nwarps;
                ent[i] = p < qn ? ld_cg(&Qin[p]) : ~0ull;
            }
#pragma unroll
            for (int i = 0; i < UNROLL; ++i) {
                if (ent[i] != ~0ull) {
                    const size_t tile = (size_t)(uint32_t)ent[i] * kWarp + lane;
                    rows[i] = __ldg(&a.row_ids4[tile]);
                    msk[i] = __ldg(&a.masks[tile]);
                }
            }
            if (UPDATE == 2) {
#pragma unroll
                for (int i = 0; i < UNROLL; ++i) {
                    if (ent[i] == ~0ull) continue;
                    const uint32_t alpha = (uint32_t)(ent[i] >> 32);
                    const unsigned int h = pull_hits<PULL>(msk[i], alpha, lane);
                    const int r4[4] = {rows[i].x, rows[i].y, rows[i].z, rows[i].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (!(h & (1u << q))) continue;
                        const int u = r4[q];
                        const uint32_t bit = 1u << (u & 31);
                        // visited filter: V_curr only gains bits during a traversal, so a
                        // stale (older) word can only let through a redundant mark
                        if (a.filter && (a.vcur[u >> 5] & bit)) continue;
                        atomicOr(&a.vnext[u >> 5], bit);
                    }
                }
            } else {
                int st[4 * UNROLL], ln[4 * UNROLL];
                uint32_t pay[4 * UNROLL];
#pragma unroll
                for (int i = 0; i < UNROLL; ++i) {
                    uint32_t alpha = 0;
                    if (ent[i] != ~0ull) {
                        const uint32_t s = (uint32_t)(ent[i] >> 32);
                        alpha = (ld_cg(&Fcur[s >> 2]) >> (8 * (s & 3))) & 0xFFu;
                    }
                    // every lane of the warp runs the pull (the MMA needs the full warp)
                    const unsigned int h = ent[i] != ~0ull ? pull_hits<PULL>(msk[i], alpha, lane) : 0u;
                    const int r4[4] = {rows[i].x, rows[i].y, rows[i].z, rows[i].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = 4 * i + q;
                        st[k] = 0; ln[k] = 0; pay[k] = 0;
                        if (!(h & (1u << q))) continue;
                        const int u = r4[q];
                        const uint32_t bit = 1u << (u & 31);
                        // visited filter on the V bitmap (a subset of the visited set, see lazy)
                        if (a.filter && (a.vcur[u >> 5] & bit)) continue;
                        if (ld_cg(&a.L[u]) < 0) {
                            a.L[u] = lvl;
                            if (a.filter) atomicOr(&a.vcur[u >> 5], bit);
                            const uint32_t old = atomicOr(&Fnext[u >> 5], bit);
                            if (((old >> (u & 24)) & 0xFFu) == 0) {
                                const int s2 = u >> 3;
                                st[k] = __ldg(&a.real_ptrs[s2]);
                                ln[k] = __ldg(&a.real_ptrs[s2 + 1]) - st[k];
                                pay[k] = (uint32_t)s2;
                            }
                        }
                    }
                }
                warp_enqueue<4 * UNROLL>(a.qcap, ctrl, Qout, qcount_next, st, ln, pay, lane);
            }
        }
        if (UPDATE == 2) {
            if (!grid_barrier(ctrl, nblocks, a.phantom, gen, a.timeout_ns)) return;
            sweep<UPDATE>(a, lvl, Qout, qcount_next, nullptr);
        }
        unsigned int qnext = 0;
        if (!grid_barrier(ctrl, nblocks, a.phantom, gen, a.timeout_ns, qcount_next, &qnext)) return;
        if (qnext == 0) break;
        qprev = qn;
        qn = qnext;
    }
    if (gtid == 0) ctrl->levels = (unsigned int)lvl;
    // undo the reordering: out[v] = L[new_id[v]]
    if (a.new_id) {
        for (int v = gtid; v < a.n; v += nthreads) a.out[v] = ld_cg(&a.L[__ldg(&a.new_id[v])]);
    }
}

template <int UPDATE, int PULL, int UNROLL, int MINB>
__global__ void __launch_bounds__(kBfsBlock, MINB) bfs_kernel(BfsArgs a) {
    bfs_body<UPDATE, PULL, UNROLL>(a);
    fold_status(a.ctrl);
}

// Stage-1 pull of single tiles, for the exhaustive check of both back-ends.
template <int PULL>
__global__ void debug_pull_kernel(const uint32_t* __restrict__ masks, const uint8_t* __restrict__ alpha, int tiles,
                                  uint8_t* __restrict__ hits) {
    const int lane = threadIdx.x & 31;
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int t = w; t < tiles; t += nw) {
        const uint32_t m = masks[(size_t)t * kWarp + lane];
        hits[(size_t)t * kWarp + lane] = (uint8_t)pull_hits<PULL>(m, alpha[t], lane);
    }
}

// ---------------------------------------------------------------- launching

template <int UPDATE, int PULL, int UNROLL, int MINB>
static void* kernel_ptr() {
    return reinterpret_cast<void*>(&bfs_kernel<UPDATE, PULL, UNROLL, MINB>);
}

static void* pick_kernel(int update, int pull, int unroll, int minb) {
#define BLEST_PICK(U, P, R, M) \
    if (update == U && pull == P && unroll == R && minb == M) return kernel_ptr<U, P, R, M>();
#define BLEST_PICK_M(U, P, R) BLEST_PICK(U, P, R, 2) BLEST_PICK(U, P, R, 3)
    BLEST_PICK_M(1, 0, 1) BLEST_PICK_M(1, 0, 2) BLEST_PICK_M(1, 1, 1) BLEST_PICK_M(1, 1, 2)
    BLEST_PICK_M(2, 0, 1) BLEST_PICK_M(2, 0, 2) BLEST_PICK_M(2, 1, 1) BLEST_PICK_M(2, 1, 2)
#undef BLEST_PICK_M
#undef BLEST_PICK
    return nullptr;
}

int bfs_max_blocks_per_sm(int update, int pull, int unroll, int minb) {
    void* k = pick_kernel(update, pull, unroll, minb);
    if (!k) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kBfsBlock, 0) != cudaSuccess) return 0;
    return nb;
}

int bfs_threads_per_block() { return kBfsBlock; }

cudaError_t launch_debug_pull(const uint32_t* d_masks, const uint8_t* d_alpha, int32_t tiles, int pull,
                              uint8_t* d_hits, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>(((int64_t)tiles * kWarp + 255) / 256, 4096);
    if (pull == 1) debug_pull_kernel<1><<<blocks, 256, 0, st>>>(d_masks, d_alpha, tiles, d_hits);
    else debug_pull_kernel<0><<<blocks, 256, 0, st>>>(d_masks, d_alpha, tiles, d_hits);
    return cudaGetLastError();
}

cudaError_t launch_bfs_kernel(const BfsLaunch& L, cudaStream_t stream) {
    void* k = pick_kernel(L.update, L.pull, L.unroll, L.minb);
    if (!k) return cudaErrorInvalidValue;
    BfsArgs a;
    a.n = L.n;
    a.nwords = (L.n + 31) / 32;
    a.qcap = L.qcap;
    a.real_ptrs = L.real_ptrs;
    a.row_ids4 = reinterpret_cast<const int4*>(L.row_ids);
    a.masks = L.masks;
    a.new_id = L.new_id;
    a.L = L.levels_internal;
    a.vcur = L.vcur;
    a.vnext = L.vnext;
    for (int i = 0; i < 3; ++i) { a.F[i] = L.F[i]; a.Q[i] = L.Q[i]; }
    a.ctrl = reinterpret_cast<Ctrl*>(L.ctrl);
    a.level_sizes = L.level_sizes;
    a.level_cap = L.level_cap;
    a.roots = L.roots_device;
    a.nroots = L.nroots;
    for (int i = 0; i < kInlineRoots; ++i) a.inline_roots[i] = i < L.nroots ? L.roots_host[i] : 0;
    a.out = L.out;
    a.timeout_ns = L.timeout_ns;
    a.phantom = L.phantom;
    a.filter = L.filter;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel(k, dim3((unsigned)L.grid), dim3(kBfsBlock), args, 0, stream);
}

}  // namespace blest
