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
    int32_t n, nwords, nss;
    unsigned int qcap;
    const int32_t* __restrict__ real_ptrs;
    const int4* __restrict__ row_ids4;
    const uint32_t* __restrict__ masks;
    const int32_t* __restrict__ goff;     // compact layout: first group of each slice set (nss + 1)
    const int4* __restrict__ rows_c;      // compact layout: 4 row ids per group
    const uint32_t* __restrict__ masks_c; // compact layout: 4 packed masks per group
    const int32_t* __restrict__ new_id;  // NULL: identity, L is the output
    int32_t* L;
    // V_curr and V_next, dense bitmaps.  V_next always contains V_curr (stage 1 only
    // adds marks; the sweep copies V_next into V_curr), so a hit row's test against
    // both is one 4-byte load of its V_next word.
    uint32_t* vcur;
    uint32_t* vnext;
    uint32_t* dirty;                      // 1 bit per V_next word touched on a sparse level (NULL = never sparse)
    uint32_t* F[3];
    unsigned long long* Q[3];
    Ctrl* ctrl;
    int32_t* level_sizes;
    unsigned long long* level_times;      // with level_sizes: 2 globaltimer stamps per level
    unsigned long long* arrive_first;     // with level_sizes: earliest / latest block end of stage 1
    unsigned long long* arrive_last;      // (entries [0, cap)) and of the lazy sweep ([cap, 2 cap))
    int32_t level_cap;
    const int32_t* roots;                 // device list (used when nroots > kInlineRoots)
    int32_t nroots;
    int32_t inline_roots[kInlineRoots];
    int32_t* out;                         // output in original ids (unused when new_id is NULL)
    uint64_t timeout_ns;
    unsigned int phantom;
    int filter;                           // 1 = skip rows already in V_curr; 2/3 = also V_next (L2 / L1) while few are visited
    const int32_t* __restrict__ old_of;   // BVSS id -> original id (with direct)
    int direct;                           // 1: the sweeps write levels straight to out (original ids)
    int sched;                            // stage-1 schedule of the double-buffered path: 0 static, 1 dynamic
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
// LAYOUT 1 enqueues the slice set's VSSs of the compact layout (group offset,
// group count, alpha) instead of VSS ids.
//
// Sparse levels (stage 1 set a dirty bit per touched V_next word): the warp
// visits only the 32-word blocks whose dirty word is nonzero, clears it, and
// treats the other words of the block as unchanged.
//
// SHARD (sharded traversal): every rank sweeps every word, so all ranks finalise
// the same level, but a rank enqueues only the slice sets it owns (s mod world =
// rank), and the number of newly reached rows is always counted.
template <int UPDATE, int LAYOUT, bool SHARD = false>
__device__ __forceinline__ void sweep(const BfsArgs& a, int lvl, unsigned long long* Qout, unsigned long long* qcount,
                                      uint32_t* Fout, bool sparse, int world = 1, int rank = 0) {
    // Work split: in round k, warp w of block B takes the block of 32 words
    // B + (w + 16 k) gridDim.x, so consecutive 32-word blocks go to consecutive
    // thread blocks: the orderings put the hubs, whose slice sets carry most of
    // the queue entries, at the lowest ids, and one SM must not write them all
    // while the rest of the grid waits at the barrier.  Queue space is reserved
    // once per block and round (thread 0, after the warps posted their totals in
    // shared memory), not once per warp: the queue size is one address that
    // every block hits during a sweep.
    constexpr int kWarpsPerBlock = kBfsBlock / kWarp;
    __shared__ unsigned int s_off[kWarpsPerBlock];
    __shared__ unsigned int s_base;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nblk = (a.nwords + kWarp - 1) / kWarp;
    const int round = (int)gridDim.x * kWarpsPerBlock;
    unsigned int fresh = 0;   // rows this lane gave a level
    for (int r0 = (int)blockIdx.x; r0 < nblk; r0 += round) {   // block-uniform bound
        const int b = r0 + warp * (int)gridDim.x;
        const int t0 = b * kWarp;
        const int t = t0 + lane;
        uint32_t live = b < nblk ? 0xFFFFFFFFu : 0u;
        if (sparse && b < nblk) {
            live = ld_cg(&a.dirty[b]);   // the same word in every lane
            if (live != 0u && lane == 0) a.dirty[b] = 0u;
        }
        uint32_t diff = 0;
        int rp[5] = {0, 0, 0, 0, 0};   // VSS (or group) offsets of the word's 4 slice sets and the next
        if (t < a.nwords && ((live >> lane) & 1u)) {
            const uint32_t nx = ld_cg(&a.vnext[t]);
            const uint32_t cu = ld_cg(&a.vcur[t]);
            // issued with the bitmap loads, not after them: their addresses do not depend on diff
            const int32_t* ptrs = LAYOUT == 1 ? a.goff : a.real_ptrs;
#pragma unroll
            for (int q = 0; q < 5; ++q)
                if (4 * t + q <= a.nss) rp[q] = __ldg(&ptrs[4 * t + q]);
            diff = nx ^ cu;
            if (diff) {
                a.vcur[t] = nx;
                if (UPDATE == 1) Fout[t] = diff;
                fresh += (unsigned int)__popc(diff);
            }
        }
        // level writes, transposed: for each of the warp's 32 words with new
        // rows, the 32 lanes store that word's 32 levels as one coalesced line
        // (direct: each lane reads its row's original id, 8 words at a time so
        // that those reads overlap, and stores its level there)
        unsigned int pend = __ballot_sync(0xffffffffu, diff != 0u);
        if (a.direct) {
            while (pend) {
                int o[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    o[j] = -1;
                    if (pend) {
                        const int src = __ffs(pend) - 1;
                        pend &= pend - 1;
                        const uint32_t dw = __shfl_sync(0xffffffffu, diff, src);
                        if ((dw >> lane) & 1u) o[j] = __ldg(&a.old_of[(t0 + src) * kWarp + lane]);
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (o[j] >= 0) a.out[o[j]] = lvl;
            }
        } else {
            while (pend) {
                const int src = __ffs(pend) - 1;
                pend &= pend - 1;
                const uint32_t dw = __shfl_sync(0xffffffffu, diff, src);
                if ((dw >> lane) & 1u) a.L[(t0 + src) * kWarp + lane] = lvl;
            }
        }
        int st[4], ln[4], tot[4];
        uint32_t pay[4];
        unsigned int cnt = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t byte = (diff >> (8 * q)) & 0xFFu;
            st[q] = 0; ln[q] = 0; tot[q] = 0; pay[q] = 0;
            if (byte && (!SHARD || (4 * t + q) % world == rank)) {
                // a row of slice set s exists, so s < nss and rp[q + 1] was loaded
                const int s = 4 * t + q;
                st[q] = rp[q];
                if (LAYOUT == 1) {
                    tot[q] = rp[q + 1] - rp[q];
                    ln[q] = (tot[q] + 31) >> 5;
                } else {
                    ln[q] = rp[q + 1] - rp[q];
                }
                pay[q] = UPDATE == 2 ? byte : (uint32_t)s;
            }
            cnt += (unsigned int)ln[q];
        }
        const unsigned int incl = warp_inclusive_scan(cnt, lane);
        if (lane == 31) s_off[warp] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int run = 0;
            for (int w = 0; w < kWarpsPerBlock; ++w) {
                const unsigned int x = s_off[w];
                s_off[w] = run;
                run += x;
            }
            unsigned int base = 0;
            if (run) {
                base = (unsigned int)atomicAdd(qcount, (unsigned long long)run);
                if (base + run > a.qcap || base + run < base) {
                    raise_error(a.ctrl, 7u);
                    base = 0xFFFFFFFFu;
                }
            }
            s_base = base;
        }
        __syncthreads();
        // s_off and s_base are rewritten only after the next round's first barrier
        const unsigned int base = s_base;
        if (base != 0xFFFFFFFFu && __shfl_sync(0xffffffffu, incl, 31) != 0u)
            warp_write_entries<4, LAYOUT == 1>(Qout, base + s_off[warp] + incl - cnt, cnt, st, ln, pay, tot, lane);
    }
    if (UPDATE == 2 && (SHARD || a.filter >= 2)) {
        fresh = __reduce_add_sync(0xffffffffu, fresh);
        if (lane == 0 && fresh) atomicAdd(&a.ctrl->reached, fresh);
    }
}

// ---------------------------------------------------------- hit handling
// Each phase below issues its memory operations for all of a lane's hits
// (up to 4 per virtual slice set) before it uses any result, so a lane waits
// for one round trip per phase rather than one per hit.

// Lazy marking (Algorithm 3, stage 1): set the V_next bit of every hit row,
// skipping rows already in V_curr (visited filter, filt 1) and, with filt 2 or
// 3, rows another warp has already marked in V_next at this level (read at L2,
// or through L1 where a line can be older but the load is cheap).  Both bitmaps
// only gain bits during a traversal, so a stale (older) word can only let
// through a redundant mark, never suppress a needed one.  The V_next test pays
// off while most hit rows are unvisited (marks then repeat on the same rows)
// and costs an extra L2 load per hit once most are visited; the kernel applies
// it only while fewer than n/4 rows have a level.
template <int NV>
__device__ __forceinline__ void mark_rows(const BfsArgs& a, const int4 (&rows)[NV], unsigned int hm, int filt,
                                          uint32_t* dirty) {
    int u[4 * NV];
    uint32_t w[4 * NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        u[4 * i + 0] = rows[i].x; u[4 * i + 1] = rows[i].y; u[4 * i + 2] = rows[i].z; u[4 * i + 3] = rows[i].w;
    }
    if (filt == 2) {
#pragma unroll
        for (int k = 0; k < 4 * NV; ++k) {
            w[k] = 0u;
            if ((hm >> k) & 1u) {
                w[k] = ld_cg(&a.vnext[u[k] >> 5]);   // V_next contains V_curr
            }
        }
    } else if (filt == 3) {   // V_next through L1: staler, so more redundant marks, but cheaper loads
#pragma unroll
        for (int k = 0; k < 4 * NV; ++k) {
            w[k] = 0u;
            if ((hm >> k) & 1u) {
                w[k] = a.vnext[u[k] >> 5];
            }
        }
    } else if (filt) {
#pragma unroll
        for (int k = 0; k < 4 * NV; ++k) w[k] = (hm >> k) & 1u ? a.vcur[u[k] >> 5] : 0u;
    } else {
#pragma unroll
        for (int k = 0; k < 4 * NV; ++k) w[k] = 0u;
    }
#pragma unroll
    for (int k = 0; k < 4 * NV; ++k) {
        const uint32_t bit = 1u << (u[k] & 31);
        if (((hm >> k) & 1u) && !(w[k] & bit)) {
            atomicOr(&a.vnext[u[k] >> 5], bit);
            if (dirty) atomicOr(&dirty[u[k] >> 10], 1u << ((u[k] >> 5) & 31));
        }
    }
}

// Eager update (Algorithm 2): for every hit row not yet visited, set its level
// and its frontier bit with a returning atomicOr; the lane that sets the first
// bit of a slice set's frontier byte enqueues that slice set's VSS range.
template <int NV>
__device__ __forceinline__ void eager_update(const BfsArgs& a, const int4 (&rows)[NV], unsigned int hm, int lvl,
                                             uint32_t* Fnext, unsigned long long* Qout, unsigned long long* qcount_next,
                                             int lane) {
    constexpr int K = 4 * NV;
    int u[K];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        u[4 * i + 0] = rows[i].x; u[4 * i + 1] = rows[i].y; u[4 * i + 2] = rows[i].z; u[4 * i + 3] = rows[i].w;
    }
    // phase 1: visited filter on the V bitmap (a subset of the visited set)
    if (a.filter) {
        uint32_t w[K];
#pragma unroll
        for (int k = 0; k < K; ++k) w[k] = (hm >> k) & 1u ? a.vcur[u[k] >> 5] : 0u;
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (w[k] & (1u << (u[k] & 31))) hm &= ~(1u << k);
    }
    // phase 2: level check, with the VSS range of each hit row's slice set loaded
    // alongside (needed only if this lane claims the row, but it saves a round trip)
    int lv[K], rp0[K], rp1[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        lv[k] = 0; rp0[k] = 0; rp1[k] = 0;
        if ((hm >> k) & 1u) {
            lv[k] = ld_cg(&a.L[u[k]]);
            rp0[k] = __ldg(&a.real_ptrs[u[k] >> 3]);
            rp1[k] = __ldg(&a.real_ptrs[(u[k] >> 3) + 1]);
        }
    }
    unsigned int newm = 0;
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (((hm >> k) & 1u) && lv[k] < 0) newm |= 1u << k;
    // phase 3: claim
    uint32_t old[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        old[k] = 0xFFFFFFFFu;
        if ((newm >> k) & 1u) {
            const uint32_t bit = 1u << (u[k] & 31);
            a.L[u[k]] = lvl;
            if (a.filter) atomicOr(&a.vcur[u[k] >> 5], bit);
            old[k] = atomicOr(&Fnext[u[k] >> 5], bit);
        }
    }
    // phase 4: the first setter of a slice set's byte enqueues its VSS range
    int st[K], ln[K];
    uint32_t pay[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        st[k] = 0; ln[k] = 0; pay[k] = 0;
        if (((newm >> k) & 1u) && ((old[k] >> (u[k] & 24)) & 0xFFu) == 0) {
            st[k] = rp0[k];
            ln[k] = rp1[k] - rp0[k];
            pay[k] = (uint32_t)(u[k] >> 3);
        }
    }
    warp_enqueue<K>(a.qcap, a.ctrl, Qout, qcount_next, st, ln, pay, lane, ln);
}

// ---------------------------------------------------------- staged stage 1
// Lazy stage 1 with a per-warp TMA ring: lane 0 streams the 512-byte row-id and
// 128-byte mask tiles of the warp's upcoming virtual slice sets into a ring of
// DEPTH shared-memory stages with cp.async.bulk (L2 evict-first: the BVSS
// stream is read once per level and must not push the bitmaps and levels out
// of L2), each stage completing on its own mbarrier.  The warp processes tile
// k from shared memory while tiles k+1 .. k+DEPTH-1 are in flight, so memory
// parallelism does not depend on registers or occupancy.  Queue entries are
// fetched 32 at a time (one per lane) one window ahead.  Every mbarrier wait
// is bounded by the barrier timeout.
constexpr int kStageBytes = 512 + 128;

template <int DEPTH>
__host__ __device__ constexpr int ring_bytes_per_warp() { return DEPTH * (kStageBytes + 8); }

// All 32 lanes wait for the phase of parity `parity` of the mbarrier, bounded
// by timeout_ns; true when it completed.  Every lane takes part in each vote.
__device__ __forceinline__ bool warp_wait_stage(uint32_t bar, uint32_t parity, uint64_t timeout_ns) {
    bool done = mbar_try_wait(bar, parity);
    if (__all_sync(0xffffffffu, done)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (!done) done = mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, done)) return true;
        if (__any_sync(0xffffffffu, global_timer_ns() - t0 > timeout_ns)) return false;
    }
}

template <int PULL, int DEPTH, int U>
__device__ __forceinline__ bool stage1_staged(const BfsArgs& a, const unsigned long long* __restrict__ Qin,
                                              unsigned int qn, unsigned char* ring, uint32_t& uses, uint64_t pol,
                                              int lane, int gwarp, int nwarps, int filt, uint32_t* dirty) {
    static_assert(DEPTH >= 2 * U, "the ring must hold at least two groups of tiles");
    int4* rows = reinterpret_cast<int4*>(ring);
    uint32_t* msk = reinterpret_cast<uint32_t*>(ring + DEPTH * 512);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(ring + DEPTH * kStageBytes);
    const unsigned int nk = qn > (unsigned int)gwarp ? (qn - (unsigned int)gwarp + (unsigned int)nwarps - 1) / nwarps : 0u;
    if (nk == 0) return true;
    // queue entries k = 32 j + lane of window j, one window ahead (DEPTH + U <= 32)
    auto load_window = [&](unsigned int j) -> unsigned long long {
        const unsigned int k = j * 32u + (unsigned int)lane;
        return k < nk ? ld_cg(&Qin[(size_t)gwarp + (size_t)k * (size_t)nwarps]) : 0ull;
    };
    unsigned int wcur = 0;
    unsigned long long e0 = load_window(0);
    unsigned long long e1 = nk > 32u ? load_window(1) : 0ull;
    auto entry = [&](unsigned int k) -> unsigned long long {
        const unsigned long long x0 = __shfl_sync(0xffffffffu, e0, (int)(k & 31u));
        const unsigned long long x1 = __shfl_sync(0xffffffffu, e1, (int)(k & 31u));
        return (k >> 5) == wcur ? x0 : x1;
    };
    auto issue = [&](unsigned int k) {
        const unsigned long long ent = entry(k);
        if (lane == 0) {
            const uint32_t s = (uses + k) % DEPTH;
            const uint32_t nu = (uint32_t)ent;
            const uint32_t bar = smem_addr(&bars[s]);
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, kStageBytes);
            bulk_g2s(smem_addr(&rows[s * 32]), a.row_ids4 + (size_t)nu * kWarp, 512, bar, pol);
            bulk_g2s(smem_addr(&msk[s * 32]), a.masks + (size_t)nu * kWarp, 128, bar, pol);
        }
    };
    const unsigned int pro = nk < (unsigned int)DEPTH ? nk : (unsigned int)DEPTH;
    for (unsigned int k = 0; k < pro; ++k) issue(k);
    for (unsigned int k = 0; k < nk; k += U) {
        if ((k >> 5) != wcur) {   // U divides 32, so a group never straddles two windows
            e0 = e1;
            ++wcur;
            e1 = (wcur + 1u) * 32u < nk ? load_window(wcur + 1u) : 0ull;
        }
        int4 r[U];
        uint32_t m[U], alpha[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            r[j] = make_int4(0, 0, 0, 0);
            m[j] = 0u;
            alpha[j] = 0u;
            if (k + j >= nk) continue;
            const uint32_t g = uses + k + j;
            const uint32_t s = g % DEPTH;
            if (!warp_wait_stage(smem_addr(&bars[s]), (g / DEPTH) & 1u, a.timeout_ns)) {
                // give up: record the timeout, then wait (bounded again) for this warp's
                // other copies in flight so that none lands after the block has left
                if (lane == 0) raise_error(a.ctrl, 6u);
                for (unsigned int t = k + j + 1; t < nk && t < k + j + DEPTH; ++t)
                    warp_wait_stage(smem_addr(&bars[(uses + t) % DEPTH]), ((uses + t) / DEPTH) & 1u, a.timeout_ns);
                uses += nk;
                return false;
            }
            r[j] = rows[s * 32 + lane];
            m[j] = msk[s * 32 + lane];
            alpha[j] = (uint32_t)(entry(k + j) >> 32) & 0xFFu;
        }
        __syncwarp();   // the stages may be refilled once every lane holds its tiles in registers
#pragma unroll
        for (int j = 0; j < U; ++j)
            if (k + j + DEPTH < nk) issue(k + j + DEPTH);
        unsigned int hm = 0;
#pragma unroll
        for (int j = 0; j < U; ++j) hm |= pull_hits<PULL>(m[j], alpha[j], lane) << (4 * j);
        mark_rows<U>(a, r, hm, filt, dirty);
    }
    uses += nk;
    return true;
}

// ------------------------------------------------------------- unpermute
// out[v] = L[new_id[v]] in original ids, eight vertices per thread in flight
// (traversals whose sweeps wrote L, not out directly).
__device__ __forceinline__ void unpermute(const BfsArgs& a, int gtid, int nthreads) {
    constexpr int K = 8;
    for (int64_t b = gtid; b < a.n; b += (int64_t)K * nthreads) {
        int u[K];
        int lv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int64_t v = b + (int64_t)k * nthreads;
            u[k] = v < a.n ? __ldg(&a.new_id[v]) : -1;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) lv[k] = u[k] >= 0 ? ld_cg(&a.L[u[k]]) : -1;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int64_t v = b + (int64_t)k * nthreads;
            if (v < a.n) a.out[v] = lv[k];
        }
    }
}

// --------------------------------------------------------- tile loads
// The lane's 4 row ids and 4 packed masks of a queued virtual slice set.
// Layout 0 (Section 3.1.2): every VSS holds 32 lanes x 4 slices, padded.
// Layout 1 (compact): the VSS is ng = bits 40..44 + 1 consecutive groups of 4
// slices starting at group bits 0..31; lanes >= ng hold nothing (mask 0).
// Both streams are read once per level, with an L2 evict-first hint.
template <int LAYOUT>
__device__ __forceinline__ void load_tile(const BfsArgs& a, unsigned long long e, int lane, uint64_t pol, int4& r,
                                          uint32_t& m) {
    if (LAYOUT == 1) {
        const uint32_t ng = (uint32_t)(e >> 40) + 1u;
        if ((uint32_t)lane < ng) {
            const size_t g = (size_t)(uint32_t)e + (size_t)lane;
            r = ld_stream_v4(&a.rows_c[g], pol);
            m = ld_stream_u32(&a.masks_c[g], pol);
        }
    } else {
        const size_t tile = (size_t)(uint32_t)e * kWarp + lane;
        r = ld_stream_v4(&a.row_ids4[tile], pol);
        m = ld_stream_u32(&a.masks[tile], pol);
    }
}

// ------------------------------------------------ double-buffered stage 1
// Lazy stage 1 with a two-deep software pipeline in registers: while the hits
// of group g are filtered and marked, the row-id and mask tiles of group g+1
// are already in flight and the queue entries of group g+2 are being read, so
// a warp no longer waits for the queue, the tiles and the filter one after
// another.  A group is U queue entries.
//
// Schedules.  Static (sched 0): warp w takes entries w, w + W, w + 2W, ... (W =
// warps), U at a time.  Static + dynamic tail (sched 1, on queues of at least
// 16 entries per warp): the first 7/8 of the queue is split statically as
// above, and a warp that has finished its static
// share takes chunks of the last 1/8 from the level's counter in the control
// block (guided self-scheduling: (entries left) / 2W at its previous grab,
// within [2U, 64]), so blocks on faster SMs absorb the end of the level.
constexpr unsigned int kChunkMax = 64;

template <int PULL, int U, int LAYOUT, int PD>
__device__ __forceinline__ void stage1_pipelined(const BfsArgs& a, const unsigned long long* __restrict__ Qin,
                                                 unsigned int qn, uint64_t pol, int lane, int gwarp, int nwarps,
                                                 int filt, unsigned int* work, uint32_t* dirty) {
    // the dynamic tail only pays on long queues: on a short one nearly every warp
    // would go straight to the counter and the atomics would serialise
    const bool dyn = work != nullptr && qn >= 16u * (unsigned int)nwarps;
    const unsigned int stride = (unsigned int)nwarps * U;
    const unsigned int slim = dyn ? qn - qn / 8u : qn;   // end of the static part
    unsigned int sbase = (unsigned int)gwarp;
    if (!dyn && sbase >= qn) return;
    unsigned int c_lo = 0, c_hi = 0, seen = slim;   // dynamic tail: current chunk, last position seen
    // the queue entries of the warp's next group (~0 past the end; positions only grow)
    auto next_group = [&](unsigned long long (&e)[U]) {
        unsigned int p[U];
        if (sbase < slim) {
#pragma unroll
            for (int i = 0; i < U; ++i) {
                const unsigned int q = sbase + (unsigned int)i * (unsigned int)nwarps;
                p[i] = q < slim ? q : 0xFFFFFFFFu;
            }
            sbase += stride;
        } else if (dyn) {
            if (c_lo >= c_hi && seen < qn) {
                const unsigned int left = qn - seen;
                unsigned int c = left / (2u * (unsigned int)nwarps);
                c = c < 2u * U ? 2u * U : (c > kChunkMax ? kChunkMax : c);
                unsigned int s0 = 0;
                if (lane == 0) s0 = atomicAdd(work, c);
                s0 = __shfl_sync(0xffffffffu, s0, 0);
                const unsigned int left_now = qn - slim;             // positions slim + [0, left_now)
                seen = s0 < left_now ? slim + s0 : qn;
                c_lo = seen;
                c_hi = s0 < left_now ? (left_now - s0 < c ? qn : seen + c) : qn;
            }
#pragma unroll
            for (int i = 0; i < U; ++i) p[i] = c_lo + (unsigned int)i < c_hi ? c_lo + (unsigned int)i : 0xFFFFFFFFu;
            c_lo = c_lo + U < c_hi ? c_lo + U : c_hi;
        } else {
#pragma unroll
            for (int i = 0; i < U; ++i) p[i] = 0xFFFFFFFFu;
        }
#pragma unroll
        for (int i = 0; i < U; ++i) e[i] = p[i] != 0xFFFFFFFFu ? ld_cg(&Qin[p[i]]) : ~0ull;
    };
    auto fetch_tiles = [&](const unsigned long long (&e)[U], int4 (&r)[U], uint32_t (&m)[U]) {
#pragma unroll
        for (int i = 0; i < U; ++i) {
            r[i] = make_int4(0, 0, 0, 0);
            m[i] = 0u;
            if (e[i] != ~0ull) load_tile<LAYOUT>(a, e[i], lane, pol, r[i], m[i]);
        }
    };
    // PD = prefetch distance: the tiles of the next PD groups are in flight and the
    // queue entries of the group after them are being read while group 0 is handled
    unsigned long long e[PD + 2][U];
    int4 r[PD + 1][U];
    uint32_t m[PD + 1][U];
#pragma unroll
    for (int k = 0; k < PD; ++k) {
        next_group(e[k]);
        fetch_tiles(e[k], r[k], m[k]);
    }
    next_group(e[PD]);
    while (e[0][0] != ~0ull) {
        fetch_tiles(e[PD], r[PD], m[PD]);
        next_group(e[PD + 1]);
        unsigned int hm = 0;
#pragma unroll
        for (int i = 0; i < U; ++i)   // e[0][i] is the same in every lane, so the MMA runs warp-wide
            if (e[0][i] != ~0ull) hm |= pull_hits<PULL>(m[0][i], (uint32_t)(e[0][i] >> 32) & 0xFFu, lane) << (4 * i);
        mark_rows<U>(a, r[0], hm, filt, dirty);
#pragma unroll
        for (int k = 0; k < PD; ++k)
#pragma unroll
            for (int i = 0; i < U; ++i) {
                r[k][i] = r[k + 1][i];
                m[k][i] = m[k + 1][i];
            }
#pragma unroll
        for (int k = 0; k <= PD; ++k)
#pragma unroll
            for (int i = 0; i < U; ++i) e[k][i] = e[k + 1][i];
    }
}

// -------------------------------------------------------------------- kernel

template <int UPDATE, int PULL, int UNROLL, int DEPTH, int LAYOUT>
__device__ __forceinline__ void bfs_body(const BfsArgs& a) {
    const int lane = threadIdx.x & 31;
    const int gtid = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int nthreads = (int)(gridDim.x * blockDim.x);
    const int gwarp = gtid >> 5;
    const int nwarps = nthreads >> 5;
    const unsigned int nblocks = gridDim.x;
    unsigned int bar = 0;   // barriers passed; the next one is number bar
    Ctrl* ctrl = a.ctrl;
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    // DEPTH 4 or 8: a shared-memory ring per warp; DEPTH 2 and 3 keep their stages in registers
    unsigned char* ring = dyn_smem + (threadIdx.x >> 5) * (DEPTH > 3 ? ring_bytes_per_warp<DEPTH>() : 0);
    uint32_t ring_uses = 0;
    const uint64_t pol = l2_evict_first_policy();
    if (DEPTH > 3) {
        if (lane == 0) {
            unsigned long long* bars = reinterpret_cast<unsigned long long*>(ring + DEPTH * kStageBytes);
            for (int i = 0; i < DEPTH; ++i) mbar_init(smem_addr(&bars[i]), 1);
            mbar_init_fence();
        }
        __syncwarp();
    }

    if (gtid == 0 && a.level_sizes) a.level_times[1] = global_timer_ns();   // kernel entry (block 0)
    // level 0: mark the sources (V_curr, V_next and the dirty bits were cleared before launch).
    // A level is sparse when its queue (or source list) is short against the bitmap: then
    // stage 1 records the V_next words it touches and the sweep visits only those.
    const unsigned int sparse_cap = a.dirty ? (unsigned int)(a.nwords >> 6) : 0u;
    const bool sparse0 = a.dirty != nullptr && (unsigned int)a.nroots <= sparse_cap;
    for (int i = gtid; i < a.nroots; i += nthreads) {
        const int r = a.nroots <= kInlineRoots ? a.inline_roots[i] : a.roots[i];
        atomicOr(&a.vnext[r >> 5], 1u << (r & 31));
        if (sparse0) atomicOr(&a.dirty[r >> 10], 1u << ((r >> 5) & 31));
    }
    if (!grid_barrier(ctrl, nblocks, a.phantom, bar, a.timeout_ns)) return;
    if (gtid == 0 && a.level_sizes) a.level_times[0] = global_timer_ns();
    sweep<UPDATE, LAYOUT>(a, 0, a.Q[1], ring_word(ctrl, bar), a.F[1], sparse0);
    unsigned int qn = 0, qprev = 0;
    if (!grid_barrier(ctrl, nblocks, a.phantom, bar, a.timeout_ns, &qn)) return;

    int lvl = 1;
    for (;; ++lvl) {
        if (qn > a.qcap) qn = a.qcap;   // only after an overflow, which already raised an error
        if (gtid == 0) {
            ctrl->work[(lvl + 1) & 1] = 0;   // counter of the next level (this level's is work[lvl & 1])
            if (a.level_sizes && lvl - 1 < a.level_cap) {
                a.level_sizes[lvl - 1] = (int32_t)qn;
                a.level_times[2 * lvl] = global_timer_ns();    // stage 1 of level lvl starts
            }
        }
        const unsigned long long* Qin = a.Q[lvl % 3];
        if (UPDATE == 1) {
            // clear the frontier bytes of level lvl-1 (read last level, rewritten at lvl+1),
            // counted from the last thread of the grid: on a short queue the stage-1 items
            // go to the first warps, and a clear (a store that waits for its queue load)
            // would delay their loads by a round trip
            const unsigned long long* Qp = a.Q[(lvl + 2) % 3];
            unsigned char* Fold = reinterpret_cast<unsigned char*>(a.F[(lvl + 2) % 3]);
            for (unsigned int i = (unsigned int)(nthreads - 1 - gtid); i < qprev; i += (unsigned int)nthreads)
                Fold[(uint32_t)(ld_cg(&Qp[i]) >> 32)] = 0;
        }
        const uint32_t* Fcur = a.F[lvl % 3];
        uint32_t* Fnext = a.F[(lvl + 1) % 3];
        unsigned long long* Qout = a.Q[(lvl + 1) % 3];
        // the next queue's size: the word of the barrier that ends this level
        // (the lazy update passes one barrier between stage 1 and its sweep)
        unsigned long long* qcount_next = ring_word(ctrl, bar + (UPDATE == 2 ? 1u : 0u));

        // stage 1: pull the queued virtual slice sets, round-robin over warps
        // the lazy filter of this level: the V_next test only while few rows are visited
        // filters 2 and 3 test V_next while fewer than n/4 rows are visited, then V_curr;
        // filter 4 tests V_next (through L1) at every level
        const int filt = a.filter == 4 ? 3
                                       : ((a.filter >= 2 && ld_cg(&ctrl->reached) >= (unsigned int)a.n / 4u) ? 1
                                                                                                          : a.filter);
        const bool sparse = UPDATE == 2 && a.dirty != nullptr && qn <= sparse_cap;
        uint32_t* dirty = sparse ? a.dirty : nullptr;
        if (DEPTH == 2 || DEPTH == 3) {
            stage1_pipelined<PULL, UNROLL, LAYOUT, (DEPTH == 3 ? 2 : 1)>(a, Qin, qn, pol, lane, gwarp, nwarps, filt,
                                                   a.sched ? &ctrl->work[lvl & 1] : nullptr, dirty);
        } else if (DEPTH > 3) {
            stage1_staged<PULL, (DEPTH > 3 ? DEPTH : 2 * UNROLL), UNROLL>(a, Qin, qn, ring, ring_uses, pol, lane,
                                                                            gwarp, nwarps, filt, dirty);
        } else
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
                rows[i] = make_int4(0, 0, 0, 0);
                msk[i] = 0u;
                if (ent[i] != ~0ull) load_tile<LAYOUT>(a, ent[i], lane, pol, rows[i], msk[i]);
            }
            if (UPDATE == 2) {
                unsigned int hm = 0;   // bit 4i+q: sub-slot q of VSS i hit
#pragma unroll
                for (int i = 0; i < UNROLL; ++i)
                    if (ent[i] != ~0ull)
                        hm |= pull_hits<PULL>(msk[i], (uint32_t)(ent[i] >> 32) & 0xFFu, lane) << (4 * i);
                mark_rows<UNROLL>(a, rows, hm, filt, dirty);
            } else {
                uint32_t alpha[UNROLL];
#pragma unroll
                for (int i = 0; i < UNROLL; ++i) {
                    alpha[i] = 0;
                    if (ent[i] != ~0ull) {
                        const uint32_t s = (uint32_t)(ent[i] >> 32);
                        alpha[i] = (ld_cg(&Fcur[s >> 2]) >> (8 * (s & 3))) & 0xFFu;
                    }
                }
                unsigned int hm = 0;
#pragma unroll
                for (int i = 0; i < UNROLL; ++i)   // every lane runs the pull (the MMA needs the full warp)
                    hm |= (ent[i] != ~0ull ? pull_hits<PULL>(msk[i], alpha[i], lane) : 0u) << (4 * i);
                eager_update<UNROLL>(a, rows, hm, lvl, Fnext, Qout, qcount_next, lane);
            }
        }
        if (a.level_sizes && lvl - 1 < a.level_cap) {
            // record when this block finished stage 1 (first and last over blocks)
            __syncthreads();
            if (threadIdx.x == 0) {
                const unsigned long long t = global_timer_ns();
                atomicMin(&a.arrive_first[lvl - 1], t);
                atomicMax(&a.arrive_last[lvl - 1], t);
            }
        }
        if (UPDATE == 2) {
            if (!grid_barrier(ctrl, nblocks, a.phantom, bar, a.timeout_ns)) return;
            if (gtid == 0 && a.level_sizes && lvl - 1 < a.level_cap) a.level_times[2 * lvl + 1] = global_timer_ns();
            sweep<UPDATE, LAYOUT>(a, lvl, Qout, qcount_next, nullptr, sparse);
            if (a.level_sizes && lvl - 1 < a.level_cap) {
                __syncthreads();
                if (threadIdx.x == 0) {
                    const unsigned long long t = global_timer_ns();
                    atomicMin(&a.arrive_first[a.level_cap + lvl - 1], t);
                    atomicMax(&a.arrive_last[a.level_cap + lvl - 1], t);
                }
            }
        }
        unsigned int qnext = 0;
        if (!grid_barrier(ctrl, nblocks, a.phantom, bar, a.timeout_ns, &qnext)) return;
        if (qnext == 0) break;
        qprev = qn;
        qn = qnext;
    }
    if (gtid == 0) {
        ctrl->levels = (unsigned int)lvl;
        if (a.level_sizes && lvl < a.level_cap) a.level_times[2 * lvl + 2] = global_timer_ns();   // traversal end
    }
    // undo the reordering: out[v] = L[new_id[v]]
    if (a.new_id && !a.direct) unpermute(a, gtid, nthreads);
    if (a.level_sizes && lvl < a.level_cap) {
        __syncthreads();
        if (gtid == 0) a.level_times[2 * lvl + 3] = global_timer_ns();   // block 0 done with its share
    }
}

// ------------------------------------------------------- sharded traversal
// One rank's share of a single-source traversal whose pull is partitioned by
// slice set (rank r owns the slice sets s with s mod world = r), one launch per
// step so that the ranks' exchange of V_next words sits between the steps of a
// level: pull (stage 1 over the rank's own queue), then, after the exchange, the
// finalisation sweep of the merged words, identical on every rank.  Lazy update,
// padded layout, queues Q[level & 1].

// Level 0: mark the root in V_next, then the level-0 sweep.
__global__ void shard_root_kernel(BfsArgs a, int32_t root) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.vnext[root >> 5], 1u << (root & 31));
}

__global__ void __launch_bounds__(kBfsBlock, 2) shard_pull_kernel(BfsArgs a, int lvl) {
    const int lane = threadIdx.x & 31;
    const int gtid = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int gwarp = gtid >> 5;
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    Ctrl* ctrl = a.ctrl;
    // the queue sizes are ring words 0 and 1 (no grid barrier runs in these launches)
    unsigned int qn = (unsigned int)ld_cg(ring_word(ctrl, (unsigned int)lvl & 1u));
    if (qn > a.qcap) qn = a.qcap;   // only after an overflow, which already raised an error
    if (gtid == 0) *ring_word(ctrl, (unsigned int)(lvl + 1) & 1u) = 0ull;   // written by this level's sweep
    const int filt = a.filter == 4 ? 3
                                   : ((a.filter >= 2 && ld_cg(&ctrl->reached) >= (unsigned int)a.n / 4u) ? 1
                                                                                                      : a.filter);
    stage1_pipelined<0, 2, 0, 1>(a, a.Q[lvl & 1], qn, l2_evict_first_policy(), lane, gwarp, nwarps, filt, nullptr,
                                 nullptr);
    fold_status(ctrl);
}

__global__ void __launch_bounds__(kBfsBlock, 2) shard_sweep_kernel(BfsArgs a, int lvl, int world, int rank) {
    sweep<2, 0, true>(a, lvl, a.Q[(lvl + 1) & 1], ring_word(a.ctrl, (unsigned int)(lvl + 1) & 1u), nullptr, false,
                      world, rank);
    fold_status(a.ctrl);
}

// The rank's V_next words out (to_vis = 0) or the merged words in (to_vis = 1).
__global__ void shard_words_kernel(uint32_t* vnext, uint32_t* words, int nwords, int to_vis) {
    for (int t = (int)(blockIdx.x * blockDim.x + threadIdx.x); t < nwords; t += (int)(gridDim.x * blockDim.x)) {
        if (to_vis) vnext[t] = words[t];
        else words[t] = vnext[t];
    }
}

// dst[i] = OR over j < count of src[j * words + i]: the merge of all-gathered words.
__global__ void or_words_kernel(uint32_t* dst, const uint32_t* src, int64_t words, int count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v = 0u;
        for (int j = 0; j < count; ++j) v |= __ldg(&src[(int64_t)j * words + i]);
        dst[i] = v;
    }
}

template <int UPDATE, int PULL, int UNROLL, int MINB, int DEPTH, int LAYOUT>
__global__ void __launch_bounds__(kBfsBlock, MINB) bfs_kernel(BfsArgs a) {
    bfs_body<UPDATE, PULL, UNROLL, DEPTH, LAYOUT>(a);
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

template <int UPDATE, int PULL, int UNROLL, int MINB, int DEPTH, int LAYOUT>
static void* kernel_ptr() {
    return reinterpret_cast<void*>(&bfs_kernel<UPDATE, PULL, UNROLL, MINB, DEPTH, LAYOUT>);
}

static void* pick_kernel(int update, int pull, int unroll, int minb, int depth, int layout) {
    if (layout == 1) {
        // compact layout: lazy, register path (plain or double-buffered), 2 blocks per SM
#define BLEST_PICK_C(P, R, D) \
    if (update == 2 && pull == P && unroll == R && minb == 2 && depth == D) return kernel_ptr<2, P, R, 2, D, 1>();
        BLEST_PICK_C(0, 1, 0) BLEST_PICK_C(0, 2, 0) BLEST_PICK_C(0, 1, 2) BLEST_PICK_C(0, 2, 2)
        BLEST_PICK_C(1, 1, 0) BLEST_PICK_C(1, 2, 0) BLEST_PICK_C(1, 1, 2) BLEST_PICK_C(1, 2, 2)
#undef BLEST_PICK_C
        return nullptr;
    }
#define BLEST_PICK(U, P, R, M, D) \
    if (update == U && pull == P && unroll == R && minb == M && depth == D) return kernel_ptr<U, P, R, M, D, 0>();
#define BLEST_PICK_M(U, P, R) BLEST_PICK(U, P, R, 2, 0) BLEST_PICK(U, P, R, 3, 0)
    BLEST_PICK_M(1, 0, 1) BLEST_PICK_M(1, 0, 2) BLEST_PICK_M(1, 1, 1) BLEST_PICK_M(1, 1, 2)
    BLEST_PICK_M(2, 0, 1) BLEST_PICK_M(2, 0, 2) BLEST_PICK_M(2, 1, 1) BLEST_PICK_M(2, 1, 2)
    // staged (TMA ring) lazy variants: ring depth 4 or 8, unroll = tiles consumed per step
#define BLEST_PICK_S(P) BLEST_PICK(2, P, 1, 2, 4) BLEST_PICK(2, P, 2, 2, 4) BLEST_PICK(2, P, 1, 2, 8) \
    BLEST_PICK(2, P, 2, 2, 8) BLEST_PICK(2, P, 4, 2, 8)
    BLEST_PICK_S(0) BLEST_PICK_S(1)
    // register-pipelined lazy variants (depth 2: tiles one group ahead, 3: two groups ahead)
    BLEST_PICK(2, 0, 1, 2, 2) BLEST_PICK(2, 0, 2, 2, 2) BLEST_PICK(2, 1, 1, 2, 2) BLEST_PICK(2, 1, 2, 2, 2)
    BLEST_PICK(2, 0, 1, 2, 3) BLEST_PICK(2, 0, 2, 2, 3) BLEST_PICK(2, 1, 1, 2, 3) BLEST_PICK(2, 1, 2, 2, 3)
#undef BLEST_PICK_S
#undef BLEST_PICK_M
#undef BLEST_PICK
    return nullptr;
}

static size_t ring_smem_bytes(int depth) {
    if (depth == 4) return (size_t)(kBfsBlock / kWarp) * ring_bytes_per_warp<4>();
    if (depth == 8) return (size_t)(kBfsBlock / kWarp) * ring_bytes_per_warp<8>();
    return 0;
}

int bfs_max_blocks_per_sm(int update, int pull, int unroll, int minb, int depth, int layout) {
    void* k = pick_kernel(update, pull, unroll, minb, depth, layout);
    if (!k) return 0;
    const size_t smem = ring_smem_bytes(depth);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    // the register paths keep almost nothing in shared memory: give L1 the whole
    // carveout, where the visited-filter words of stage 1 are cached
    if (smem == 0) cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kBfsBlock, smem) != cudaSuccess) return 0;
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

static BfsArgs make_args(const BfsLaunch& L) {
    BfsArgs a;
    a.n = L.n;
    a.nwords = (L.n + 31) / 32;
    a.nss = (L.n + 7) / 8;
    a.qcap = L.qcap;
    a.real_ptrs = L.real_ptrs;
    a.row_ids4 = reinterpret_cast<const int4*>(L.row_ids);
    a.masks = L.masks;
    a.goff = L.goff;
    a.rows_c = reinterpret_cast<const int4*>(L.rows_c);
    a.masks_c = L.masks_c;
    a.new_id = L.new_id;
    a.L = L.levels_internal;
    a.vcur = L.vcur;
    a.vnext = L.vnext;
    a.dirty = L.dirty;
    for (int i = 0; i < 3; ++i) { a.F[i] = L.F[i]; a.Q[i] = L.Q[i]; }
    a.ctrl = reinterpret_cast<Ctrl*>(L.ctrl);
    a.level_sizes = L.level_sizes;
    a.level_times = L.level_times;
    a.arrive_first = L.arrive_first;
    a.arrive_last = L.arrive_last;
    a.level_cap = L.level_cap;
    a.roots = L.roots_device;
    a.nroots = L.nroots;
    for (int i = 0; i < kInlineRoots; ++i) a.inline_roots[i] = i < L.nroots ? L.roots_host[i] : 0;
    a.out = L.out;
    a.timeout_ns = L.timeout_ns;
    a.phantom = L.phantom;
    a.filter = L.filter;
    a.old_of = L.old_of;
    a.direct = L.direct;
    a.sched = L.sched;
    return a;
}

cudaError_t launch_bfs_kernel(const BfsLaunch& L, cudaStream_t stream) {
    void* k = pick_kernel(L.update, L.pull, L.unroll, L.minb, L.depth, L.layout);
    if (!k) return cudaErrorInvalidValue;
    const size_t smem = ring_smem_bytes(L.depth);
    BfsArgs a = make_args(L);
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel(k, dim3((unsigned)L.grid), dim3(kBfsBlock), args, smem, stream);
}

cudaError_t launch_shard_step(const BfsLaunch& L, int step, int lvl, int world, int rank, int32_t root,
                              uint32_t* words, cudaStream_t stream) {
    const BfsArgs a = make_args(L);
    const int nwords = (L.n + 31) / 32;
    const int wblocks = (int)std::min<int64_t>(((int64_t)nwords + 255) / 256, 4096);
    switch (step) {
        case kShardRoot:
            shard_root_kernel<<<1, 32, 0, stream>>>(a, root);
            break;
        case kShardPull:
            shard_pull_kernel<<<L.grid, kBfsBlock, 0, stream>>>(a, lvl);
            break;
        case kShardWordsOut:
            shard_words_kernel<<<std::max(wblocks, 1), 256, 0, stream>>>(a.vnext, words, nwords, 0);
            break;
        case kShardWordsIn:
            shard_words_kernel<<<std::max(wblocks, 1), 256, 0, stream>>>(a.vnext, words, nwords, 1);
            break;
        case kShardSweep:
            shard_sweep_kernel<<<L.grid, kBfsBlock, 0, stream>>>(a, lvl, world, rank);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_or_words(uint32_t* dst, const uint32_t* src, int64_t words, int count, cudaStream_t stream) {
    const int blocks = (int)std::min<int64_t>((words + 255) / 256, 4096);
    or_words_kernel<<<std::max(blocks, 1), 256, 0, stream>>>(dst, src, words, count);
    return cudaGetLastError();
}

}  // namespace blest
