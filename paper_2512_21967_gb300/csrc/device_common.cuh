// Device helpers shared by the BLEST kernels: a bounded grid barrier for
// persistent cooperative kernels, global-timer reads, L1-bypassing loads of
// state that other SMs write during a launch, and warp scans.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace blest {

constexpr int kWarp = 32;

// Control block (device memory, zeroed before every traversal).
struct Ctrl {
    unsigned int spare0;
    unsigned int error;        // first blest_status raised on the device (0 = none)
    unsigned int spare1[4];
    unsigned int levels;       // levels processed
    unsigned int reached;      // rows given a level so far (counted only when a filter needs it)
    unsigned int work[2];      // dynamic stage-1 schedule: next queue position, index = level & 1
    unsigned int pad[6];
};
static_assert(sizeof(Ctrl) == 64, "Ctrl is one 64-byte block");

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int* p) {
    return *(const volatile unsigned int*)p;
}

// Loads of data written by other blocks in the same launch: cache at L2 only.
template <class T>
__device__ __forceinline__ T ld_cg(const T* p) { return __ldcg(p); }

// Control words live in one 256-byte device block: the Ctrl struct at byte 0,
// the grid barrier's ring of four 64-bit words alone on the cache line at byte
// 128, and the sticky status word at byte 192.  Bytes [0, 192) are cleared
// before every traversal.
constexpr int kCtrlBytes = 256;
constexpr int kCtrlClearBytes = 192;
constexpr int kRingWord = 32;     // unsigned-int index of the barrier ring
constexpr int kStickyWord = 48;   // unsigned-int index of the sticky status

// Word i of the barrier ring.  Barrier number b of a launch uses word b & 3: its
// high half counts the blocks that arrived, its low half is the size of the
// queue that the phase ending at barrier b fills (the queue appends add to it),
// so the next level's queue size comes back with the load that sees the last
// arrival.  The low half never carries into the high half: a phase appends each
// VSS at most once and VSS indices are 32-bit.
__device__ __forceinline__ unsigned long long* ring_word(void* ctrl, unsigned int i) {
    return reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned int*>(ctrl) + kRingWord) + (i & 3u);
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Reduction with release semantics at GPU scope: it releases the calling
// thread's earlier writes (and, through a preceding __syncthreads, its block's).
__device__ __forceinline__ void red_release_gpu_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_gpu_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid barrier for a cooperative launch (all blocks co-resident).  `count` is
// the number of barriers this block has passed (the same in every block and
// every thread); barrier number b uses ring word b & 3 (see ring_word).  Thread
// 0 of each block arrives by adding 1 << 32 to the word with a release
// reduction, which releases its block's writes (ordered before it by
// __syncthreads), and polls the word with acquire loads until all
// nblocks + extra arrivals are counted.  The load that sees the last arrival has
// acquired every block's writes and carries the low half, which every block
// returns through *published (the next queue size).  Block 0 then clears word
// (b + 2) & 3: every block has arrived at barrier b, so none still polls barrier
// b - 2, the word's previous use; and the clear is released with block 0's
// arrival at barrier b + 1, before which no block adds to the word or arrives on
// it.  The wait is bounded: after timeout_ns it records BLEST_ERR_TIMEOUT (6) in
// ctrl->error and returns false, as it does when an error has been recorded (read
// with the first poll and every 32 polls; an error recorded by a block arriving
// late is seen at the next barrier).  `extra` adds phantom participants (test
// hook: a barrier that can never complete).
__device__ __forceinline__ bool grid_barrier(Ctrl* ctrl, unsigned int nblocks, unsigned int extra,
                                             unsigned int& count, uint64_t timeout_ns,
                                             unsigned int* published = nullptr) {
    __shared__ int s_ok;
    __shared__ unsigned int s_pub;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long* w = ring_word(ctrl, count);
        const unsigned int need = nblocks + extra;
        red_release_gpu_u64(w, 1ull << 32);
        unsigned int err = ld_volatile_u32(&ctrl->error);   // in flight with the first poll
        unsigned long long f = 0;
        const uint64_t t0 = global_timer_ns();
        unsigned int spins = 0;
        for (;;) {
            f = ld_acquire_gpu_u64(w);
            if ((unsigned int)(f >> 32) >= need) break;
            if ((++spins & 31u) == 0) {
                err |= ld_volatile_u32(&ctrl->error);
                if (err) break;
                if (global_timer_ns() - t0 > timeout_ns) {
                    atomicCAS(&ctrl->error, 0u, 6u);
                    err = 6u;
                    break;
                }
            }
            if (spins > 64) __nanosleep(32);
        }
        if (err == 0u && blockIdx.x == 0) st_relaxed_gpu_u64(ring_word(ctrl, count + 2u), 0ull);
        s_ok = err == 0u;
        s_pub = (unsigned int)f;
    }
    __syncthreads();
    count += 1u;
    if (published) *published = s_pub;
    return s_ok != 0;
}

// ------------------------------------------------ TMA bulk copies + mbarriers

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Generic-proxy accesses to shared memory before a later async-proxy (TMA) write.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Streaming loads of read-once data (the BVSS tiles): no L1 allocation, L2
// eviction policy from createpolicy (evict-first), so that the reused working
// set (visited bitmap in L1; levels, bitmaps and queues in L2) stays resident.
__device__ __forceinline__ int4 ld_stream_v4(const int4* p, uint64_t pol) {
    int4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t* p, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// 1-D bulk copy global -> shared (TMA), completing `bytes` on the mbarrier.
// src, dst and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar), "l"(pol)
        : "memory");
}

__device__ __forceinline__ void raise_error(Ctrl* ctrl, unsigned int code) {
    atomicCAS(&ctrl->error, 0u, code);
}

__device__ __forceinline__ unsigned int warp_inclusive_scan(unsigned int v, int lane) {
#pragma unroll
    for (int d = 1; d < kWarp; d <<= 1) {
        unsigned int t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

// Every block folds the traversal's status into the sticky word (byte 192),
// which the host reads at synchronisation; the first failure wins.
__device__ __forceinline__ void fold_status(Ctrl* ctrl) {
    if (threadIdx.x == 0) {
        const unsigned int e = ld_volatile_u32(&ctrl->error);
        if (e) atomicCAS(reinterpret_cast<unsigned int*>(ctrl) + kStickyWord, 0u, e);
    }
}

// Queue entry i of a slot: the VSS id st + i with the payload in the upper 32
// bits, or, for the compact layout (GROUPS), the VSS that starts at group
// st + 32 i of a slice set covering tot groups, with its group count - 1 in
// bits 40..44 (payload = the 8-bit alpha in bits 32..39).
template <bool GROUPS>
__device__ __forceinline__ unsigned long long queue_entry(int st, uint32_t pay, int tot, int i) {
    if (!GROUPS) return (unsigned long long)(unsigned int)(st + i) | ((unsigned long long)pay << 32);
    const int left = tot - 32 * i;
    const unsigned int ng = (unsigned int)(left < 32 ? left : 32) - 1u;
    return (unsigned long long)(unsigned int)(st + 32 * i) | ((unsigned long long)pay << 32) |
           ((unsigned long long)ng << 40);
}

// Writes lane i's entries of up to NS slots (a slice set's VSS range, see
// queue_entry) at Qout[pos ...), pos = the lane's first position.  Short runs
// are written by their lane; runs longer than 16 entries (hub slice sets) by
// the whole warp together, since a lane-serial loop would make the warp wait
// for its busiest lane.  Every lane of the warp must call it.
template <int NS, bool GROUPS>
__device__ __forceinline__ void warp_write_entries(unsigned long long* Qout, unsigned int pos, unsigned int cnt,
                                                   const int (&st)[NS], const int (&ln)[NS],
                                                   const uint32_t (&pay)[NS], const int (&tot)[NS], int lane) {
    const bool big = cnt > 16;
    if (!big) {
#pragma unroll
        for (int q = 0; q < NS; ++q)
            for (int i = 0; i < ln[q]; ++i) Qout[pos++] = queue_entry<GROUPS>(st[q], pay[q], tot[q], i);
    }
    unsigned int bigmask = __ballot_sync(0xffffffffu, big);
    while (bigmask) {
        const int src = __ffs(bigmask) - 1;
        bigmask &= bigmask - 1;
        unsigned int p = __shfl_sync(0xffffffffu, pos, src);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int s0 = __shfl_sync(0xffffffffu, st[q], src);
            const int l0 = __shfl_sync(0xffffffffu, ln[q], src);
            const uint32_t p0 = __shfl_sync(0xffffffffu, pay[q], src);
            const int t0 = GROUPS ? __shfl_sync(0xffffffffu, tot[q], src) : 0;
            for (int i = lane; i < l0; i += kWarp) Qout[p + i] = queue_entry<GROUPS>(s0, p0, t0, i);
            p += (unsigned int)l0;
        }
    }
}

// Warp-aggregated queue append (Section 4.2): one atomicAdd on the queue size
// per warp, then warp_write_entries.  Raises BLEST_ERR_INTERNAL (7) instead of
// writing past qcap.
template <int NS, bool GROUPS = false>
__device__ __forceinline__ void warp_enqueue(unsigned int qcap, Ctrl* ctrl, unsigned long long* Qout,
                                             unsigned long long* qcount, const int (&st)[NS], const int (&ln)[NS],
                                             const uint32_t (&pay)[NS], int lane, const int (&tot)[NS]) {
    unsigned int cnt = 0;
#pragma unroll
    for (int q = 0; q < NS; ++q) cnt += (unsigned int)ln[q];
    const unsigned int incl = warp_inclusive_scan(cnt, lane);
    const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    unsigned int base = 0;
    if (lane == 31) base = (unsigned int)atomicAdd(qcount, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    if (base + total > qcap || base + total < base) {
        if (lane == 0) raise_error(ctrl, 7u);
        return;
    }
    warp_write_entries<NS, GROUPS>(Qout, base + incl - cnt, cnt, st, ln, pay, tot, lane);
}

// Warp-coalesced queue append for one range per lane: lane i appends the VSS
// range [st, st + ln) with payload pay.  One atomicAdd per warp reserves the
// warp's total; then entry j of the warp's output (j = lane, lane + 32, ...) is
// written by lane j mod 32, which finds the lane owning j by a binary search
// over the warp's exclusive prefix of ln (5 shuffle steps), so every store
// instruction writes 32 consecutive entries (256 contiguous bytes).
__device__ __forceinline__ void warp_enqueue_coalesced(unsigned int qcap, Ctrl* ctrl, unsigned long long* Qout,
                                                       unsigned long long* qcount, int st, int ln, uint32_t pay,
                                                       int lane) {
    const unsigned int incl = warp_inclusive_scan((unsigned int)ln, lane);
    const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    unsigned int base = 0;
    if (lane == 31) base = (unsigned int)atomicAdd(qcount, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    if (base + total > qcap || base + total < base) {
        if (lane == 0) raise_error(ctrl, 7u);
        return;
    }
    const unsigned int excl = incl - (unsigned int)ln;
    for (unsigned int j0 = 0; j0 < total; j0 += kWarp) {
        const unsigned int j = j0 + (unsigned int)lane;
        // owner = largest lane L with excl(L) <= j (lanes with ln = 0 share their
        // successor's excl and are skipped because the search takes the largest)
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const unsigned int e = __shfl_sync(0xffffffffu, excl, lo + step);
            if (e <= j) lo += step;
        }
        const unsigned int e_own = __shfl_sync(0xffffffffu, excl, lo);
        const int s_own = __shfl_sync(0xffffffffu, st, lo);
        const uint32_t p_own = __shfl_sync(0xffffffffu, pay, lo);
        if (j < total)
            Qout[base + j] = (unsigned long long)(unsigned int)(s_own + (int)(j - e_own)) |
                             ((unsigned long long)p_own << 32);
    }
}

}  // namespace blest
