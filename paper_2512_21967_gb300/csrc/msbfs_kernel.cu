// Multi-source BFS as a Boolean SpMM over BVSS (Section 2: k frontiers stacked
// column-wise form an n x k frontier matrix).  One persistent cooperative
// launch runs up to 256 sources; each vertex carries W = ceil(k / 64) 64-bit
// words of frontier and of visited bits.  Per level:
//   stage 1: warps take queued virtual slice sets round-robin.  The 8 x k
//     frontier tile of the slice set (8 W words) is loaded once per VSS by 8 W
//     lanes and broadcast by shuffles; each lane ORs, for each of its 4 slices,
//     the k-bit words of the columns its mask selects -- y_u |= OR_{j in mask}
//     X[8s + j] -- and marks the result in V_next[u] with returnless 64-bit
//     atomicOrs (the lazy marking of Algorithm 3, k bits at a time).
//   stage 2: a coalesced sweep over vertices: diff = V_next ^ V_curr becomes
//     the next frontier, newly set bits give levels, and the slice sets of
//     vertices with any new bit are enqueued with one atomicAdd per warp.
// The tensor-core form of this product would need the 8-bit masks unpacked to
// an f16/b1 operand per VSS; with K = 8 columns per slice set the work is
// memory-bound, so it stays on the CUDA cores.
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
    int32_t* lint;       // k x n, BVSS ids
    int32_t* out;        // k x n, original ids (== lint when new_id is NULL)
    uint32_t* dirty;     // one bit per slice set touched by a mark in a sparse level (cleared by the sweep)
    const int32_t* roots;
    Ctrl* ctrl;
    int32_t* level_sizes;
    int32_t level_cap;
    uint64_t timeout_ns;
    unsigned int phantom;
};

template <int W>
__device__ __forceinline__ void ms_sweep(const MsArgs& a, int lvl, unsigned long long* Qout, unsigned int* qcount) {
    const int lane = threadIdx.x & 31;
    const size_t n = (size_t)a.n;
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int nchunks = (a.n + kWarp - 1) / kWarp;
    // one row per lane, 32 consecutive rows per warp step (they share bitmap
    // lines); consecutive chunks go to consecutive thread blocks so that the hub
    // rows at the lowest ids, whose slice sets carry most queue entries, are
    // spread over the SMs
    for (int c = (int)blockIdx.x + (int)(threadIdx.x >> 5) * (int)gridDim.x; c < nchunks; c += nwarps) {
        const int u = c * kWarp + lane;
        bool any = false;
        if (u < a.n) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const size_t idx = (size_t)u * W + w;
                const unsigned long long nx = ld_cg(&a.vnext[idx]);
                const unsigned long long cu = ld_cg(&a.vcur[idx]);
                unsigned long long d = nx ^ cu;
                a.front[idx] = d;
                if (d) {
                    a.vcur[idx] = nx;
                    any = true;
                    while (d) {
                        const int b = __ffsll((long long)d) - 1;
                        a.lint[(size_t)(w * 64 + b) * n + (size_t)u] = lvl;
                        d &= d - 1;
                    }
                }
            }
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
template <int W>
__device__ __forceinline__ void ms_sweep_sparse(const MsArgs& a, int lvl, unsigned long long* Qout,
                                                unsigned int* qcount) {
    const int lane = threadIdx.x & 31;
    const int wpb = (int)(blockDim.x >> 5);
    const size_t n = (size_t)a.n;
    const int nss = (a.n + 7) >> 3;
    const int dwords = (nss + 31) >> 5;
    // block-strided over dirty words so that every warp of a block runs the same iterations
    for (int t0 = (int)blockIdx.x * wpb; t0 < dwords; t0 += (int)gridDim.x * wpb) {
        const int t = t0 + (int)(threadIdx.x >> 5);
        const uint32_t dw = t < dwords ? ld_cg(&a.dirty[t]) : 0u;
        if (lane == 0 && dw) a.dirty[t] = 0u;
        const int s = 32 * t + lane;
        bool any = false;
        if ((dw >> lane) & 1u) {
            for (int j = 0; j < 8; ++j) {
                const int u = 8 * s + j;
                if (u >= a.n) break;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const size_t idx = (size_t)u * W + w;
                    const unsigned long long nx = ld_cg(&a.vnext[idx]);
                    const unsigned long long cu = ld_cg(&a.vcur[idx]);
                    unsigned long long d = nx ^ cu;
                    a.front[idx] = d;
                    if (d) {
                        a.vcur[idx] = nx;
                        any = true;
                        while (d) {
                            const int b = __ffsll((long long)d) - 1;
                            a.lint[(size_t)(w * 64 + b) * n + (size_t)u] = lvl;
                            d &= d - 1;
                        }
                    }
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

template <int W>
__device__ __forceinline__ void ms_body(const MsArgs& a) {
    const int lane = threadIdx.x & 31;
    const int gtid = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int nthreads = (int)(gridDim.x * blockDim.x);
    const int gwarp = gtid >> 5;
    const int nwarps = nthreads >> 5;
    unsigned int gen = 0;
    Ctrl* ctrl = a.ctrl;

    for (int i = gtid; i < a.k; i += nthreads) {
        const int r = a.roots[i];
        atomicOr(&a.vnext[(size_t)r * W + (i >> 6)], 1ull << (i & 63));
    }
    if (!grid_barrier(ctrl, gridDim.x, a.phantom, gen, a.timeout_ns)) return;
    ms_sweep<W>(a, 0, a.Q[1], &ctrl->qcount[1]);
    unsigned int qn = 0;
    if (!grid_barrier(ctrl, gridDim.x, a.phantom, gen, a.timeout_ns, &ctrl->qcount[1], &qn)) return;

    int lvl = 1;
    for (;; ++lvl) {
        if (qn > a.qcap) qn = a.qcap;   // only after an overflow, which already raised an error
        // few queued VSSs: track the touched slice sets and sweep only those
        const bool sparse = (unsigned long long)qn * 128ull <= (unsigned long long)a.n;
        if (gtid == 0) {
            ctrl->qcount[(lvl + 2) & 3] = 0;
            if (a.level_sizes && lvl - 1 < a.level_cap) a.level_sizes[lvl - 1] = (int32_t)qn;
        }
        const unsigned long long* Qin = a.Q[lvl % 3];
        unsigned long long* Qout = a.Q[(lvl + 1) % 3];
        unsigned int* qcount_next = &ctrl->qcount[(lvl + 1) & 3];
        for (unsigned int p = (unsigned int)gwarp; p < qn; p += (unsigned int)nwarps) {
            const unsigned long long ent = ld_cg(&Qin[p]);
            const uint32_t nu = (uint32_t)ent;
            const int s = (int)(ent >> 32);
            // 8 x k frontier tile of slice set s: lane j*W + w holds word w of column 8s + j
            unsigned long long fw = 0;
            if (lane < 8 * W) {
                const int col = 8 * s + lane / W;
                if (col < a.n) fw = ld_cg(&a.front[(size_t)col * W + (lane % W)]);
            }
            const unsigned int nzb = __ballot_sync(0xffffffffu, fw != 0ull);
            uint32_t alpha = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if ((nzb >> (j * W)) & ((1u << W) - 1u)) alpha |= 1u << j;
            const size_t tile = (size_t)nu * kWarp + lane;
            const int4 r = __ldg(&a.row_ids4[tile]);
            const uint32_t m = __ldg(&a.masks[tile]) & (alpha * 0x01010101u);
            unsigned long long y[4][W];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int w = 0; w < W; ++w) y[q][w] = 0ull;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (!((alpha >> j) & 1u)) continue;   // warp-uniform
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const unsigned long long v = __shfl_sync(0xffffffffu, fw, j * W + w);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if ((m >> (8 * q + j)) & 1u) y[q][w] |= v;
                }
            }
            const int r4[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    if (!y[q][w]) continue;
                    // sources that already reached the row need no mark; V_curr only gains
                    // bits during a traversal, so a stale word can only let a mark through
                    const unsigned long long fresh = y[q][w] & ~a.vcur[(size_t)r4[q] * W + w];
                    if (fresh) {
                        atomicOr(&a.vnext[(size_t)r4[q] * W + w], fresh);
                        if (sparse) atomicOr(&a.dirty[r4[q] >> 8], 1u << ((r4[q] >> 3) & 31));
                    }
                }
        }
        if (!grid_barrier(ctrl, gridDim.x, a.phantom, gen, a.timeout_ns)) return;
        if (sparse) ms_sweep_sparse<W>(a, lvl, Qout, qcount_next);
        else ms_sweep<W>(a, lvl, Qout, qcount_next);
        unsigned int qnext = 0;
        if (!grid_barrier(ctrl, gridDim.x, a.phantom, gen, a.timeout_ns, qcount_next, &qnext)) return;
        if (qnext == 0) break;
        qn = qnext;
    }
    if (gtid == 0) ctrl->levels = (unsigned int)lvl;
    // out[i*n + v] = level of v from source i (original ids), -1 if unreached
    const int64_t total = (int64_t)a.k * a.n;
    for (int64_t x = gtid; x < total; x += nthreads) {
        const int i = (int)(x / a.n);
        const int v = (int)(x - (int64_t)i * a.n);
        const int u = a.new_id ? __ldg(&a.new_id[v]) : v;
        const bool reached = (ld_cg(&a.vcur[(size_t)u * W + (i >> 6)]) >> (i & 63)) & 1ull;
        a.out[x] = reached ? ld_cg(&a.lint[(size_t)i * a.n + u]) : -1;
    }
}

template <int W>
__global__ void __launch_bounds__(kMsBlock) msbfs_kernel(MsArgs a) {
    ms_body<W>(a);
    fold_status(a.ctrl);
}

template <class T>
cudaError_t grow(T*& p, int64_t& cap, int64_t need, int copies = 1) {
    if (need <= cap) return cudaSuccess;
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
    cudaFree(s.roots);
    cudaFree(s.dirty);
    s = MsbfsState();
}

int run_msbfs(MsbfsState& s, const MsbfsLaunchCommon& c, const std::vector<int32_t>& roots, int32_t* d_out,
              cudaStream_t st, const char** err) {
    const int64_t k_all = (int64_t)roots.size();
    if (k_all == 0 || c.n == 0) return 0;
    cudaError_t e = cudaSuccess;
    for (int64_t i0 = 0; i0 < k_all; i0 += 256) {
        const int k = (int)std::min<int64_t>(256, k_all - i0);
        const int W = k <= 64 ? 1 : (k <= 128 ? 2 : 4);
        const int64_t words = (int64_t)c.n * W;
        int64_t cap_v = s.words_cap, cap_n = s.words_cap, cap_f = s.words_cap;
        if ((e = grow(s.vcur, cap_v, words)) != cudaSuccess) break;
        if ((e = grow(s.vnext, cap_n, words)) != cudaSuccess) break;
        if ((e = grow(s.front, cap_f, words)) != cudaSuccess) break;
        s.words_cap = std::min(cap_v, std::min(cap_n, cap_f));
        if ((e = grow(s.Q, s.qcap, std::max<int64_t>(c.nvss, 1), 3)) != cudaSuccess) break;
        if (c.new_id && (e = grow(s.lint, s.lint_cap, (int64_t)k * c.n)) != cudaSuccess) break;
        if ((e = grow(s.roots, s.roots_cap, k)) != cudaSuccess) break;
        const int64_t dwords = ((int64_t)c.nss + 31) / 32;
        if ((e = grow(s.dirty, s.dirty_cap, dwords)) != cudaSuccess) break;
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
        a.lint = c.new_id ? s.lint : out;
        a.out = out;
        a.roots = s.roots;
        a.dirty = s.dirty;
        a.ctrl = reinterpret_cast<Ctrl*>(c.ctrl);
        a.level_sizes = c.level_sizes;
        a.level_cap = c.level_cap;
        a.timeout_ns = c.timeout_ns;
        a.phantom = c.phantom;
        void* kfn = W == 1 ? (void*)&msbfs_kernel<1> : (W == 2 ? (void*)&msbfs_kernel<2> : (void*)&msbfs_kernel<4>);
        int nb = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, kMsBlock, 0)) != cudaSuccess) break;
        if (nb <= 0) { *err = "msbfs kernel cannot be resident"; return 5; }
        if (c.blocks_per_sm > 0) nb = std::min(nb, c.blocks_per_sm);
        void* args[] = {&a};
        if ((e = cudaLaunchCooperativeKernel(kfn, dim3((unsigned)(nb * c.sms)), dim3(kMsBlock), args, 0, st)) != cudaSuccess) break;
    }
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? 4 : 5;
    }
    return 0;
}

}  // namespace blest
