// Device construction of the BVSS arrays (Section 3.1) from a symmetric CSR
// whose rows are sorted.  A is the adjacency of the transposed graph, so the
// nonzeros of column c of A are CSR row c; slice set s gathers columns
// [8s, 8s+8), which are the contiguous CSR entries rp[8s] .. rp[8s+8).
//
//  1. rank:    each entry (row u from column list j of slice set s) computes its
//              position in the (u, j)-sorted merge of the 8 sorted lists with 7
//              binary searches, and scatters key (u << 3 | j) there;
//  2. heads:   a merged entry starts a slice when its row differs from its
//              predecessor's (or it opens a slice set);
//  3. scan:    exclusive scan of the head flags numbers the slices;
//  4. count:   slices per slice set -> VSSs per slice set = ceil(count / 128);
//              exclusive scan -> realPtrs;
//  5. place:   slice k of slice set s goes to VSS realPtrs[s] + k / 128, lane
//              (k mod 128) mod 32, sub-slot (k mod 128) / 32 (Section 3.1.2);
//              its mask is the OR of the bits j of the entries of its row;
//  6. finish:  virtualToReal, per-VSS slice counts, and padding of the last VSS
//              of every slice set: zero masks and the row id of its last real
//              slice (the text asks for dummy ids; any in-range value is inert).
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "bfs_launch.h"
#include "device_common.cuh"

namespace blest {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* smem, int64_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += t;
    }
    if (lane == 31) smem[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t y = lane < (int)(blockDim.x >> 5) ? smem[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, y, d);
            if (lane >= d) y += t;
        }
        smem[lane] = y;   // inclusive over warps
    }
    __syncthreads();
    const int64_t warp_off = wid > 0 ? smem[wid - 1] : 0;
    *total = smem[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_off + x - v;
}

template <class T>
__global__ void scan_reduce_kernel(const T* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
    __shared__ int64_t smem[32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += (int64_t)in[base + i];
    int64_t total;
    block_exclusive_scan(s, smem, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void scan_sums_kernel(int64_t* sums, int64_t nb) {
    __shared__ int64_t smem[32];
    int64_t carry = 0;
    for (int64_t off = 0; off < nb; off += blockDim.x) {
        const int64_t i = off + threadIdx.x;
        const int64_t v = i < nb ? sums[i] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, smem, &total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
        __syncthreads();
    }
}

template <class T, class U>
__global__ void scan_apply_kernel(const T* __restrict__ in, int64_t n, const int64_t* __restrict__ sums,
                                  U* __restrict__ out, int64_t grand_total_index) {
    __shared__ int64_t smem[32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int64_t vals[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        vals[i] = base + i < n ? (int64_t)in[base + i] : 0;
        s += vals[i];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(s, smem, &total) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = (U)run;
        run += vals[i];
    }
    // the last element of the whole input also writes the grand total at out[n]
    if (grand_total_index >= 0 && base <= n - 1 && n - 1 < base + kScanItems) out[n] = (U)run;
}

// out[0..n] = exclusive scan of in[0..n), out[n] = total.  tmp >= ceil(n / chunk) int64.
template <class T, class U>
cudaError_t exclusive_scan(const T* in, int64_t n, U* out, int64_t* tmp, cudaStream_t st) {
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(U), st);
    const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    scan_reduce_kernel<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, tmp);
    scan_sums_kernel<<<1, 1024, 0, st>>>(tmp, nb);
    scan_apply_kernel<T, U><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, tmp, out, n);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- build steps

__device__ __forceinline__ int64_t upper_bound_i32(const int32_t* a, int64_t lo, int64_t hi, int64_t x) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)__ldg(&a[mid]) <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* a, int64_t lo, int64_t hi, int64_t x) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)__ldg(&a[mid]) < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void rank_scatter_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t n,
                                    int64_t nnz, uint32_t* __restrict__ merged, int32_t* __restrict__ ss_of) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = upper_bound_i32(rp, 0, (int64_t)n + 1, e) - 1;   // rp[c] <= e < rp[c+1]
        const int32_t s = (int32_t)(c >> 3);
        const int j = (int)(c & 7);
        const int64_t u = __ldg(&ci[e]);
        int64_t b[9];
#pragma unroll
        for (int q = 0; q <= 8; ++q) {
            const int64_t col = (int64_t)s * 8 + q;
            b[q] = __ldg(&rp[col < n ? col : n]);
        }
        int64_t rank = e - b[j];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q == j || b[q] == b[q + 1]) continue;
            rank += (q < j ? upper_bound_i32(ci, b[q], b[q + 1], u) : lower_bound_i32(ci, b[q], b[q + 1], u)) - b[q];
        }
        merged[b[0] + rank] = ((uint32_t)u << 3) | (uint32_t)j;
        ss_of[e] = s;
    }
}

__global__ void head_kernel(const uint32_t* __restrict__ merged, const int32_t* __restrict__ ss_of, int64_t nnz,
                            uint32_t* __restrict__ head) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = 1;
        if (i > 0 && ss_of[i] == ss_of[i - 1] && (merged[i] >> 3) == (merged[i - 1] >> 3)) h = 0;
        head[i] = h;
    }
}

__global__ void count_kernel(const int32_t* __restrict__ rp, int32_t n, int32_t nss, const int32_t* __restrict__ slice_idx,
                             int32_t* __restrict__ cnt, int32_t* __restrict__ first_slice, int32_t* __restrict__ nvss) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nss; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c0 = s * 8, c1 = c0 + 8 < n ? c0 + 8 : n;
        const int64_t e0 = rp[c0], e1 = rp[c1];
        const int32_t k = slice_idx[e1] - slice_idx[e0];
        cnt[s] = k;
        first_slice[s] = slice_idx[e0];
        nvss[s] = (k + 127) / 128;
    }
}

__global__ void place_kernel(const uint32_t* __restrict__ merged, const int32_t* __restrict__ ss_of,
                             const uint32_t* __restrict__ head, const int32_t* __restrict__ slice_idx, int64_t nnz,
                             const int32_t* __restrict__ first_slice, const int32_t* __restrict__ real_ptrs,
                             int32_t* __restrict__ row_ids, uint8_t* __restrict__ mask_bytes) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x) {
        if (!head[i]) continue;
        const int32_t s = ss_of[i];
        const uint32_t u = merged[i] >> 3;
        uint32_t m = 0;
        for (int64_t k = i; k < nnz && ss_of[k] == s && (merged[k] >> 3) == u; ++k) m |= 1u << (merged[k] & 7u);
        const int64_t k = (int64_t)slice_idx[i] - first_slice[s];
        const int64_t nu = (int64_t)real_ptrs[s] + k / 128;
        const int kk = (int)(k % 128), lane = kk & 31, sub = kk >> 5;
        row_ids[nu * 128 + lane * 4 + sub] = (int32_t)u;
        mask_bytes[(nu * 32 + lane) * 4 + sub] = (uint8_t)m;
    }
}

__global__ void finish_kernel(const int32_t* __restrict__ real_ptrs, int32_t nss, const int32_t* __restrict__ cnt,
                              int64_t nvss, int32_t* __restrict__ v2r, int32_t* __restrict__ vss_count,
                              int32_t* __restrict__ row_ids) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t nu = w; nu < nvss; nu += nw) {
        const int64_t s = upper_bound_i32(real_ptrs, 0, (int64_t)nss + 1, nu) - 1;
        const int64_t within = nu - real_ptrs[s];
        const int64_t rest = (int64_t)cnt[s] - within * 128;
        const int c = (int)(rest < 128 ? rest : 128);
        if (lane == 0) { v2r[nu] = (int32_t)s; vss_count[nu] = c; }
        if (c < 128) {
            const int last = c - 1;
            const int32_t pad = row_ids[nu * 128 + (last & 31) * 4 + (last >> 5)];
            for (int k = c + lane; k < 128; k += 32) row_ids[nu * 128 + (k & 31) * 4 + (k >> 5)] = pad;
        }
    }
}

__global__ void udiv_kernel(const int32_t* __restrict__ row_ids, const int32_t* __restrict__ vss_count, int64_t nvss,
                            double* __restrict__ per_vss) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t nu = w; nu < nvss; nu += nw) {
        const int c = vss_count[nu];
        double acc = 0.0;
        int cols = 0;
        for (int q = 0; q < 4; ++q) {
            const int cq = c - 32 * q < 0 ? 0 : (c - 32 * q > 32 ? 32 : c - 32 * q);
            if (cq == 0) break;
            const bool live = lane < cq;
            const double u = live ? (double)row_ids[nu * 128 + lane * 4 + q] : 0.0;
            double s = u;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
            const double mean = s / cq;
            double v = live ? (u - mean) * (u - mean) : 0.0;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            acc += sqrt(v / cq);
            ++cols;
        }
        if (lane == 0) per_vss[nu] = cols ? acc / cols : 0.0;
    }
}

// ------------------------------------------------------------ compact layout

// Groups of slice set s: ceil(c_s / 4), c_s = 128 (VSSs - 1) + slices of its last VSS.
__global__ void compact_count_kernel(const int32_t* __restrict__ real_ptrs, const int32_t* __restrict__ vss_count,
                                     int32_t nss, int32_t* __restrict__ groups) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nss; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v0 = real_ptrs[s], v1 = real_ptrs[s + 1];
        const int64_t c = v1 > v0 ? 128ll * (v1 - v0 - 1) + vss_count[v1 - 1] : 0;
        groups[s] = (int32_t)((c + 3) / 4);
    }
}

// A warp per padded VSS nu (slice set s, i-th of s): its slice k (lane k % 32,
// sub-slot k / 32) is slice 128 i + k of s, stored at group goff[s] + 32 i + k / 4,
// sub-slot k % 4.  The lane holding the last slice of s pads the rest of its group.
__global__ void compact_place_kernel(const int32_t* __restrict__ real_ptrs, const int32_t* __restrict__ v2r,
                                     const int32_t* __restrict__ row_ids, const uint32_t* __restrict__ masks,
                                     const int32_t* __restrict__ vss_count, int64_t nvss,
                                     const int32_t* __restrict__ goff, int32_t* __restrict__ rows_c,
                                     uint8_t* __restrict__ mask_bytes_c) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t nu = w; nu < nvss; nu += nw) {
        const int32_t s = v2r[nu];
        const int64_t i = nu - real_ptrs[s];
        const int c = vss_count[nu];
        const bool last_vss = nu + 1 == real_ptrs[s + 1];
        const uint32_t m = masks[nu * 32 + lane];
        for (int q = 0; q < 4; ++q) {
            const int k = 32 * q + lane;
            if (k >= c) break;
            const int64_t kk = 128 * i + k;                       // slice index within s
            const int64_t slot = 4 * (int64_t)goff[s] + kk;       // group * 4 + sub-slot
            const int32_t row = row_ids[nu * 128 + lane * 4 + q];
            rows_c[slot] = row;
            mask_bytes_c[slot] = (uint8_t)((m >> (8 * q)) & 0xFFu);
            if (last_vss && k == c - 1)
                for (int64_t p = slot + 1; (p & 3) != 0; ++p) rows_c[p] = row;   // masks were zeroed
        }
    }
}

int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65536) g = 65536;
    return (int)g;
}

}  // namespace

#define BLEST_CK(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) { *err = cudaGetErrorString(e_); rc = e_ == cudaErrorMemoryAllocation ? 4 : 5; goto done; } \
    } while (0)

int build_bvss_device(const int32_t* d_rp, const int32_t* d_ci, int32_t n, int64_t nnz, cudaStream_t st,
                      DeviceBvss& out, const char** err) {
    int rc = 0;
    const int32_t nss = (n + 7) / 8;
    uint32_t* merged = nullptr;
    int32_t* ss_of = nullptr;
    uint32_t* head = nullptr;
    int32_t* slice_idx = nullptr;
    int32_t *cnt = nullptr, *first = nullptr, *nvss_s = nullptr;
    int64_t* tmp = nullptr;
    int32_t total_vss = 0;
    const int64_t nb = (std::max<int64_t>(nnz, nss) + kScanChunk - 1) / kScanChunk + 1;
    out.n = n;
    out.nss = nss;
    BLEST_CK(cudaMalloc(&out.real_ptrs, sizeof(int32_t) * ((size_t)nss + 1)));
    BLEST_CK(cudaMalloc(&merged, sizeof(uint32_t) * (size_t)std::max<int64_t>(nnz, 1)));
    BLEST_CK(cudaMalloc(&ss_of, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1)));
    BLEST_CK(cudaMalloc(&head, sizeof(uint32_t) * (size_t)std::max<int64_t>(nnz, 1)));
    BLEST_CK(cudaMalloc(&slice_idx, sizeof(int32_t) * ((size_t)nnz + 1)));
    BLEST_CK(cudaMalloc(&cnt, sizeof(int32_t) * (size_t)std::max(nss, 1)));
    BLEST_CK(cudaMalloc(&first, sizeof(int32_t) * (size_t)std::max(nss, 1)));
    BLEST_CK(cudaMalloc(&nvss_s, sizeof(int32_t) * (size_t)std::max(nss, 1)));
    BLEST_CK(cudaMalloc(&tmp, sizeof(int64_t) * (size_t)nb));
    if (nnz > 0) {
        rank_scatter_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(d_rp, d_ci, n, nnz, merged, ss_of);
        head_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(merged, ss_of, nnz, head);
        BLEST_CK(cudaGetLastError());
    }
    BLEST_CK(exclusive_scan(head, nnz, slice_idx, tmp, st));
    if (nss > 0) {
        count_kernel<<<grid_for(nss, 256), 256, 0, st>>>(d_rp, n, nss, slice_idx, cnt, first, nvss_s);
        BLEST_CK(cudaGetLastError());
    }
    BLEST_CK(exclusive_scan(nvss_s, (int64_t)nss, out.real_ptrs, tmp, st));
    BLEST_CK(cudaMemcpyAsync(&total_vss, out.real_ptrs + nss, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BLEST_CK(cudaStreamSynchronize(st));
    {
        int32_t unpadded = 0;
        BLEST_CK(cudaMemcpy(&unpadded, slice_idx + nnz, sizeof(int32_t), cudaMemcpyDeviceToHost));
        out.unpadded = unpadded;
    }
    out.nvss = total_vss;
    BLEST_CK(cudaMalloc(&out.v2r, sizeof(int32_t) * (size_t)std::max<int64_t>(total_vss, 1)));
    BLEST_CK(cudaMalloc(&out.vss_count, sizeof(int32_t) * (size_t)std::max<int64_t>(total_vss, 1)));
    BLEST_CK(cudaMalloc(&out.row_ids, sizeof(int32_t) * 128 * (size_t)std::max<int64_t>(total_vss, 1)));
    BLEST_CK(cudaMalloc(&out.masks, sizeof(uint32_t) * 32 * (size_t)std::max<int64_t>(total_vss, 1)));
    BLEST_CK(cudaMemsetAsync(out.masks, 0, sizeof(uint32_t) * 32 * (size_t)std::max<int64_t>(total_vss, 1), st));
    if (nnz > 0 && total_vss > 0) {
        place_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(merged, ss_of, head, slice_idx, nnz, first, out.real_ptrs,
                                                         out.row_ids, reinterpret_cast<uint8_t*>(out.masks));
        finish_kernel<<<grid_for((int64_t)total_vss * 32, 256), 256, 0, st>>>(out.real_ptrs, nss, cnt, total_vss,
                                                                              out.v2r, out.vss_count, out.row_ids);
        BLEST_CK(cudaGetLastError());
    }
    BLEST_CK(cudaStreamSynchronize(st));
done:
    cudaFree(merged);
    cudaFree(ss_of);
    cudaFree(head);
    cudaFree(slice_idx);
    cudaFree(cnt);
    cudaFree(first);
    cudaFree(nvss_s);
    cudaFree(tmp);
    if (rc != 0) free_bvss_device(out);
    return rc;
}

int build_compact_device(const DeviceBvss& b, cudaStream_t st, DeviceCompact& out, const char** err) {
    int rc = 0;
    int32_t* groups = nullptr;
    int64_t* tmp = nullptr;
    int32_t total = 0;
    const int64_t nb = ((int64_t)b.nss + kScanChunk - 1) / kScanChunk + 1;
    BLEST_CK(cudaMalloc(&out.goff, sizeof(int32_t) * ((size_t)b.nss + 1)));
    BLEST_CK(cudaMalloc(&groups, sizeof(int32_t) * (size_t)std::max(b.nss, 1)));
    BLEST_CK(cudaMalloc(&tmp, sizeof(int64_t) * (size_t)nb));
    if (b.nss > 0) {
        compact_count_kernel<<<grid_for(b.nss, 256), 256, 0, st>>>(b.real_ptrs, b.vss_count, b.nss, groups);
        BLEST_CK(cudaGetLastError());
    }
    BLEST_CK(exclusive_scan(groups, (int64_t)b.nss, out.goff, tmp, st));
    BLEST_CK(cudaMemcpyAsync(&total, out.goff + b.nss, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BLEST_CK(cudaStreamSynchronize(st));
    out.groups = total;
    BLEST_CK(cudaMalloc(&out.rows, sizeof(int32_t) * 4 * (size_t)std::max<int64_t>(total, 1)));
    BLEST_CK(cudaMalloc(&out.masks, sizeof(uint32_t) * (size_t)std::max<int64_t>(total, 1)));
    BLEST_CK(cudaMemsetAsync(out.masks, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(total, 1), st));
    if (b.nvss > 0) {
        compact_place_kernel<<<grid_for(b.nvss * 32, 256), 256, 0, st>>>(
            b.real_ptrs, b.v2r, b.row_ids, b.masks, b.vss_count, b.nvss, out.goff, out.rows,
            reinterpret_cast<uint8_t*>(out.masks));
        BLEST_CK(cudaGetLastError());
    }
    BLEST_CK(cudaStreamSynchronize(st));
done:
    cudaFree(groups);
    cudaFree(tmp);
    if (rc != 0) free_compact_device(out);
    return rc;
}

void free_compact_device(DeviceCompact& c) {
    cudaFree(c.goff);
    cudaFree(c.rows);
    cudaFree(c.masks);
    c.goff = c.rows = nullptr;
    c.masks = nullptr;
    c.groups = 0;
}

void free_bvss_device(DeviceBvss& b) {
    cudaFree(b.real_ptrs);
    cudaFree(b.v2r);
    cudaFree(b.row_ids);
    cudaFree(b.masks);
    cudaFree(b.vss_count);
    b.real_ptrs = b.v2r = b.row_ids = b.vss_count = nullptr;
    b.masks = nullptr;
}

int update_divergence_device(const DeviceBvss& b, cudaStream_t st, double* out, const char** err) {
    int rc = 0;
    double* per = nullptr;
    std::vector<double> h;
    *out = 0.0;
    if (b.nvss == 0) return 0;
    BLEST_CK(cudaMalloc(&per, sizeof(double) * (size_t)b.nvss));
    udiv_kernel<<<grid_for(b.nvss * 32, 256), 256, 0, st>>>(b.row_ids, b.vss_count, b.nvss, per);
    BLEST_CK(cudaGetLastError());
    h.resize((size_t)b.nvss);
    BLEST_CK(cudaMemcpyAsync(h.data(), per, sizeof(double) * (size_t)b.nvss, cudaMemcpyDeviceToHost, st));
    BLEST_CK(cudaStreamSynchronize(st));
    {
        double s = 0.0;
        for (double v : h) s += v;
        *out = s / (double)b.nvss;
    }
done:
    cudaFree(per);
    return rc;
}

}  // namespace blest
