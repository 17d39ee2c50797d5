// Distance statistics of multi-source traversals, the applications the paper
// names for its multi-source form (Section 6: closeness centrality and graph
// diameter).  For every source row of a k x n level array (-1 = unreached):
// the number of reached vertices, the sum of their levels and the largest
// level.  Closeness (reached - 1) / sum and the diameter bound max over
// sources of the largest level follow on the host.  The statistics do not
// depend on the vertex order, so any row layout of the levels works.
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"

namespace blest {

namespace {

constexpr int kStatsThreads = 256;

// Block (x, y) reduces chunk x of row y; one atomic per statistic per block.
__global__ void __launch_bounds__(kStatsThreads) distance_stats_kernel(const int32_t* __restrict__ lv, int64_t n,
                                                                      int64_t chunk,
                                                                      unsigned long long* __restrict__ reached,
                                                                      unsigned long long* __restrict__ sum,
                                                                      int* __restrict__ ecc) {
    const int64_t row = blockIdx.y;
    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    const int32_t* r = lv + row * n;
    unsigned long long c = 0, s = 0;
    int m = -1;
    for (int64_t v = lo + threadIdx.x; v < hi; v += kStatsThreads) {
        const int x = __ldcs(&r[v]);   // read once
        if (x >= 0) {
            c += 1;
            s += (unsigned long long)x;
            m = x > m ? x : m;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, d);
        s += __shfl_xor_sync(0xffffffffu, s, d);
        const int o = __shfl_xor_sync(0xffffffffu, m, d);
        m = o > m ? o : m;
    }
    __shared__ unsigned long long sc[kStatsThreads / kWarp], ss[kStatsThreads / kWarp];
    __shared__ int sm[kStatsThreads / kWarp];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sc[w] = c; ss[w] = s; sm[w] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kStatsThreads / kWarp; ++i) {
            c += sc[i];
            s += ss[i];
            m = sm[i] > m ? sm[i] : m;
        }
        if (c) {
            atomicAdd(&reached[row], c);
            atomicAdd(&sum[row], s);
            atomicMax(&ecc[row], m);
        }
    }
}

}  // namespace

// lv: k rows of n int32 levels (device).  acc: 2k u64 (reached, sum) + k int
// (ecc), cleared here.  Asynchronous on st.
cudaError_t launch_distance_stats(const int32_t* lv, int32_t k, int64_t n, unsigned long long* acc, int* ecc,
                                  cudaStream_t st) {
    if (k <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 2 * (size_t)k, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ecc, 0xFF, sizeof(int) * (size_t)k, st);   // -1
    if (e != cudaSuccess || n == 0) return e;
    // about 600 blocks in total, chunks of whole 256-thread sweeps
    int64_t chunks = (600 + k - 1) / k;
    int64_t chunk = (n + chunks - 1) / chunks;
    chunk = (chunk + kStatsThreads - 1) / kStatsThreads * kStatsThreads;
    chunks = (n + chunk - 1) / chunk;
    distance_stats_kernel<<<dim3((unsigned)chunks, (unsigned)k), kStatsThreads, 0, st>>>(lv, n, chunk, acc, acc + k,
                                                                                         ecc);
    return cudaGetLastError();
}

}  // namespace blest
