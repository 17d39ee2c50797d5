// BFS-tree (parent array) output, the other result form of Section 2: after a
// traversal, parent[v] is the smallest original id among the neighbours of v
// that are one level closer to the sources (so the tree is unique); a source
// is its own parent and an unreached vertex has parent -1.
//
// One pass over the BVSS: a warp per virtual slice set (slice set s from
// virtualToReal) loads the levels of the 8 columns of s once; each lane, for
// each of its 4 slices (u, mask) with level[u] >= 1, offers every column c of
// the mask with level[c] = level[u] - 1 to u through an atomicMin on u's
// candidate (in original ids).  A second kernel maps the result back to
// original ids.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "device_common.cuh"

namespace blest {

namespace {

__global__ void parents_kernel(const int32_t* __restrict__ v2r, const int4* __restrict__ rows4,
                               const uint32_t* __restrict__ masks, int64_t nvss, const int32_t* __restrict__ L,
                               const int32_t* __restrict__ old_of, int32_t n, int32_t* __restrict__ cand) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t nu = w; nu < nvss; nu += nw) {
        const int s = __ldg(&v2r[nu]);
        // levels of the slice set's columns, one per lane 0..7
        int lc = -1;
        if (lane < 8 && 8 * s + lane < n) lc = __ldg(&L[8 * s + lane]);
        int lcol[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) lcol[j] = __shfl_sync(0xffffffffu, lc, j);
        const int4 r = __ldg(&rows4[nu * kWarp + lane]);
        const uint32_t m = __ldg(&masks[nu * kWarp + lane]);
        const int r4[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t mq = (m >> (8 * q)) & 0xFFu;
            if (!mq) continue;
            const int u = r4[q];
            const int lu = __ldg(&L[u]);
            if (lu < 1) continue;
            int best = INT_MAX;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (!((mq >> j) & 1u) || lcol[j] != lu - 1) continue;
                const int c = 8 * s + j;
                const int oc = old_of ? __ldg(&old_of[c]) : c;
                best = oc < best ? oc : best;
            }
            if (best != INT_MAX) atomicMin(&cand[u], best);
        }
    }
}

// out[v] (original ids): v for a source, cand[new_id[v]] for a reached vertex, -1 otherwise.
__global__ void parents_unpermute_kernel(const int32_t* __restrict__ L, const int32_t* __restrict__ cand,
                                         const int32_t* __restrict__ new_id, int32_t n, int32_t* __restrict__ out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int u = new_id ? __ldg(&new_id[v]) : (int)v;
        const int lu = __ldg(&L[u]);
        out[v] = lu < 0 ? -1 : (lu == 0 ? (int)v : __ldg(&cand[u]));
    }
}

__global__ void fill_kernel(int32_t* p, int32_t n, int32_t value) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = value;
}

int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65536) g = 65536;
    return (int)g;
}

}  // namespace

// L: internal levels (BVSS ids) of a finished traversal; cand: n int32 scratch;
// old_of: BVSS id -> original id (NULL = identity); new_id: original -> BVSS.
cudaError_t launch_parents(const int32_t* v2r, const int32_t* row_ids, const uint32_t* masks, int64_t nvss,
                           const int32_t* L, const int32_t* old_of, const int32_t* new_id, int32_t n, int32_t* cand,
                           int32_t* out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    fill_kernel<<<grid_for(n, 256), 256, 0, st>>>(cand, n, INT_MAX);
    if (nvss > 0)
        parents_kernel<<<grid_for(nvss * kWarp, 256), 256, 0, st>>>(v2r, reinterpret_cast<const int4*>(row_ids), masks,
                                                                    nvss, L, old_of, n, cand);
    parents_unpermute_kernel<<<grid_for(n, 256), 256, 0, st>>>(L, cand, new_id, n, out);
    return cudaGetLastError();
}

}  // namespace blest
