// Host-side launch descriptions of the traversal kernels (no device code here).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace blest {

constexpr int kInlineRoots = 16;

// One fused single-frontier traversal (bfs_kernel.cu).
struct BfsLaunch {
    int update = 2;            // 1 eager, 2 lazy
    int pull = 0;              // 0 CUDA cores, 1 b1 MMA
    int unroll = 2;            // 1, 2
    int minb = 2;              // __launch_bounds__ minimum blocks per SM: 2 or 3
    int filter = 1;            // 1: skip marks of rows already in V_curr; 2: also V_next (lazy)
    int direct = 0;            // 1: sweeps write levels to out through old_of, no unpermute (lazy)
    const int32_t* old_of = nullptr;   // BVSS id -> original id (direct)
    int sched = 0;             // double-buffered stage 1: 0 static round-robin, 1 dynamic (guided)
    int depth = 0;             // lazy stage 1 prefetch: 0 none, 2/3 register pipeline, 4/8 TMA ring stages
    int layout = 0;            // 0: tau-padded VSSs (Section 3.1.2); 1: compact groups (lazy, depth 0 or 2)
    int grid = 0;              // blocks (co-resident)
    int32_t n = 0;
    unsigned int qcap = 0;     // entries per queue buffer
    const int32_t* real_ptrs = nullptr;
    const int32_t* row_ids = nullptr;
    const uint32_t* masks = nullptr;
    const int32_t* goff = nullptr;      // compact layout arrays (layout 1)
    const int32_t* rows_c = nullptr;
    const uint32_t* masks_c = nullptr;
    const int32_t* new_id = nullptr;
    int32_t* levels_internal = nullptr;
    uint32_t* vcur = nullptr;           // ceil(n/32) words: V_curr
    uint32_t* vnext = nullptr;          // ceil(n/32) words: V_next (always contains V_curr)
    uint32_t* dirty = nullptr;          // ceil(nwords / 32) words, zero before launch (NULL: no sparse levels)
    uint32_t* F[3] = {nullptr, nullptr, nullptr};
    unsigned long long* Q[3] = {nullptr, nullptr, nullptr};
    void* ctrl = nullptr;      // 256-byte control block (device_common.cuh)
    int32_t* level_sizes = nullptr;
    unsigned long long* level_times = nullptr;   // 2 * level_cap + 2 entries
    unsigned long long* arrive_first = nullptr;  // 2 level_cap entries each: stage 1, then sweep
    unsigned long long* arrive_last = nullptr;
    int32_t level_cap = 0;
    const int32_t* roots_device = nullptr;
    int32_t roots_host[kInlineRoots] = {0};
    int32_t nroots = 0;
    int32_t* out = nullptr;
    uint64_t timeout_ns = 2000000000ull;
    unsigned int phantom = 0;
};

int bfs_max_blocks_per_sm(int update, int pull, int unroll, int minb, int depth, int layout);

// Steps of the sharded single-source traversal (bfs_kernel.cu): mark the root,
// pull this rank's queue, copy the rank's V_next words out, copy the merged
// words in, and the finalisation sweep (which enqueues the rank's own slice sets).
enum ShardStep { kShardRoot = 0, kShardPull = 1, kShardWordsOut = 2, kShardWordsIn = 3, kShardSweep = 4 };
cudaError_t launch_shard_step(const BfsLaunch& L, int step, int lvl, int world, int rank, int32_t root,
                              uint32_t* words, cudaStream_t stream);
// dst[i] = OR over j < count of src[j * words + i].
cudaError_t launch_or_words(uint32_t* dst, const uint32_t* src, int64_t words, int count, cudaStream_t stream);
int bfs_threads_per_block();
cudaError_t launch_bfs_kernel(const BfsLaunch& L, cudaStream_t stream);

// Device BVSS arrays (bvss_build.cu).
struct DeviceBvss {
    int32_t n = 0;
    int32_t nss = 0;
    int64_t nvss = 0;
    int64_t unpadded = 0;
    int32_t* real_ptrs = nullptr;   // nss + 1
    int32_t* v2r = nullptr;         // nvss
    int32_t* row_ids = nullptr;     // 128 * nvss
    uint32_t* masks = nullptr;      // 32 * nvss
    int32_t* vss_count = nullptr;   // nvss
};

// Compact BVSS layout, derived from the tau-padded one: slice k of slice set s
// (in row order) is sub-slot k % 4 of group goff[s] + k / 4; only the last
// group of a slice set is padded (row id of its last slice, mask 0).  A VSS is
// up to 32 consecutive groups of one slice set, so every slice set has the same
// number of VSSs as in the padded layout.
struct DeviceCompact {
    int64_t groups = 0;
    int32_t* goff = nullptr;        // nss + 1 (goff[nss] = groups)
    int32_t* rows = nullptr;        // 4 * groups
    uint32_t* masks = nullptr;      // groups
};
int build_compact_device(const DeviceBvss& b, cudaStream_t st, DeviceCompact& out, const char** err);
void free_compact_device(DeviceCompact& c);

// Builds the BVSS of the (sorted, symmetric) device CSR.  Allocates the arrays
// of `out` with cudaMalloc.  Returns a blest_status code; err gets a message.
int build_bvss_device(const int32_t* d_rp, const int32_t* d_ci, int32_t n, int64_t nnz, cudaStream_t st,
                      DeviceBvss& out, const char** err);
void free_bvss_device(DeviceBvss& b);
// Update divergence of the BVSS (mean over VSSs of the mean column std-dev).
int update_divergence_device(const DeviceBvss& b, cudaStream_t st, double* out, const char** err);

// Tile-level pull used by blest_debug_pull.
cudaError_t launch_debug_pull(const uint32_t* d_masks, const uint8_t* d_alpha, int32_t tiles, int pull,
                              uint8_t* d_hits, cudaStream_t st);

}  // namespace blest
