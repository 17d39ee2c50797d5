// Host-side description of the multi-source traversal (msbfs_kernel.cu).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "msbfs_bits.h"

namespace blest {

constexpr int kMsbfsChunk = 256;   // most sources per launch (the default launch size)

// 64-bit words per vertex of each bit matrix for a launch of k sources, with
// launches of at most `chunk` sources (64, 128 or 256).
inline int msbfs_words(int64_t k, int chunk = kMsbfsChunk) {
    const int64_t kc = std::min<int64_t>(k, chunk);
    return kc <= 64 ? 1 : (kc <= 128 ? 2 : 4);
}

// int32 entries of the vertex-major level buffer for k sources: n rows of the
// largest launch's source count rounded up to a multiple of 8.
inline int64_t msbfs_level_entries(int32_t n, int64_t k, int chunk = kMsbfsChunk) {
    const int64_t kc = std::min<int64_t>(k, chunk);
    return ((kc + 7) & ~int64_t(7)) * (int64_t)n;
}

// 64-bit words of the level bit planes for k sources: msbfs_planes(n) planes of
// n vertices x W words (plane p holds bit p of every (vertex, source) level).
inline int64_t msbfs_plane_words(int32_t n, int64_t k, int chunk = kMsbfsChunk) {
    return (int64_t)msbfs_planes(n) * (int64_t)n * msbfs_words(k, chunk);
}

// Device buffers of a multi-source traversal, grown on demand and kept with
// the handle between calls.  A state whose buffers the caller allocated
// (caller_owned) is never reallocated: a launch it is too small for fails.
struct MsbfsState {
    bool caller_owned = false;
    int64_t words_cap = 0;             // u64 words per bitmap (n * W)
    unsigned long long* vcur = nullptr;
    unsigned long long* vnext = nullptr;
    unsigned long long* front = nullptr;
    int64_t qcap = 0;
    unsigned long long* Q = nullptr;   // 3 * qcap
    int64_t lint_cap = 0;              // int32 entries of the vertex-major level buffer
    int32_t* lint = nullptr;
    int64_t planes_cap = 0;            // u64 words of the level bit planes
    unsigned long long* planes = nullptr;
    int64_t roots_cap = 0;
    int32_t* roots = nullptr;
    int64_t dirty_cap = 0;             // words of the dirty-slice-set bitmap
    uint32_t* dirty = nullptr;
};

struct MsbfsLaunchCommon {
    int32_t n = 0, nss = 0;
    int64_t nvss = 0;
    const int32_t* real_ptrs = nullptr;
    const int32_t* row_ids = nullptr;
    const uint32_t* masks = nullptr;
    const int32_t* new_id = nullptr;    // NULL = identity
    unsigned int* ctrl = nullptr;       // 64-byte control block + sticky word at [16]
    int sms = 0;
    int blocks_per_sm = 0;
    uint64_t timeout_ns = 2000000000ull;
    unsigned int phantom = 0;
    int32_t* level_sizes = nullptr;
    int32_t level_cap = 0;
    int pull = 0;                       // 0 CUDA-core OR of frontier words, 1 b1 tensor-core MMAs
    int chunk = kMsbfsChunk;            // sources per launch: 64, 128 or 256
    int levels_layout = 0;              // 0 vertex-major levels, 1 bit planes
    int visited_filter = 2;             // 1: test V_curr before each mark, 2: V_next, 0: mark every hit word
};

// Runs k = roots.size() traversals (sources already in BVSS ids) in launches of
// at most c.chunk sources, writing out[i*n + v] in original ids.  Returns a
// blest_status code (device-side status is folded into the sticky word).
int run_msbfs(MsbfsState& s, const MsbfsLaunchCommon& c, const std::vector<int32_t>& roots, int32_t* d_out,
              cudaStream_t st, const char** err);
void free_msbfs_state(MsbfsState& s);

}  // namespace blest
