// Single-source traversal for callers that cannot allocate device memory.
//
// Some callers must never call cudaMalloc: plugins and embedded runtimes whose
// host application owns every device allocation and hands them only the
// buffers they work on, and services whose device memory is budgeted up front
// so that no request can fail or stall on an allocation.  For them,
// blest_bfs_static_scratch runs the same fused traversal kernel as
// blest_bfs_device, but every working buffer it needs -- control block,
// internal levels, visited bitmaps, eager frontier bitmaps and the three VSS
// queues -- lives in the file-scope device array g_scratch below.  Its size is
// fixed at compile time (about 21 MiB) and every GPU that loads this library
// holds it until the process exits.  The caller passes the BVSS arrays and the
// output; nothing here allocates.
//
// Host code must not take the address of g_scratch directly: in host code that
// name is only a host-side stand-in for the device variable.  The device
// address is obtained once per device with cudaGetSymbolAddress, with that
// device current, the first time the entry point runs on it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/blest.h"
#include "bfs_launch.h"

namespace blest {
void set_last_error(const std::string& msg);   // api.cu
}

namespace {

constexpr int32_t kScratchMaxVertices = 1 << 21;          // 2,097,152
constexpr int64_t kScratchMaxVss = 1 << 19;               // 524,288 virtual slice sets
constexpr size_t kWordsMax = kScratchMaxVertices / 32;
constexpr size_t kOffCtrl = 0;
constexpr size_t kOffLevels = 256;
constexpr size_t kOffVcur = kOffLevels + sizeof(int32_t) * kScratchMaxVertices;
constexpr size_t kOffVnext = kOffVcur + sizeof(uint32_t) * kWordsMax;
constexpr size_t kOffF = kOffVnext + sizeof(uint32_t) * kWordsMax;
constexpr size_t kOffQ = kOffF + 3 * sizeof(uint32_t) * kWordsMax;
constexpr size_t kScratchBytes = kOffQ + 3 * sizeof(unsigned long long) * (size_t)kScratchMaxVss;
constexpr int kStickyWord = 48;        // control-block layout of device_common.cuh

static_assert(kOffVcur % 16 == 0 && kOffVnext % 16 == 0 && kOffF % 16 == 0 && kOffQ % 16 == 0, "scratch sub-arrays stay 16-byte aligned");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_dev[kMaxDevices] = {nullptr};
int g_sms[kMaxDevices] = {0};

blest_status fail(blest_status s, const std::string& m) {
    blest::set_last_error(m);
    return s;
}

}  // namespace

extern "C" blest_status blest_bfs_static_scratch(int32_t n, int64_t num_vss, const int32_t* d_real_ptrs,
                                                 const int32_t* d_row_ids, const uint32_t* d_masks,
                                                 const int32_t* d_new_id, int32_t src_bvss, int32_t* d_levels,
                                                 int32_t update, void* stream) {
    if (n < 1 || num_vss < 0) return fail(BLEST_ERR_INVALID_ARG, "n must be >= 1 and num_vss >= 0");
    if (n > kScratchMaxVertices || num_vss > kScratchMaxVss)
        return fail(BLEST_ERR_TOO_LARGE, "static scratch holds at most 2,097,152 vertices and 524,288 virtual "
                                         "slice sets; use blest_bfs_device for larger graphs");
    if (!d_real_ptrs || !d_levels || (num_vss > 0 && (!d_row_ids || !d_masks)))
        return fail(BLEST_ERR_INVALID_ARG, "NULL device array");
    if (src_bvss < 0 || src_bvss >= n) return fail(BLEST_ERR_INVALID_ARG, "source outside [0, n)");
    if (update != BLEST_UPDATE_EAGER && update != BLEST_UPDATE_LAZY)
        return fail(BLEST_ERR_INVALID_ARG, "update must be BLEST_UPDATE_EAGER or BLEST_UPDATE_LAZY");
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return fail(BLEST_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(BLEST_ERR_CUDA, "device index out of range");
    unsigned char* base = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_dev[dev]) {
            void* p = nullptr;
            if ((e = cudaGetSymbolAddress(&p, g_scratch)) != cudaSuccess)
                return fail(BLEST_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            if ((e = cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
                return fail(BLEST_ERR_CUDA, cudaGetErrorString(e));
            g_scratch_dev[dev] = static_cast<unsigned char*>(p);
        }
        base = g_scratch_dev[dev];
        sms = g_sms[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t words = (size_t)(n + 31) / 32;
    blest::BfsLaunch L;
    L.update = update == BLEST_UPDATE_EAGER ? 1 : 2;
    L.pull = 0;
    L.unroll = 2;
    L.minb = 2;
    L.filter = 1;
    const int per_sm = blest::bfs_max_blocks_per_sm(L.update, L.pull, L.unroll, L.minb, L.depth, 0);
    if (per_sm <= 0) return fail(BLEST_ERR_CUDA, "traversal kernel cannot be resident");
    L.grid = per_sm * sms;
    L.n = n;
    L.qcap = (unsigned int)(num_vss > 0 ? num_vss : 1);
    L.real_ptrs = d_real_ptrs;
    L.row_ids = d_row_ids;
    L.masks = d_masks;
    L.new_id = d_new_id;
    L.levels_internal = d_new_id ? reinterpret_cast<int32_t*>(base + kOffLevels) : d_levels;
    L.vcur = reinterpret_cast<uint32_t*>(base + kOffVcur);
    L.vnext = reinterpret_cast<uint32_t*>(base + kOffVnext);
    for (int i = 0; i < 3; ++i) {
        L.F[i] = reinterpret_cast<uint32_t*>(base + kOffF) + i * words;
        L.Q[i] = reinterpret_cast<unsigned long long*>(base + kOffQ) + (size_t)i * (size_t)L.qcap;
    }
    L.ctrl = base + kOffCtrl;
    L.nroots = 1;
    L.roots_host[0] = src_bvss;
    L.out = d_levels;
    L.timeout_ns = 2000000000ull;
    // Everything the kernel expects to start at zero (or at -1 for levels) is
    // cleared here: the array keeps whatever the previous call left in it.
    unsigned int* ctrl = reinterpret_cast<unsigned int*>(base + kOffCtrl);
    if ((e = cudaMemsetAsync(ctrl, 0, 256, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(L.levels_internal, 0xFF, sizeof(int32_t) * (size_t)n, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(L.vcur, 0, sizeof(uint32_t) * words, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(L.vnext, 0, sizeof(uint32_t) * words, st)) != cudaSuccess ||
        (L.update == 1 && (e = cudaMemsetAsync(L.F[0], 0, 3 * sizeof(uint32_t) * words, st)) != cudaSuccess))
        return fail(BLEST_ERR_CUDA, std::string("clearing scratch: ") + cudaGetErrorString(e));
    if ((e = blest::launch_bfs_kernel(L, st)) != cudaSuccess)
        return fail(BLEST_ERR_CUDA, std::string("traversal launch: ") + cudaGetErrorString(e));
    unsigned int sticky = 0;
    if ((e = cudaMemcpyAsync(&sticky, ctrl + kStickyWord, sizeof(sticky), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(BLEST_ERR_CUDA, std::string("traversal: ") + cudaGetErrorString(e));
    if (sticky == BLEST_ERR_TIMEOUT) return fail(BLEST_ERR_TIMEOUT, "a grid barrier timed out");
    if (sticky) return fail((blest_status)sticky, "device-side consistency check failed");
    return BLEST_OK;
}
