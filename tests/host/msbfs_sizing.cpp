// The multi-source launcher splits k sources into chunks of at most 256 and sizes
// each chunk's buffers with msbfs_words / msbfs_plane_words; a caller that
// allocates a launch's state up front (the query server) sizes it with the same
// functions for the whole k.  Checks that every chunk fits that state and that
// each buffer holds what the kernel indexes: n * W words with 64 W >= k, and
// msbfs_planes(n) level planes of n * W words, enough bits for level n - 1.
#include <cstdio>

#include "msbfs_launch.h"

int main() {
    int failures = 0;
    const int32_t ns[] = {1, 7, 32, 33, 1000, 4194304};
    for (int32_t n : ns) {
        for (int64_t k = 1; k <= 2048; ++k) {
            const int whole_w = blest::msbfs_words(k);
            const int64_t whole_l = blest::msbfs_plane_words(n, k);
            for (int64_t i0 = 0; i0 < k; i0 += blest::kMsbfsChunk) {
                const int64_t kc = k - i0 < blest::kMsbfsChunk ? k - i0 : blest::kMsbfsChunk;
                const int w = blest::msbfs_words(kc);
                const int64_t l = blest::msbfs_plane_words(n, kc);
                const int planes = blest::msbfs_planes(n);
                const int64_t rows = blest::msbfs_level_entries(n, kc);
                const int64_t stride = rows / n;
                const bool ok = w <= whole_w && l <= whole_l && 64 * w >= kc && (w == 1 || w == 2 || w == 4) &&
                                l == (int64_t)planes * n * w && (int64_t)(n - 1) < ((int64_t)1 << planes) &&
                                rows <= blest::msbfs_level_entries(n, k) && rows % n == 0 && stride % 8 == 0 &&
                                stride >= kc && stride < kc + 8;
                if (!ok) {
                    if (failures < 10)
                        std::printf("n=%d k=%lld chunk at %lld: words %d/%d levels %lld/%lld\n", n, (long long)k,
                                    (long long)i0, w, whole_w, (long long)l, (long long)whole_l);
                    ++failures;
                }
            }
        }
    }
    std::printf("failures=%d\n", failures);
    return failures ? 1 : 0;
}
