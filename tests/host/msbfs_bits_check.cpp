// The bit-plane helpers of the multi-source traversal against their plain
// definition: transpose8x8 against a double loop on random and structured
// matrices, levels_of_8 against per-source bit sums, msbfs_planes against the
// largest level an n-vertex graph can have.
#include <cstdio>
#include <random>

#include "msbfs_bits.h"

int main() {
    int failures = 0;
    std::mt19937_64 rng(12345);
    for (int it = 0; it < 200000; ++it) {
        const uint64_t x = it < 64 ? (1ull << it) : rng();
        const uint64_t y = blest::transpose8x8(x);
        uint64_t want = 0;
        for (int r = 0; r < 8; ++r)
            for (int c = 0; c < 8; ++c)
                if ((x >> (8 * r + c)) & 1ull) want |= 1ull << (8 * c + r);
        if (y != want && failures++ < 5) std::printf("transpose %016llx -> %016llx want %016llx\n",
                                                     (unsigned long long)x, (unsigned long long)y,
                                                     (unsigned long long)want);
    }
    for (int it = 0; it < 20000; ++it) {
        uint64_t pw[8];
        int lv[64];
        for (int i = 0; i < 64; ++i) lv[i] = (int)(rng() & 0xFF);
        for (int p = 0; p < 8; ++p) {
            pw[p] = 0;
            for (int i = 0; i < 64; ++i) pw[p] |= (uint64_t)((lv[i] >> p) & 1) << i;
        }
        for (int c = 0; c < 8; ++c) {
            const uint64_t got = blest::levels_of_8(pw, c);
            for (int j = 0; j < 8; ++j)
                if ((int)((got >> (8 * j)) & 0xFF) != lv[8 * c + j] && failures++ < 10)
                    std::printf("levels_of_8 c=%d j=%d got %d want %d\n", c, j, (int)((got >> (8 * j)) & 0xFF),
                                lv[8 * c + j]);
        }
    }
    for (int it = 0; it < 20000; ++it) {
        uint64_t pw[16];
        int lv[64];
        for (int i = 0; i < 64; ++i) lv[i] = (int)(rng() & 0xFFFF);
        for (int p = 0; p < 16; ++p) {
            pw[p] = 0;
            for (int i = 0; i < 64; ++i) pw[p] |= (uint64_t)((lv[i] >> p) & 1) << i;
        }
        for (int c = 0; c < 8; ++c) {
            uint64_t lo, hi;
            blest::levels_of_8x16(pw, c, lo, hi);
            for (int j = 0; j < 8; ++j) {
                const int got = (int)((lo >> (8 * j)) & 0xFF) | ((int)((hi >> (8 * j)) & 0xFF) << 8);
                if (got != lv[8 * c + j] && failures++ < 10)
                    std::printf("levels_of_8x16 c=%d j=%d got %d want %d\n", c, j, got, lv[8 * c + j]);
            }
        }
    }
    const int32_t ns[] = {1, 2, 3, 4, 7, 8, 255, 256, 257, 4194304, 16777216, 2147483647};
    for (int32_t n : ns) {
        const int p = blest::msbfs_planes(n);
        // the largest level, n - 1, must fit, and (for n > 1) one plane fewer must not hold n - 1
        // unless n - 1 < 2^(p - 1)
        const bool fits = p >= 31 || ((int64_t)(n - 1) < ((int64_t)1 << p));
        if (!fits && failures++ < 20) std::printf("planes(%d) = %d too few\n", n, p);
        if (p > 1 && p < 31 && (int64_t)n < ((int64_t)1 << (p - 1)) && failures++ < 20)
            std::printf("planes(%d) = %d more than needed\n", n, p);
    }
    std::printf("failures=%d\n", failures);
    return failures ? 1 : 0;
}
