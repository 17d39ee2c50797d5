// Bit-plane level helpers of the multi-source traversal (msbfs_kernel.cu),
// host- and device-callable so that a host test can check them bit by bit.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define BLEST_HD __host__ __device__ __forceinline__
#else
#define BLEST_HD inline
#endif

namespace blest {

// Planes needed for the levels of an n-vertex graph: every level is below n,
// so bit_length(n) bits hold it.
BLEST_HD int msbfs_planes(int32_t n) {
    int p = 1;
    while (p < 31 && ((int64_t)1 << p) <= (int64_t)n) ++p;
    return p;
}

// 8 x 8 bit-matrix transpose: byte r of x holds row r (bit c = column c); the
// result's byte c holds column c (bit r = row r).  Three delta swaps over the
// 2 x 2, 4 x 4 and 8 x 8 blocks (the classic recursive block transpose).
BLEST_HD uint64_t transpose8x8(uint64_t x) {
    uint64_t t;
    t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
    x = x ^ t ^ (t << 7);
    t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
    x = x ^ t ^ (t << 14);
    t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
    x = x ^ t ^ (t << 28);
    return x;
}

// Levels of 8 sources from up to 8 planes: pw[p] holds bit p of each source's
// level at bits 8 c .. 8 c + 7 (source 8 c + j at bit 8 c + j).  Byte j of the
// result is the level of source 8 c + j (below 256).
BLEST_HD uint64_t levels_of_8(const uint64_t (&pw)[8], int c) {
    uint64_t rows = 0;
#ifdef __CUDACC__
#pragma unroll
#endif
    for (int p = 0; p < 8; ++p) rows |= ((pw[p] >> (8 * c)) & 0xFFull) << (8 * p);
    return transpose8x8(rows);
}

// Levels of 8 sources from up to 16 planes (levels below 65536): byte j of lo
// and of hi hold bits 0..7 and 8..15 of the level of source 8 c + j.
BLEST_HD void levels_of_8x16(const uint64_t (&pw)[16], int c, uint64_t& lo, uint64_t& hi) {
    uint64_t r0 = 0, r1 = 0;
#ifdef __CUDACC__
#pragma unroll
#endif
    for (int p = 0; p < 8; ++p) {
        r0 |= ((pw[p] >> (8 * c)) & 0xFFull) << (8 * p);
        r1 |= ((pw[8 + p] >> (8 * c)) & 0xFFull) << (8 * p);
    }
    lo = transpose8x8(r0);
    hi = transpose8x8(r1);
}

}  // namespace blest
