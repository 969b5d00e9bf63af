// Counter-based random numbers for the GA: Philox4x32 with 10 rounds
// (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11).  A 128-bit counter and a 64-bit key map to four 32-bit words; the
// library keys the stream with the dock seed and counts (individual,
// generation, run, call), so any word can be recomputed anywhere without
// stored state.
#pragma once

#include <stdint.h>

namespace adgb {

struct Philox4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                           uint32_t c3, uint32_t k0, uint32_t k1) {
    constexpr uint32_t MUL_A = 0xD2511F53u, MUL_B = 0xCD9E8D57u;  // round multipliers
    constexpr uint32_t BUMP_A = 0x9E3779B9u, BUMP_B = 0xBB67AE85u;  // key schedule (Weyl)
#pragma unroll
    for (int round = 0; round < 10; round++) {
        const uint64_t pa = (uint64_t)MUL_A * c0;
        const uint64_t pb = (uint64_t)MUL_B * c2;
        const uint32_t a_hi = (uint32_t)(pa >> 32), a_lo = (uint32_t)pa;
        const uint32_t b_hi = (uint32_t)(pb >> 32), b_lo = (uint32_t)pb;
        c0 = b_hi ^ c1 ^ k0;
        c1 = b_lo;
        c2 = a_hi ^ c3 ^ k1;
        c3 = a_lo;
        k0 += BUMP_A;
        k1 += BUMP_B;
    }
    return {c0, c1, c2, c3};
}

// Word `w` of the stream of (individual k, generation gen, run).
__host__ __device__ __forceinline__ uint32_t ga_word(uint64_t seed, int run, uint32_t gen, int k,
                                                     int w) {
    const Philox4 o = philox4x32_10((uint32_t)k, gen, (uint32_t)run, (uint32_t)(w >> 2),
                                    (uint32_t)seed, (uint32_t)(seed >> 32));
    switch (w & 3) {
        case 0: return o.x;
        case 1: return o.y;
        case 2: return o.z;
        default: return o.w;
    }
}

// Uniform in [0, 1) with 24 bits, exact in float.
__host__ __device__ __forceinline__ float unit24(uint32_t x) {
    return (float)(x >> 8) * (1.0f / 16777216.0f);
}

// Index below n from one word (multiply-shift).
__host__ __device__ __forceinline__ int index_below(uint32_t x, int n) {
    return (int)(((uint64_t)x * (uint64_t)n) >> 32);
}

}  // namespace adgb
