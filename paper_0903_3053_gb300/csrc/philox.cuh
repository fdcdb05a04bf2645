// philox.cuh -- device Philox4x32-10 counter-based generator.
//
// Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds, each multiplying counter words 0 and 2 by two fixed odd
// 32-bit constants, the high halves of the products xor-ed with the other two
// counter words and the round key, the low halves passed through; the 64-bit
// key advances by a Weyl sequence between rounds.  It replaces the paper's
// stateful RANMAR (Sec. 2.2): a counter-based stream needs no per-thread state
// in memory and gives every site its own reproducible numbers.
#pragma once
#include <cstdint>

namespace mc {

// Tags in the top byte of counter word 2 (what the numbers are used for).
constexpr uint32_t kTagIsingInit = 0x01000000u;
constexpr uint32_t kTagIsingMetro = 0x02000000u;
constexpr uint32_t kTagSu2Init = 0x11000000u;
constexpr uint32_t kTagSu2Heatbath = 0x12000000u;
constexpr uint32_t kTagSu2Direction = 0x13000000u;

struct PhiloxKey {
    uint32_t k0, k1;
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, PhiloxKey key)
{
    constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
    constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
    uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hi0 = __umulhi(kMul0, x.x);
        const uint32_t lo0 = kMul0 * x.x;
        const uint32_t hi1 = __umulhi(kMul1, x.z);
        const uint32_t lo1 = kMul1 * x.z;
        x = make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
        k0 += kWeyl0;
        k1 += kWeyl1;
    }
    return x;
}

// The ten round keys of one 64-bit key.  A thread that draws many blocks under
// the same key computes them once: the Weyl increments then cost nothing per
// block, and each round is two 32x32->64 multiplies and two three-input xors.
struct PhiloxSchedule {
    uint32_t k0[10], k1[10];
};

__device__ __forceinline__ PhiloxSchedule philox_schedule(PhiloxKey key)
{
    PhiloxSchedule s;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        s.k0[r] = key.k0 + (uint32_t)r * 0x9E3779B9u;
        s.k1[r] = key.k1 + (uint32_t)r * 0xBB67AE85u;
    }
    return s;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, const PhiloxSchedule &ks)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * x.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * x.z;
        x = make_uint4((uint32_t)(p1 >> 32) ^ x.y ^ ks.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ x.w ^ ks.k1[r],
                       (uint32_t)p0);
    }
    return x;
}

// 32-bit random word -> float in (0, 1] with 24-bit resolution.  Exact in FP32:
// ((r >> 8) + 1) <= 2^24 is representable and the scale is a power of two.
__device__ __forceinline__ float uniform_open0(uint32_t r)
{
    return (float)((r >> 8) + 1u) * 5.9604644775390625e-8f; // 2^-24
}

}  // namespace mc
