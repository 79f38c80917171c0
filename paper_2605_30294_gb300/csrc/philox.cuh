// Philox4x32-10 counter-based generator (Salmon et al., SC'11), device side.
#pragma once

#include <cstdint>

namespace rfi {

__device__ __forceinline__ uint4 philox_round(uint4 c, uint2 k)
{
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    return make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    c = philox_round(c, k);
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
        c = philox_round(c, k);
    }
    return c;
}

// Top 24 bits of a word as a float in [0, 1) (exact in float).
__device__ __forceinline__ float u24(uint32_t r) { return (float)(r >> 8) * (1.0f / 16777216.0f); }

}  // namespace rfi
