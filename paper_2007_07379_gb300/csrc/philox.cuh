// Philox4x32-10 on the device (Salmon, Moraes, Dror, Shaw, SC'11): ten
// rounds of two 32x32->64 multiplies by 0xD2511F53 / 0xCD9E8D57 with the key
// advanced by the Weyl increments 0x9E3779B9 / 0xBB67AE85 between rounds.
#pragma once
#include <cstdint>

namespace pb {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    // one widening multiply gives both halves of each product
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1,
                   (uint32_t)p0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

}  // namespace pb
