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

// The same function for the counters (g, sw, p, j) of one chain group g
// under one key, with what does not change between its calls computed once:
// the ten round keys (k + r W) and the first round's product of g.  The
// producers of a sweep launch make ~1000 calls a sweep with one (g, key):
// this saves the 18 key additions and 2 of the 40 multiplies of each.
struct PhiloxGroup {
  uint32_t K0[10], K1[10];
  uint32_t g_hi, g_lo;  // 0xD2511F53 * g
};
__device__ __forceinline__ PhiloxGroup philox_group(uint32_t g, uint32_t k0, uint32_t k1) {
  PhiloxGroup P;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    P.K0[r] = k0 + (uint32_t)r * 0x9E3779B9u;
    P.K1[r] = k1 + (uint32_t)r * 0xBB67AE85u;
  }
  const uint64_t p0 = (uint64_t)0xD2511F53u * g;
  P.g_hi = (uint32_t)(p0 >> 32);
  P.g_lo = (uint32_t)p0;
  return P;
}
__device__ __forceinline__ uint4 philox4x32_10_group(const PhiloxGroup& P, uint32_t sw, uint32_t p,
                                                     uint32_t j) {
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * p;
  uint4 c = make_uint4((uint32_t)(p1 >> 32) ^ sw ^ P.K0[0], (uint32_t)p1, P.g_hi ^ j ^ P.K1[0],
                       P.g_lo);
#pragma unroll
  for (int round = 1; round < 10; ++round) {
    const uint64_t q0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t q1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(q1 >> 32) ^ c.y ^ P.K0[round], (uint32_t)q1,
                   (uint32_t)(q0 >> 32) ^ c.w ^ P.K1[round], (uint32_t)q0);
  }
  return c;
}

}  // namespace pb
