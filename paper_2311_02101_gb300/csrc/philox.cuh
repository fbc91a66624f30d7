// Device Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
// as easy as 1, 2, 3", SC'11): ten rounds, each two 32x32 -> 64-bit products
// of counter words with the Philox multipliers, XORed with the other counter
// words and the round key; the key advances by the Weyl increments between
// rounds.
#pragma once

#include <cstdint>

#include "internal.h"

namespace rbmsat {

__host__ __device__ __forceinline__ RoundKeys philox_keys(uint32_t key0, uint32_t key1) {
  RoundKeys r;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    r.k0[i] = key0 + (uint32_t)i * 0x9E3779B9u;
    r.k1[i] = key1 + (uint32_t)i * 0xBB67AE85u;
  }
  return r;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys& K) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ K.k0[i], lo1, hi0 ^ c.w ^ K.k1[i], lo0);
  }
  return c;
}

// Hidden unit bits of 8 chains from one Philox block and the chains' packed
// threshold words (16-bit thresholds, "always on" bits 48..50): bit h of
// hp[q] |= [u_q < T_q,r] | sat_q,r for unit h = 3 w + r.
__device__ __forceinline__ void hidden_bits(const uint4& R, const uint64_t (&wd)[8], int r, int h,
                                            uint32_t (&hp)[8]) {
  const uint32_t rw[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const uint32_t lo = (uint32_t)wd[q], hi = (uint32_t)(wd[q] >> 32);
    const uint32_t T = r == 0 ? (lo & 0xFFFFu) : r == 1 ? (lo >> 16) : (hi & 0xFFFFu);
    const uint32_t sat = (hi >> (16 + r)) & 1u;
    const uint32_t u = (q & 1) ? (rw[q >> 1] >> 16) : (rw[q >> 1] & 0xFFFFu);
    hp[q] |= ((uint32_t)(u < T) | sat) << h;
  }
}

// 16-bit lane q (0..7) of a Philox output block.
__device__ __forceinline__ uint32_t lane16(const uint4& r, int q) {
  const uint32_t w = q < 2 ? r.x : q < 4 ? r.y : q < 6 ? r.z : r.w;
  return (q & 1) ? (w >> 16) : (w & 0xFFFFu);
}

}  // namespace rbmsat
