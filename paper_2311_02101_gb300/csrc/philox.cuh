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

// Samples the hidden units h = 3 w .. min(3 w + 3, nh) - 1 of one clause for
// 8 chains (Eq. 2 / Eq. 6 with the negation transform). Unit h draws from the
// Philox block at counter (clause, chain-octet | h << 24, round, hidden phase),
// chain q taking its 16-bit lane q; the threshold word w of chain q is
// tab[row[q] * words + w] (thresholds min(P, 65535) in bits 16 r .. 16 r + 15,
// [P == 65536] in bit 48 + r), and bit h of hp[q] becomes [u < P]. A full word
// computes its three Philox blocks in straight-line code so that their
// multiply chains interleave, and reads the words only after them.
__device__ __forceinline__ void hidden_word(const unsigned long long* tab, const int (&row)[8],
                                            int words, int w, int nh, uint32_t clause,
                                            uint32_t octet, uint32_t t, const RoundKeys& K,
                                            uint32_t (&hp)[8]) {
  const int h0 = 3 * w;
  const int nr = nh - h0 < 3 ? nh - h0 : 3;
  uint4 R0, R1 = make_uint4(0, 0, 0, 0), R2 = make_uint4(0, 0, 0, 0);
  const uint32_t cy = octet | ((uint32_t)h0 << 24);
  if (nr == 3) {
    R0 = philox4x32_10(make_uint4(clause, cy, t, kPhaseHidden), K);
    R1 = philox4x32_10(make_uint4(clause, cy + (1u << 24), t, kPhaseHidden), K);
    R2 = philox4x32_10(make_uint4(clause, cy + (2u << 24), t, kPhaseHidden), K);
  } else {
    R0 = philox4x32_10(make_uint4(clause, cy, t, kPhaseHidden), K);
    if (nr == 2) R1 = philox4x32_10(make_uint4(clause, cy + (1u << 24), t, kPhaseHidden), K);
  }
  const uint32_t keep = (1u << nr) - 1u;
  const uint32_t r0[4] = {R0.x, R0.y, R0.z, R0.w}, r1[4] = {R1.x, R1.y, R1.z, R1.w},
                 r2[4] = {R2.x, R2.y, R2.z, R2.w};
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const unsigned long long wq = tab[row[q] * words + w];
    const uint32_t lo = (uint32_t)wq, hi = (uint32_t)(wq >> 32);
    const int sh = 16 * (q & 1);
    const uint32_t u0 = (r0[q >> 1] >> sh) & 0xFFFFu, u1 = (r1[q >> 1] >> sh) & 0xFFFFu,
                   u2 = (r2[q >> 1] >> sh) & 0xFFFFu;
    const uint32_t bits = (uint32_t)(u0 < (lo & 0xFFFFu)) | ((uint32_t)(u1 < (lo >> 16)) << 1) |
                          ((uint32_t)(u2 < (hi & 0xFFFFu)) << 2) | ((hi >> 16) & 7u);
    hp[q] |= (bits & keep) << h0;
  }
}

// 16-bit lane q (0..7) of a Philox output block.
__device__ __forceinline__ uint32_t lane16(const uint4& r, int q) {
  const uint32_t w = q < 2 ? r.x : q < 4 ? r.y : q < 6 ? r.z : r.w;
  return (q & 1) ? (w >> 16) : (w & 0xFFFFu);
}

}  // namespace rbmsat
