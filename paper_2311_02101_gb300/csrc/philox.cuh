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

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;  // multiplier of counter word x
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;  // multiplier of counter word z

// Rounds FIRST .. 9 of Philox4x32-10 on counter state c.
template <int FIRST>
__device__ __forceinline__ uint4 philox_rounds(uint4 c, const RoundKeys& K) {
#pragma unroll
  for (int i = FIRST; i < 10; ++i) {
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c.x;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ K.k0[i], (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ K.k1[i], (uint32_t)p0);
  }
  return c;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys& K) {
  return philox_rounds<0>(c, K);
}

__device__ __forceinline__ uint32_t word_of(const uint4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// acc |= mask when x < w (unsigned): one compare and one predicated OR
__device__ __forceinline__ void or_below(uint32_t& acc, uint32_t x, uint32_t w, uint32_t mask) {
  asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
      : "+r"(acc)
      : "r"(x), "r"(w), "r"(mask));
}

// Hidden draws of one clause for 8 chains (Eq. 2 / Eq. 6 with the negation
// transform) from the chains' pattern records. Unit h draws from the Philox
// block at counter (clause, chain-octet | h << 24, round, hidden phase),
// chain q taking 16-bit lane q (low half of word q / 2 for even q, high half
// for odd q), and bit h of hp[q] becomes [u < P]. Record word 1 + h holds
// (min(P, 65535) << 16) | [P == 65536]: with u moved into the high half of
// a 32-bit word x, the draw is [x < word] (in a group with a saturated unit,
// x keeps only u, so that 0xFFFF0001 is above every x). tab points at the
// group's records as 16-byte chunks and row4[q] is chain q's record in
// chunks; chunk j holds words 4j .. 4j + 3,
// i.e. units 4j - 1 .. 4j + 2 (word 0 of chunk 0 is the free energy).
// hidden_words draws words I0 .. I0 + NW - 1 of chunk j (those below hi);
// its NW Philox blocks run as straight-line code so that their multiply
// chains interleave. With FE it also adds the free energy to fe[q].
template <bool SAT, int I0, int NW, bool FE>
__device__ __forceinline__ void hidden_words(const uint4* tab, const int (&row4)[8], int j, int hi,
                                             uint32_t clause, uint32_t cy, uint32_t t,
                                             uint32_t phase, const RoundKeys& K,
                                             uint32_t (&hp)[8], float (&fe)[8]) {
  uint4 R[NW];
  if (I0 + NW <= hi) {
#pragma unroll
    for (int i = 0; i < NW; ++i)
      R[i] = philox4x32_10(make_uint4(clause, cy + ((uint32_t)(I0 + i) << 24), t, phase), K);
  } else {
#pragma unroll
    for (int i = 0; i < NW; ++i)
      R[i] = I0 + i < hi ? philox4x32_10(make_uint4(clause, cy + ((uint32_t)(I0 + i) << 24), t,
                                                    phase),
                                         K)
                         : make_uint4(0u, 0u, 0u, 0u);
  }
  // the hidden-pattern bit of each word's unit 4 j + I0 + i - 1 (0 past hi,
  // so that OR changes nothing)
  uint32_t mk[NW];
#pragma unroll
  for (int i = 0; i < NW; ++i) mk[i] = I0 + i < hi ? 1u << (4 * j + I0 + i - 1) : 0u;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const uint4 r = tab[row4[q] + j];
    if (FE) fe[q] += __uint_as_float(r.x);
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      // u in the high half of x: the low-half draw moves up; with a saturated
      // unit in the group (word 0xFFFF0001) the high-half draw drops the low
      // half, so x stays below it
      const uint32_t word = word_of(R[i], q >> 1);
      const uint32_t x = (q & 1) ? (SAT ? (word & 0xFFFF0000u) : word) : (word << 16);
      or_below(hp[q], x, word_of(r, I0 + i), mk[i]);
    }
  }
}

// All hidden draws (and the free energy) of one clause for 8 chains. ONE:
// every group's record is one chunk (L <= 3), so no later chunk exists.
// clause is the clause's index within its formula and phase the hidden
// phase with the formula's batch index in bits 8..31.
template <bool SAT, bool ONE>
__device__ __forceinline__ void hidden_draws(const uint4* tab, const int (&row4)[8], int chunks,
                                             int nh, uint32_t clause, uint32_t octet, uint32_t t,
                                             uint32_t phase, const RoundKeys& K,
                                             uint32_t (&hp)[8], float (&fe)[8]) {
  // chunk 0: free energy and units 0..2
  const uint32_t cy0 = octet | (0xFFu << 24);  // unit of word 0 is -1
  hidden_words<SAT, 1, 3, true>(tab, row4, 0, nh + 1 < 4 ? nh + 1 : 4, clause, cy0, t, phase, K, hp,
                                 fe);
  if (ONE) return;
  for (int j = 1; j < chunks; ++j) {
    const int h0 = 4 * j - 1;
    const int hi = nh - h0 < 4 ? nh - h0 : 4;
    const uint32_t cy = octet | ((uint32_t)h0 << 24);
    hidden_words<SAT, 0, 2, false>(tab, row4, j, hi, clause, cy, t, phase, K, hp, fe);
    if (hi > 2) hidden_words<SAT, 2, 2, false>(tab, row4, j, hi, clause, cy, t, phase, K, hp, fe);
  }
}

// 16-bit lane q (0..7) of a Philox output block.
__device__ __forceinline__ uint32_t lane16(const uint4& r, int q) {
  const uint32_t w = q < 2 ? r.x : q < 4 ? r.y : q < 6 ? r.z : r.w;
  return (q & 1) ? (w >> 16) : (w & 0xFFFFu);
}

}  // namespace rbmsat
