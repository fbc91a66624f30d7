// Parallel-tempering swap rounds between adjacent temperatures of the chain
// ensemble (the paper's temperature ensemble, Sec. 4.2, with the replica
// exchange it leaves to future work, Sec. 7).
//
// Chains form E contiguous temperature blocks of S chains. In a round with
// parity p, chain a = e S + k of every block e = p, p + 2, ... (e + 1 < E) and
// chain b = a + S exchange states (x and nu) iff
//   D = F_e(x_a) + F_{e+1}(x_b) - F_e(x_b) - F_{e+1}(x_a) >= Tc[u],
// the Metropolis rule min(1, exp(D)) for exchanging two states between the
// targets exp(-F_e) and exp(-F_{e+1}). The free energies are the exact
// fixed-point sums of rint(2^20 F_c) over clauses (int64), u is the 16-bit
// draw of chain a at counter (0, a >> 3, round, swap phase), lane a & 7, and
// Tc[u] = ceil(2^20 ln(u / 65536)) is computed once on the host (Tc[0] =
// INT64_MIN). All decisions are integer comparisons.
//   k_pt_energy  one thread = one clause x 8 chains: truth patterns (as the
//                gather), the fixed-point free energy at the chain's own
//                temperature and at its partner's; int64 atomics (exact).
//   k_pt_decide  one thread per pair.
//   k_pt_swap    one thread = one variable x the 8 lower chains of an octet:
//                exchanges the state bytes and nu of the accepted pairs.
#include <cstdint>

#include "internal.h"
#include "philox.cuh"

namespace rbmsat {

namespace {

constexpr int kPtClauses = 64;  // clauses per block of the energy pass

// partner temperature of a chain at temperature e in a round of parity p
// (-1: no partner)
__device__ __forceinline__ int pt_partner(int e, int E, int parity) {
  if (((e - parity) & 1) == 0) return e + 1 < E ? e + 1 : -1;
  return e >= 1 ? e - 1 : -1;
}

__global__ void __launch_bounds__(256) k_pt_energy(DevFormula F, DevTables T, const uint8_t* xt,
                                                   int B, int Bp, int S, int E, int parity,
                                                   unsigned long long* Fown,
                                                   unsigned long long* Foth) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g8 = blockIdx.x * 32 + lane, b0 = g8 * 8;
  const int c0 = blockIdx.y * kPtClauses, c1 = min(c0 + kPtClauses, F.m);
  int e[8], ep[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    e[q] = min((b0 + q) / S, E - 1);
    ep[q] = pt_partner(e[q], E, parity);
  }
  long long own[8], oth[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) own[q] = oth[q] = 0;
  for (int c = c0 + warp; c < c1; c += 8) {
    const int grp = __ldg(F.cl_grp + c);
    if (grp < 0) continue;  // an empty clause has no clause RBM
    const int o = __ldg(F.cl_off + c);
    const int len = __ldg(F.cl_off + c + 1) - o;
    // byte q of lo0|lo1 (hi0|hi1): bits 0..7 (8..15) of chain q's truth pattern
    uint32_t lo0 = 0, lo1 = 0, hi0 = 0, hi1 = 0;
    for (int k = 0; k < len; ++k) {
      const int32_t lv = __ldg(F.lit_var + o + k);
      const uint2 x8 =
          __ldg(reinterpret_cast<const uint2*>(xt + (size_t)(lv & 0x7FFFFFFF) * Bp + b0));
      const uint32_t flip = lv < 0 ? 0x01010101u : 0u;
      if (k < 8) {
        lo0 |= (x8.x ^ flip) << k;
        lo1 |= (x8.y ^ flip) << k;
      } else {
        hi0 |= (x8.x ^ flip) << (k - 8);
        hi1 |= (x8.y ^ flip) << (k - 8);
      }
    }
    const int32_t* fq = T.feq + T.meta[grp].feq_off;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t lo = q < 4 ? lo0 : lo1, hi = q < 4 ? hi0 : hi1;
      const int p = (int)((lo >> (8 * (q & 3))) & 0xFFu) | (int)(((hi >> (8 * (q & 3))) & 0xFFu) << 8);
      own[q] += __ldg(fq + (e[q] << len) + p);
      if (ep[q] >= 0) oth[q] += __ldg(fq + (ep[q] << len) + p);
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (b0 + q >= B) continue;
    atomicAdd(Fown + b0 + q, (unsigned long long)own[q]);
    if (ep[q] >= 0) atomicAdd(Foth + b0 + q, (unsigned long long)oth[q]);
  }
}

__global__ void k_pt_decide(DevChains C, int S, int E, int parity, uint32_t t, int pairs,
                            const long long* Tc, const long long* Fown, const long long* Foth,
                            uint8_t* flag, int* n_acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pairs) return;
  const int e = parity + 2 * (i / S);
  const int a = e * S + i % S, b = a + S;
  const long long D = Fown[a] + Fown[b] - Foth[b] - Foth[a];
  const uint4 r = philox4x32_10(make_uint4(0u, (uint32_t)(a >> 3), t, kPhaseSwap), C.keys);
  const uint32_t u = lane16(r, a & 7);
  const bool ok = D >= Tc[u];
  flag[a] = ok ? 1 : 0;
  if (ok) atomicAdd(n_acc, 1);
}

__global__ void __launch_bounds__(256) k_pt_swap(DevChains C, int n, int S, int parity, int octets,
                                                 const uint8_t* flag, int vg0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int o8 = blockIdx.x * 32 + lane;  // octet among the lower members
  const int i = (vg0 + blockIdx.y) * 8 + warp;
  if (o8 >= octets || i >= n) return;
  const int per = S / 8;
  const int a0 = (parity + 2 * (o8 / per)) * S + 8 * (o8 % per), b0 = a0 + S;
  const uint64_t f = *reinterpret_cast<const uint64_t*>(flag + a0);
  if (!f) return;
  const uint64_t mask = f * 0xFFull;
  uint64_t* xa = reinterpret_cast<uint64_t*>(C.xt + (size_t)i * C.Bp + a0);
  uint64_t* xb = reinterpret_cast<uint64_t*>(C.xt + (size_t)i * C.Bp + b0);
  const uint64_t va = *xa, vb = *xb;
  *xa = (va & ~mask) | (vb & mask);
  *xb = (vb & ~mask) | (va & mask);
  float* na = C.nu + (size_t)i * C.Bp + a0;
  float* nb = C.nu + (size_t)i * C.Bp + b0;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if ((f >> (8 * q)) & 1u) {
      const float tmp = na[q];
      na[q] = nb[q];
      nb[q] = tmp;
    }
}

}  // namespace

cudaError_t launch_pt_round(const DevFormula& F, const DevTables& T, const DevChains& C, int S,
                            int E, int parity, uint32_t t, const long long* Tc, long long* Fown,
                            long long* Foth, uint8_t* flag, int* n_acc, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(Fown, 0, sizeof(long long) * C.Bp, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(Foth, 0, sizeof(long long) * C.Bp, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, C.Bp, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n_acc, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (F.m > 0) {
    dim3 grid(C.Bp / kChainTile, (F.m + kPtClauses - 1) / kPtClauses);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    k_pt_energy<<<grid, 256, 0, st>>>(F, T, C.xt, C.B, C.Bp, S, E, parity,
                                      reinterpret_cast<unsigned long long*>(Fown),
                                      reinterpret_cast<unsigned long long*>(Foth));
  }
  const int lower_blocks = (E - parity) / 2;  // e = parity, parity + 2, ... with e + 1 < E
  const int pairs = lower_blocks * S;
  if (pairs <= 0) return cudaGetLastError();
  k_pt_decide<<<(pairs + 255) / 256, 256, 0, st>>>(C, S, E, parity, t, pairs, Tc, Fown, Foth, flag,
                                                   n_acc);
  const int octets = pairs / 8, groups = (F.n + 7) / 8;
  for (int vg0 = 0; vg0 < groups; vg0 += 65535) {
    dim3 grid((octets + 31) / 32, groups - vg0 < 65535 ? groups - vg0 : 65535);
    k_pt_swap<<<grid, 256, 0, st>>>(C, F.n, S, parity, octets, flag, vg0);
  }
  return cudaGetLastError();
}

}  // namespace rbmsat
