// Sparse-gather path of one RbmSAT Gibbs round.
//
// The paper's experiments use the accelerator's vector unit with gathers for
// the clause inputs and a segment-sum for the scatter-add (appendix "Gather
// and scatter-add operations"); this is the GB300 counterpart. It works
// directly on the literal lists, never on a dense clause-variable matrix:
//   k_gather   one thread = one clause x 8 chains: reads the clause's literal
//              truths for 8 chains at once (8 bytes per literal from the
//              variable-major state), forms the truth pattern, adds the weight
//              of unsatisfied clauses, the clause free energy (Eq. 1) and
//              draws the hidden units (Eq. 2 / Eq. 6); writes each literal's
//              scatter contribution G for the 8 chains (16 bytes).
//   k_best_keep  reduces the per-block costs / free energies in a fixed order
//              and keeps improving states (Sec. 4.2).
//   k_visible  one thread = one variable x 8 chains: pull-based scatter-sum of
//              G over the variable's literals (Eq. 7; no atomics, so the sums
//              are exact and deterministic), draws the new visible states
//              (Eq. 3), updates nu (Sec. 4.4) and copies improved states into
//              the best-so-far before they are overwritten.
// State layout: x and nu are variable-major (n x Bp) so 8 consecutive chains of
// one variable are one 8-byte (x) or 32-byte (nu) access.
#include <cstdint>

#include "internal.h"
#include "philox.cuh"

namespace rbmsat {

namespace {

__device__ __forceinline__ uint32_t step_index(const uint32_t* tdev, uint32_t t_rel) {
  return (tdev ? *tdev : 0u) + t_rel;
}

__device__ __forceinline__ int temp_of(int b, int E, int B) {
  const int e = (int)(((int64_t)b * E) / B);
  return e < E - 1 ? e : E - 1;
}

__global__ void __launch_bounds__(256) k_init(DevChains C, int n) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g8 = blockIdx.x * 32 + lane, b0 = g8 * 8;
  const int i = blockIdx.y * 8 + warp;
  if (i < n) {
    const RoundKeys K = philox_keys(C.key0, C.key1);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)g8, 0u, kPhaseInit), K);
    uint64_t x = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) x |= (uint64_t)(lane16(r, q) < 32768u) << (8 * q);
    const size_t o = (size_t)i * C.Bp + b0;
    *reinterpret_cast<uint64_t*>(C.xt + o) = x;
    *reinterpret_cast<uint64_t*>(C.best_xt + o) = x;
    const float4 v = make_float4(0.25f, 0.25f, 0.25f, 0.25f);
    reinterpret_cast<float4*>(C.nu + o)[0] = v;
    reinterpret_cast<float4*>(C.nu + o)[1] = v;
  }
  if (blockIdx.y == 0 && warp == 0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      C.best[b0 + q] = INT64_MAX;
      C.improved[b0 + q] = 0;
    }
  }
}

template <bool SAMPLE, bool FE>
__global__ void __launch_bounds__(256) k_gather(DevFormula F, DevTables T, DevChains C,
                                                const uint8_t* __restrict__ xt, int Bp,
                                                int cblock, const uint32_t* tdev,
                                                uint32_t t_rel, int64_t* cost_part,
                                                float* fe_part) {
  __shared__ int64_t s_cost[8][256];
  __shared__ float s_fe[8][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g8 = blockIdx.x * 32 + lane, b0 = g8 * 8;
  const int c_begin = blockIdx.y * cblock;
  const int c_end = min(c_begin + cblock, F.m);
  const int E = T.n_temps;

  int e[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) e[q] = (SAMPLE || FE) ? temp_of(b0 + q, E, C.B) : 0;
  int64_t cost[8];
  float fe[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    cost[q] = 0;
    fe[q] = 0.f;
  }
  RoundKeys K;
  uint32_t t = 0;
  if (SAMPLE) {
    K = philox_keys(C.key0, C.key1);
    t = step_index(tdev, t_rel);
  }

  for (int c = c_begin + warp; c < c_end; c += 8) {
    const int o = __ldg(F.cl_off + c);
    const int len = __ldg(F.cl_off + c + 1) - o;
    // truth pattern of the clause's literals for 8 chains: byte q of plo holds
    // bits 0..7 of chain q's pattern, byte q of phi bits 8..15
    uint64_t plo = 0, phi = 0;
    for (int k = 0; k < len; ++k) {
      const int32_t lv = __ldg(F.lit_var + o + k);
      const int v = lv & 0x7FFFFFFF;
      uint64_t x8 = __ldg(reinterpret_cast<const unsigned long long*>(xt + (size_t)v * Bp + b0));
      if (lv < 0) x8 ^= 0x0101010101010101ull;
      if (k < 8) plo |= x8 << k;
      else phi |= x8 << (k - 8);
    }
    int p[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      p[q] = (int)((plo >> (8 * q)) & 0xFFu) | ((int)((phi >> (8 * q)) & 0xFFu) << 8);
    const int64_t wc = __ldg(F.cl_w + c);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (p[q] == 0) cost[q] += wc;
    if (!(SAMPLE || FE) || len == 0) continue;

    const int grp = __ldg(F.cl_grp + c);
    int s[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] = grp * E + e[q];
    if (FE) {
#pragma unroll
      for (int q = 0; q < 8; ++q) fe[q] += __ldg(T.fe + __ldg(T.fe_off + s[q]) + p[q]);
    }
    if (!SAMPLE) continue;

    const int L = __ldg(T.grp_nh + grp);
    int pbase[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) pbase[q] = __ldg(T.phid_off + s[q]) + p[q] * L;
    uint32_t hp[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) hp[q] = 0;
    for (int h = 0; h < L; ++h) {
      const uint4 r = philox4x32_10(
          make_uint4((uint32_t)c, (uint32_t)g8 | ((uint32_t)h << 24), t, kPhaseHidden), K);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        hp[q] |= (uint32_t)(lane16(r, q) < __ldg(T.phid + pbase[q] + h)) << h;
    }
    int gbase[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) gbase[q] = __ldg(T.gq_off + s[q]) + (int)hp[q] * len;
    for (int k = 0; k < len; ++k) {
      uint32_t w[4];
#pragma unroll
      for (int h2 = 0; h2 < 4; ++h2) {
        const uint32_t lo = (uint16_t)__ldg(T.gq + gbase[2 * h2] + k);
        const uint32_t hi = (uint16_t)__ldg(T.gq + gbase[2 * h2 + 1] + k);
        w[h2] = lo | (hi << 16);
      }
      *reinterpret_cast<uint4*>(C.G + (size_t)(o + k) * Bp + b0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }

#pragma unroll
  for (int q = 0; q < 8; ++q) {
    s_cost[warp][lane * 8 + q] = cost[q];
    s_fe[warp][lane * 8 + q] = fe[q];
  }
  __syncthreads();
  const int tid = threadIdx.x;
  int64_t tc = 0;
  float tf = 0.f;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    tc += s_cost[w][tid];
    tf += s_fe[w][tid];
  }
  const size_t out = (size_t)blockIdx.y * Bp + (size_t)blockIdx.x * 256 + tid;
  cost_part[out] = tc;
  if (FE) fe_part[out] = tf;
}

// Block = 32 chains (lanes) x 8 warps over clause blocks; fixed summation order.
__global__ void __launch_bounds__(256) k_best_keep(DevChains C, int nblk) {
  __shared__ int64_t s_cost[8][32];
  __shared__ float s_fe[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = blockIdx.x * 32 + lane;
  int64_t c = 0;
  float f = 0.f;
  for (int k = warp; k < nblk; k += 8) {
    c += C.cost_part[(size_t)k * C.Bp + b];
    f += C.fe_part[(size_t)k * C.Bp + b];
  }
  s_cost[warp][lane] = c;
  s_fe[warp][lane] = f;
  __syncthreads();
  if (warp == 0) {
    int64_t tc = 0;
    float tf = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      tc += s_cost[w][lane];
      tf += s_fe[w][lane];
    }
    C.cost[b] = tc;
    C.fe[b] = tf;
    const bool imp = tc < C.best[b];
    if (imp) C.best[b] = tc;
    C.improved[b] = imp ? 1 : 0;
  }
}

__device__ __forceinline__ void keep_improved(const DevChains& C, size_t o, int b0,
                                              uint64_t xold) {
  const uint64_t imp = *reinterpret_cast<const uint64_t*>(C.improved + b0);
  if (imp) {
    const uint64_t mask = imp * 0xFFull;  // 0x01 flags -> 0xFF byte masks
    uint64_t* bx = reinterpret_cast<uint64_t*>(C.best_xt + o);
    *bx = (*bx & ~mask) | (xold & mask);
  }
}

__global__ void __launch_bounds__(256) k_visible(DevFormula F, DevTables T, DevChains C,
                                                 float alpha, const uint32_t* tdev,
                                                 uint32_t t_rel) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g8 = blockIdx.x * 32 + lane, b0 = g8 * 8;
  const int i = blockIdx.y * 8 + warp;
  if (i >= F.n) return;
  const uint32_t t = step_index(tdev, t_rel);
  int z[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) z[q] = 0;
  const int j_end = __ldg(F.var_off + i + 1);
  for (int jj = __ldg(F.var_off + i); jj < j_end; ++jj) {
    const int32_t jl = __ldg(F.var_lit + jj);
    const int j = jl & 0x7FFFFFFF;
    const uint4 g = __ldg(reinterpret_cast<const uint4*>(C.G + (size_t)j * C.Bp + b0));
    const uint32_t w[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int v = (int)(int16_t)((q & 1) ? (w[q >> 1] >> 16) : (w[q >> 1] & 0xFFFFu));
      z[q] += jl < 0 ? -v : v;
    }
  }
  const size_t o = (size_t)i * C.Bp + b0;
  const uint64_t xold = *reinterpret_cast<const uint64_t*>(C.xt + o);
  keep_improved(C, o, b0, xold);

  const RoundKeys K = philox_keys(C.key0, C.key1);
  const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)g8, t, kPhaseVisible), K);
  float4* nu4 = reinterpret_cast<float4*>(C.nu + o);
  float4 n0 = nu4[0], n1 = nu4[1];
  float nu[8] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
  const float keep = 1.0f - alpha;
  uint64_t xnew = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int qq = max(-T.qmax, min(T.qmax, z[q]));
    const uint32_t P = __ldg(T.pv + qq + T.qmax);
    // rho (1 - rho) with rho = P / 65536: P (65536 - P) < 2^31, scaled by 2^-32
    const float var = (float)(P * (65536u - P)) * 2.3283064365386963e-10f;
    nu[q] = keep * nu[q] + alpha * var;
    xnew |= (uint64_t)(lane16(r, q) < P) << (8 * q);
  }
  nu4[0] = make_float4(nu[0], nu[1], nu[2], nu[3]);
  nu4[1] = make_float4(nu[4], nu[5], nu[6], nu[7]);
  *reinterpret_cast<uint64_t*>(C.xt + o) = xnew;
}

__global__ void __launch_bounds__(256) k_keep_copy(DevChains C, int n) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b0 = (blockIdx.x * 32 + lane) * 8;
  const int i = blockIdx.y * 8 + warp;
  if (i >= n) return;
  const size_t o = (size_t)i * C.Bp + b0;
  keep_improved(C, o, b0, *reinterpret_cast<const uint64_t*>(C.xt + o));
}

__global__ void k_advance(uint32_t* tdev, uint32_t by) { *tdev += by; }
__global__ void k_set_u32(uint32_t* dst, uint32_t value) { *dst = value; }

// assign (B x n, chain-major, any nonzero = 1) -> xt (n x Bp, 0/1); chains
// B..Bp-1 read as all-false.
__global__ void k_transpose_in(const uint8_t* __restrict__ assign, int B, int n,
                               uint8_t* __restrict__ xt, int Bp) {
  __shared__ uint8_t tile[32][33];
  const int i0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int b = b0 + r, i = i0 + threadIdx.x;
    tile[r][threadIdx.x] = (b < B && i < n) ? (assign[(size_t)b * n + i] != 0) : 0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int i = i0 + r, b = b0 + threadIdx.x;
    if (i < n) xt[(size_t)i * Bp + b] = tile[threadIdx.x][r];
  }
}

__global__ void k_reduce_cost(const int64_t* __restrict__ part, int nblk, int Bp, int B,
                              int64_t* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  int64_t c = 0;
  for (int k = 0; k < nblk; ++k) c += part[(size_t)k * Bp + b];
  out[b] = c;
}

}  // namespace

int clause_block_for(int m) {
  const int per = (m + 255) / 256;
  return per > kClauseBlock ? per : kClauseBlock;
}

int clause_blocks_for(int m) {
  const int cb = clause_block_for(m);
  const int nb = (m + cb - 1) / cb;
  return nb > 0 ? nb : 1;
}

cudaError_t launch_init_sparse(const DevChains& C, int n, cudaStream_t st) {
  dim3 grid(C.Bp / kChainTile, (n + 7) / 8);
  k_init<<<grid, 256, 0, st>>>(C, n);
  return cudaGetLastError();
}

cudaError_t launch_gather(const DevFormula& F, const DevTables& T, const DevChains& C,
                          const uint8_t* xt, int Bp, bool sample, bool fe,
                          const uint32_t* tdev, uint32_t t_rel, int64_t* cost_part,
                          float* fe_part, cudaStream_t st) {
  const int cb = clause_block_for(F.m);
  dim3 grid(Bp / kChainTile, clause_blocks_for(F.m));
  if (sample)
    k_gather<true, true><<<grid, 256, 0, st>>>(F, T, C, xt, Bp, cb, tdev, t_rel, cost_part, fe_part);
  else if (fe)
    k_gather<false, true><<<grid, 256, 0, st>>>(F, T, C, xt, Bp, cb, tdev, t_rel, cost_part, fe_part);
  else
    k_gather<false, false><<<grid, 256, 0, st>>>(F, T, C, xt, Bp, cb, tdev, t_rel, cost_part, fe_part);
  return cudaGetLastError();
}

cudaError_t launch_best_keep(const DevFormula& F, const DevChains& C, cudaStream_t st) {
  k_best_keep<<<C.Bp / 32, 256, 0, st>>>(C, clause_blocks_for(F.m));
  return cudaGetLastError();
}

cudaError_t launch_visible(const DevFormula& F, const DevTables& T, const DevChains& C,
                           float alpha, const uint32_t* tdev, uint32_t t_rel,
                           cudaStream_t st) {
  dim3 grid(C.Bp / kChainTile, (F.n + 7) / 8);
  k_visible<<<grid, 256, 0, st>>>(F, T, C, alpha, tdev, t_rel);
  return cudaGetLastError();
}

cudaError_t launch_keep_copy(const DevChains& C, int n, cudaStream_t st) {
  dim3 grid(C.Bp / kChainTile, (n + 7) / 8);
  k_keep_copy<<<grid, 256, 0, st>>>(C, n);
  return cudaGetLastError();
}

cudaError_t launch_advance(uint32_t* tdev, uint32_t by, cudaStream_t st) {
  k_advance<<<1, 1, 0, st>>>(tdev, by);
  return cudaGetLastError();
}

cudaError_t launch_set_u32(uint32_t* dst, uint32_t value, cudaStream_t st) {
  k_set_u32<<<1, 1, 0, st>>>(dst, value);
  return cudaGetLastError();
}

cudaError_t launch_transpose_in(const uint8_t* assign, int B, int n, uint8_t* xt, int Bp,
                                cudaStream_t st) {
  dim3 grid((n + 31) / 32, Bp / 32);
  k_transpose_in<<<grid, dim3(32, 8), 0, st>>>(assign, B, n, xt, Bp);
  return cudaGetLastError();
}

cudaError_t launch_reduce_cost(const int64_t* part, int nblk, int Bp, int B,
                               int64_t* out, cudaStream_t st) {
  k_reduce_cost<<<(B + 255) / 256, 256, 0, st>>>(part, nblk, Bp, B, out);
  return cudaGetLastError();
}

}  // namespace rbmsat
