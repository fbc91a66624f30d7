// Dense tensor-core path of one Gibbs round (Sec. 4.3 "gather" and
// "scatter-add" as matrix products).
//
//   k_gemm1_step  gather: the FP8 pattern-encoding clause matrix times the
//                 +-1 chain states (tcgen05 kind::f8f6f4, see dense.cu); the
//                 epilogue decodes each clause x chain truth pattern, sums
//                 the weighted unsatisfied cost and the clause free energy
//                 (Eq. 1) per chain over its 128 rows, draws the hidden units
//                 (Eq. 2 / Eq. 6) and stores the hidden pattern (one byte per
//                 clause and chain, as the sparse path).
//   k_keep_dense  per chain: sums the per-tile partials in tile order and
//                 keeps improvements (Sec. 4.2).
//   k_gemm2       scatter-add: Z = P^T G, the variable x literal-incidence
//                 matrix P^T (+-1, BF16 or FP16) times the per-literal
//                 contributions G of the hidden patterns (Eq. 7). Incidences
//                 are sorted by variable, so a tile of 128 variables only
//                 spans its own incidence range: the product is
//                 block-diagonal and each tile loops over its own K-blocks.
//                 TMA loads P^T; 16 builder warps expand the hidden patterns
//                 into the 128-byte-swizzled G tile in shared memory (table
//                 lookups, no HBM round trip); one thread issues
//                 tcgen05.mma kind::f16; 4 epilogue warps (joined by the
//                 builders on a CTA's last tile) draw the new states (Eq. 3),
//                 update nu (Sec. 4.4) and copy improved states into the
//                 best-so-far.
// State (dense layout): x as FP8 +-1, chains x n_pad (the B operand of the
// gather); nu float and best x bytes in the same layout.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "dense_common.cuh"
#include "internal.h"
#include "philox.cuh"
#include "tc_ptx.cuh"

namespace rbmsat {

namespace {

constexpr int kBM = 128;   // TMEM lanes: clauses (GEMM1) or variables (GEMM2) per tile
constexpr int kBN = 256;   // chains per tile
constexpr int kBK1 = 128;  // GEMM1 K-block: 128 FP8
constexpr int kBK2 = 64;   // GEMM2 K-block: 64 16-bit elements
constexpr int kS1 = 3;     // GEMM1 ring stages (step mode)
constexpr int kS2 = 4;     // GEMM2 ring stages (at most)
constexpr int kStage1A = kBM * kBK1, kStage1B = kBN * kBK1;        // 16 KB, 32 KB
constexpr int kStage2A = kBM * kBK2 * 2, kStage2B = kBN * kBK2 * 2;  // 16 KB, 32 KB
constexpr int kEpi1 = 16;  // GEMM1 epilogue warps (4 per TMEM lane quarter)
constexpr int kBld = 16;   // GEMM2 builder warps (a chain and half a K-block per thread)
constexpr int kEpi2 = 4;   // GEMM2 epilogue warps (1 per lane quarter)
constexpr long long kWait = 4000000000LL;

__device__ __forceinline__ uint32_t step_index(const uint32_t* tdev, uint32_t t_rel) {
  return (tdev ? *tdev : 0u) + t_rel;
}

__host__ __device__ __forceinline__ int align16(int bytes) { return (bytes + 15) & ~15; }

__device__ __forceinline__ void stage16(void* dst, const void* src, int bytes, int tid, int nthr) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  for (int i = tid; i < bytes / 16; i += nthr) d[i] = __ldg(s + i);
}

// ---------------------------------------------------------------- GEMM1 step
struct G1Smem {
  uint64_t full[kS1];
  uint64_t empty[kS1];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint32_t tmem_slot;
  int64_t cost[2][4 * kBN];
  float fe[2][4 * kBN];
  int64_t w[kEpi1][32];
};

constexpr int kTabOff1 =
    (kS1 * (kStage1A + kStage1B) + (int)sizeof(G1Smem) + 127) / 128 * 128;

struct G1Args {
  int m, num_kb, tiles_m, tiles_n, B, Bp;
  uint32_t idesc;
  const int32_t* row_len;   // m_pad
  const int64_t* row_w;     // m_pad
  const int32_t* cl_grp;    // m
  const uint8_t* grp_same;  // m_pad / 32: rows of a 32-row group share one weight
  int64_t* cost_part;       // tiles_m x Bp
  float* fe_part;           // tiles_m x Bp
  void* H;                  // m x Bp hidden patterns
  const uint32_t* tdev;
  uint32_t t_rel;
  int* err;
};

template <bool SAMPLE, bool SM, typename HT, bool ONE>
__global__ void __launch_bounds__(64 + 32 * kEpi1, 1)
    k_gemm1_step(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const G1Args a, const DevTables T, const DevChains C) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint32_t base = (tc::smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t* ring = smem_raw + (base - tc::smem_u32(smem_raw));
  uint8_t* sA = ring;
  uint8_t* sB = ring + kS1 * kStage1A;
  G1Smem& S = *reinterpret_cast<G1Smem*>(ring + kS1 * (kStage1A + kStage1B));
  // staged tables start on a 128-byte boundary (16-byte vector stores)
  uint8_t* tabs = ring + kTabOff1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_tiles = a.tiles_m * a.tiles_n;

  // clause-RBM tables: staged in shared memory when small
  const GroupMeta* meta = T.meta;
  const uint32_t* rec = T.rec;
  if (SM) {
    const int mb = align16(T.n_groups * (int)sizeof(GroupMeta));
    stage16(tabs, T.meta, mb, threadIdx.x, blockDim.x);
    stage16(tabs + mb, T.rec, align16(T.rec_len * 4), threadIdx.x, blockDim.x);
    meta = reinterpret_cast<const GroupMeta*>(tabs);
    rec = reinterpret_cast<const uint32_t*>(tabs + mb);
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kS1; ++s) {
      tc::mbar_init(&S.full[s], 1);
      tc::mbar_init(&S.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&S.tfull[b], 1);
      tc::mbar_init(&S.tempty[b], kEpi1);
    }
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  if (warp == 1) {
    tc::tmem_alloc(&S.tmem_slot, 2 * kBN);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = S.tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
        const int tm = tile / a.tiles_n, tn = tile % a.tiles_n;
        for (int kb = 0; kb < a.num_kb; ++kb, ++g) {
          const int s = (int)(g % kS1);
          const uint32_t ph = (g / kS1) & 1u;
          ok = tc::mbar_wait(&S.empty[s], ph ^ 1u, a.err, 11, kWait);
          if (!ok) break;
          tc::mbar_arrive_expect_tx(&S.full[s], kStage1A + kStage1B);
          tc::tma_load_2d(sA + s * kStage1A, &tmA, &S.full[s], kb * kBK1, tm * kBM);
          tc::tma_load_2d(sB + s * kStage1B, &tmB, &S.full[s], kb * kBK1, tn * kBN);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      int li = 0;
      for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x, ++li) {
        const int buf = li & 1;
        ok = tc::mbar_wait(&S.tempty[buf], ((uint32_t)(li >> 1) & 1u) ^ 1u, a.err, 14, kWait);
        if (!ok) break;
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(buf * kBN);
        for (int kb = 0; kb < a.num_kb; ++kb, ++g) {
          const int s = (int)(g % kS1);
          const uint32_t ph = (g / kS1) & 1u;
          ok = tc::mbar_wait(&S.full[s], ph, a.err, 12, kWait);
          if (!ok) break;
          tc::fence_after_sync();
          const uint32_t a0 = tc::smem_u32(sA + s * kStage1A), b0 = tc::smem_u32(sB + s * kStage1B);
#pragma unroll
          for (int kk = 0; kk < kBK1 / 32; ++kk)
            tc::mma<true>(d, tc::sw128_desc(a0 + kk * 32), tc::sw128_desc(b0 + kk * 32), a.idesc,
                          (kb > 0 || kk > 0) ? 1u : 0u);
          tc::commit(&S.empty[s]);
        }
        tc::commit(&S.tfull[buf]);
      }
    }
    __syncwarp();
  } else {
    constexpr int kCols = kBN * 4 / kEpi1;  // 64 columns per epilogue warp
    const int quarter = warp & 3;
    const int ew = warp - 2;
    const int cgrp = ew / 4;
    const int t = threadIdx.x - 64;
    const int E = T.n_temps;
    uint32_t tround = 0;
    if (SAMPLE) tround = step_index(a.tdev, a.t_rel);
    int li = 0;
    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++li) {
      const int tm = tile / a.tiles_n, tn = tile % a.tiles_n;
      const int buf = li & 1;
      const int c = tm * kBM + quarter * 32 + lane;
      const int len = c < a.m ? __ldg(a.row_len + c) : 0;
      const int grp = c < a.m ? __ldg(a.cl_grp + c) : -1;
      const int64_t w = c < a.m ? __ldg(a.row_w + c) : 0;
      const int bias = (1 << len) - 1;
      const float unsat_d = -(float)bias;
      const bool same_w = __ldg(a.grp_same + tm * 4 + quarter) != 0;
      GroupMeta gm{};
      if (grp >= 0) gm = meta[grp];
      S.w[ew][lane] = w;
      __syncwarp();
      const bool ok = tc::mbar_wait(&S.tfull[buf], (uint32_t)(li >> 1) & 1u, a.err, 13, kWait);
      tc::fence_after_sync();
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) +
                             (uint32_t)(buf * kBN + cgrp * kCols);
      for (int j = 0; j < kCols / 32; ++j) {
        uint32_t r[32];
        tc::tmem_ld32(taddr + (uint32_t)(j * 32), r);
        tc::tmem_ld_wait();
        // weighted unsatisfied cost of the 32 columns over the warp's rows
        uint32_t unsat = 0;
#pragma unroll
        for (int q = 0; q < 32; ++q) unsat |= (uint32_t)(__uint_as_float(r[q]) == unsat_d) << q;
        if (!ok) unsat = 0;
        uint32_t rows = tc::transpose32(unsat, lane);
        int64_t col = 0;
        if (same_w) {
          col = (int64_t)__popc(rows) * S.w[ew][0];
        } else {
          while (rows) {
            col += S.w[ew][__ffs(rows) - 1];
            rows &= rows - 1;
          }
        }
        S.cost[buf][ew * kCols + j * 32 + lane] = col;
        // per 8 chains: free energy, hidden draws, hidden patterns
#pragma unroll
        for (int sub = 0; sub < 4; ++sub) {
          const int b0 = tn * kBN + cgrp * kCols + j * 32 + sub * 8;
          const int gb0 = C.g8_off * 8 + b0;  // global chain index
          const int e0 = temp_of(gb0, E, C.B_total, C.inv_B_total);
          const bool e_uni = e0 == temp_of(gb0 + 7, E, C.B_total, C.inv_B_total);
          int row[8];
          float f[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            // truth pattern; the mask keeps table rows in range even if the
            // accumulator is invalid after a timed-out wait
            const int p = ((__float2int_rn(__uint_as_float(r[sub * 8 + q])) + bias) >> 1) & bias;
            row[q] = ((e_uni ? e0 : temp_of(gb0 + q, E, C.B_total, C.inv_B_total)) << len) + p;
            f[q] = 0.f;
          }
          if (!SAMPLE && grp >= 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q) f[q] = __uint_as_float(rec[gm.rec_off + row[q] * gm.stride]);
          }
          if (SAMPLE && grp >= 0) {
            // free energy (record word 0) and hidden draws from the records
            const uint4* tab = reinterpret_cast<const uint4*>(rec + gm.rec_off);
            int row4[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) row4[q] = row[q] * (gm.stride >> 2);
            uint32_t hp[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) hp[q] = 0;
            const uint32_t octet = (uint32_t)(gb0 >> 3);
            const int chunks = gm.stride >> 2;
            if (!gm.sat)
              hidden_draws<false, ONE>(tab, row4, chunks, gm.nh, (uint32_t)c, octet, tround, kPhaseHidden,
                                        C.keys, hp, f);
            else
              hidden_draws<true, ONE>(tab, row4, chunks, gm.nh, (uint32_t)c, octet, tround, kPhaseHidden,
                                       C.keys, hp, f);
            HT* H = static_cast<HT*>(a.H) + (size_t)c * a.Bp + b0;
            if (sizeof(HT) == 1) {
              uint64_t v = 0;
#pragma unroll
              for (int q = 0; q < 8; ++q) v |= (uint64_t)hp[q] << (8 * q);
              *reinterpret_cast<uint64_t*>(H) = v;
            } else {
              *reinterpret_cast<uint4*>(H) = make_uint4(hp[0] | (hp[1] << 16), hp[2] | (hp[3] << 16),
                                                        hp[4] | (hp[5] << 16), hp[6] | (hp[7] << 16));
            }
          }
          const float fs = tc::column_sums8(f, lane);
          if (lane < 8) S.fe[buf][ew * kCols + j * 32 + sub * 8 + lane] = fs;
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&S.tempty[buf]);
      tc::epi_bar<32 * kEpi1>();
      for (int colx = t; colx < kBN; colx += 32 * kEpi1) {
        const int h = colx / kCols, cc = colx % kCols;
        int64_t cs = 0;
        float fsum = 0.f;
#pragma unroll
        for (int qd = 0; qd < 4; ++qd) {
          cs += S.cost[buf][(h * 4 + qd) * kCols + cc];
          fsum += S.fe[buf][(h * 4 + qd) * kCols + cc];
        }
        const size_t o = (size_t)tm * a.Bp + (size_t)tn * kBN + colx;
        a.cost_part[o] = cs;
        a.fe_part[o] = fsum;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 2 * kBN);
  }
}

// ---------------------------------------------------------------- keep
__global__ void k_keep_dense(const int64_t* __restrict__ cost_part, const float* __restrict__ fe_part,
                             int tiles_m, DevChains C) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= C.Bp) return;
  int64_t cs = 0;
  float fs = 0.f;
  int k = 0;
  // eight tiles' partials loaded ahead of their sums (the sums stay in tile order)
  for (; k + 8 <= tiles_m; k += 8) {
    int64_t cp[8];
    float fp[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      cp[j] = cost_part[(size_t)(k + j) * C.Bp + b];
      fp[j] = fe_part[(size_t)(k + j) * C.Bp + b];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      cs += cp[j];
      fs += fp[j];
    }
  }
  for (; k < tiles_m; ++k) {
    cs += cost_part[(size_t)k * C.Bp + b];
    fs += fe_part[(size_t)k * C.Bp + b];
  }
  C.cost[b] = cs;
  C.fe[b] = fs;
  const bool imp = cs < C.best[b];
  if (imp) C.best[b] = cs;
  C.improved[b] = imp ? 1 : 0;
}

// ---------------------------------------------------------------- GEMM2
struct G2Smem {
  uint64_t loaded[kS2];  // TMA / bulk copies -> builders: P^T, hidden rows, records
  uint64_t hready[kS2];  // builders' cp.async copies of the hidden patterns landed
  uint64_t built[kS2];   // builders -> MMA: G tile written
  uint64_t empty[kS2];   // MMA -> producer and builders: stage consumed
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint32_t tmem_slot;
};

// GEMM2 ring stage: P^T tile, the K-block's staged hidden patterns (64
// incidences x 256 chains) and its 64 incidence records. The G tiles the
// builders write alternate between two buffers after the ring: G of K-block g
// may be overwritten once the MMA of K-block g - 2 is done, which every
// builder knows once the records of K-block g + kStages - 2 have landed (the
// producer refilled that stage after the MMA of g - 2 released it).
template <typename HT>
struct G2Stage {
  static constexpr int kA = kStage2A;
  static constexpr int kH = kBK2 * kBN * (int)sizeof(HT);  // staged hidden patterns [u][chain]
  static constexpr int kInc = 1024;
  static constexpr int kBytes = kA + kH + kInc;  // multiple of 1024
  static constexpr int kStages = sizeof(HT) == 1 ? 4 : 3;
  static constexpr int kAhead = kStages - 2;  // K-blocks between a stage's copies and its build
  static constexpr int kB = kStage2B;
  static constexpr int kBOff = kStages * kBytes;
  static constexpr int kTabOff = (kBOff + 2 * kB + (int)sizeof(G2Smem) + 127) / 128 * 128;
};

struct G2Args {
  int n, n_pad, B, Bp, tiles_v, tiles_n;
  uint32_t idesc;
  const int32_t* kstart;   // tiles_v + 1: incidence range of each variable tile
  const int32_t* kblocks;  // tiles_v: K-blocks of each variable tile (>= 1)
  const int4* var_inc;     // incidences sorted by variable
  const uint16_t* gq16;    // contribution table as BF16 / FP16 bits (layout of T.gq)
  const void* H;           // m x Bp hidden patterns
  uint8_t* X;              // Bp x n_pad FP8 states
  float* nu;               // Bp x n_pad
  uint8_t* best_x;         // Bp x n_pad (0 / 1)
  uint8_t one, minus_one;  // FP8 encodings of +1 / -1
  bool bf16;               // G operand type (else FP16)
  float alpha;
  const uint32_t* tdev;
  uint32_t t_rel;
  int* err;
};


template <bool SM, typename HT>
__global__ void __launch_bounds__(64 + 32 * (kBld + kEpi2), 1)
    k_gemm2(const __grid_constant__ CUtensorMap tmA2, const G2Args a, const DevTables T,
            const DevChains C) {
  using St = G2Stage<HT>;
  constexpr int NS = St::kStages;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint32_t base = (tc::smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t* ring = smem_raw + (base - tc::smem_u32(smem_raw));
  G2Smem& S = *reinterpret_cast<G2Smem*>(ring + St::kBOff + 2 * St::kB);
  // staged tables start on a 128-byte boundary (16-byte vector stores)
  uint8_t* tabs = ring + St::kTabOff;
  auto stA = [&](int s) { return ring + s * St::kBytes; };
  auto stH = [&](int s) { return reinterpret_cast<HT*>(ring + s * St::kBytes + St::kA); };
  auto stI = [&](int s) {
    return reinterpret_cast<int4*>(ring + s * St::kBytes + St::kA + St::kH);
  };
  auto stB = [&](uint32_t g) { return ring + St::kBOff + (g & 1u) * St::kB; };  // G of K-block g

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_tiles = a.tiles_v * a.tiles_n;

  const uint16_t* gq = a.gq16;
  const uint32_t* pv = T.pv;
  if (SM) {
    const int gb = align16(T.gq_len * 4);  // both halves
    stage16(tabs, a.gq16, gb, threadIdx.x, blockDim.x);
    stage16(tabs + gb, T.pv, align16(T.pv_len * 4), threadIdx.x, blockDim.x);
    gq = reinterpret_cast<const uint16_t*>(tabs);
    pv = reinterpret_cast<const uint32_t*>(tabs + gb);
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(&S.loaded[s], 1);
      tc::mbar_init(&S.built[s], kBld);
      tc::mbar_init(&S.hready[s], 32 * kBld);
      tc::mbar_init(&S.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&S.tfull[b], 1);
      tc::mbar_init(&S.tempty[b], kEpi2);
    }
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmA2);
  }
  if (warp == 1) {
    tc::tmem_alloc(&S.tmem_slot, 2 * kBN);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = S.tmem_slot;

  // visible update (Eq. 3, nu of Sec. 4.4, best-keep copy) of 8 chains,
  // TMEM columns 8 c .. 8 c + 7 of accumulator buf, for the calling warp's
  // TMEM lane quarter (32 variables) of tile (tv, tn): the accumulators and
  // state loads first, then the draws and the stores
  auto visible8 = [&](int tv, int tn, int buf, int c) {
    const uint32_t tround = step_index(a.tdev, a.t_rel);
    const float keep = __fsub_rn(1.0f, a.alpha);  // the sparse path's exact FP32 operation sequence
    uint8_t* __restrict__ Xs = a.X;
    float* __restrict__ nus = a.nu;
    uint8_t* __restrict__ bxs = a.best_x;
    const uint8_t* __restrict__ impv = C.improved;
    const int quarter = warp & 3;
    const int i = tv * kBM + quarter * 32 + lane;
    const bool valid = i < a.n;
    const int b0 = tn * kBN + c * 8;
    uint32_t r[8];
    tc::tmem_ld8(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * kBN + c * 8), r);
    uint32_t xo[8];
    float nv[8];
    if (valid) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const size_t o = (size_t)(b0 + q) * a.n_pad + i;
        xo[q] = Xs[o];
        nv[q] = nus[o];
      }
    }
    const uint2 imp = *reinterpret_cast<const uint2*>(impv + b0);  // 8 flag bytes
    const uint4 R = philox4x32_10(
        make_uint4((uint32_t)i, (uint32_t)(C.g8_off + (b0 >> 3)), tround, kPhaseVisible), C.keys);
    tc::tmem_ld_wait();
    if (!valid) return;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int z = __float2int_rn(__uint_as_float(r[q]));
      const int qq = max(-T.qmax, min(T.qmax, z));
      const uint32_t P = pv[qq + T.qmax];
      const float var = __fmul_rn(__uint2float_rn(P * (65536u - P)), 2.3283064365386963e-10f);
      const size_t o = (size_t)(b0 + q) * a.n_pad + i;
      if (((q < 4 ? imp.x : imp.y) >> (8 * (q & 3))) & 0xFFu) bxs[o] = xo[q] == a.one ? 1 : 0;
      nus[o] = __fmaf_rn(keep, nv[q], __fmul_rn(a.alpha, var));
      Xs[o] = lane16(R, q) < P ? a.one : a.minus_one;
    }
  };
  constexpr int kShare = kEpi2 / 4 + kBld / 4;  // warps per lane quarter on a CTA's last tile

  if (warp == 0) {
    // producer warp: P^T tile by TMA and the K-block's incidence records by
    // one bulk copy
    uint32_t g = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
      const int tv = tile / a.tiles_n;
      const int k0 = __ldg(a.kstart + tv), k1 = __ldg(a.kstart + tv + 1);
      const int nkb = __ldg(a.kblocks + tv);
      for (int kb = 0; kb < nkb; ++kb, ++g) {
        const int s = (int)(g % NS);
        const uint32_t ph = (g / NS) & 1u;
        if (lane == 0) {
          ok = tc::mbar_wait(&S.empty[s], ph ^ 1u, a.err, 21, kWait);
          if (ok) {
            const int jj0 = k0 + kb * kBK2;
            const int nvalid = max(0, min(kBK2, k1 - jj0));
            tc::mbar_arrive_expect_tx(&S.loaded[s], (uint32_t)(St::kA + nvalid * 16));
            tc::tma_load_2d(stA(s), &tmA2, &S.loaded[s], kb * kBK2, tv * kBM);
            if (nvalid > 0)
              tc::bulk_load(stI(s), a.var_inc + jj0, (uint32_t)(nvalid * 16), &S.loaded[s]);
          }
        }
        ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
        if (!ok) break;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      int li = 0;
      for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x, ++li) {
        const int tv = tile / a.tiles_n;
        const int nkb = __ldg(a.kblocks + tv);
        const int buf = li & 1;
        ok = tc::mbar_wait(&S.tempty[buf], ((uint32_t)(li >> 1) & 1u) ^ 1u, a.err, 24, kWait);
        if (!ok) break;
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(buf * kBN);
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = (int)(g % NS);
          const uint32_t ph = (g / NS) & 1u;
          ok = tc::mbar_wait(&S.built[s], ph, a.err, 22, kWait);
          if (!ok) break;
          tc::fence_after_sync();
          const uint32_t a0 = tc::smem_u32(stA(s)), b0 = tc::smem_u32(stB(g));
#pragma unroll
          for (int kk = 0; kk < kBK2 / 16; ++kk)
            tc::mma<false>(d, tc::sw128_desc(a0 + kk * 32), tc::sw128_desc(b0 + kk * 32), a.idesc,
                           (kb > 0 || kk > 0) ? 1u : 0u);
          tc::commit(&S.empty[s]);
        }
        tc::commit(&S.tfull[buf]);
      }
    }
    __syncwarp();
  } else if (warp < 2 + kBld) {
    // builders. Copy phase: thread = 2 items (incidence u, 16 consecutive
    // chains), cp.async of their hidden-pattern bytes into the stage's staging
    // area kAhead K-blocks ahead. Build phase: thread = (4 consecutive chains,
    // 8 incidences): one record load and one load of the 4 staged patterns
    // per incidence, 4 table lookups, then one 16-byte chunk of the G tile
    // (row = chain, 128-byte swizzle) per chain.
    const int bt = threadIdx.x - 64;  // 0 .. 511
    const HT* H = static_cast<const HT*>(a.H);
    auto issue_copies = [&](int s, int jk0, int jk1, int ttn) {
      const int4* inc = stI(s);
      HT* hs = stH(s);
      const int cq = bt & 15, u0 = bt >> 4;
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const int u = u0 + 32 * it;
        if (jk0 + u < jk1) {
          const HT* src = H + (size_t)inc[u].x * a.Bp + (size_t)ttn * kBN + cq * 16;
#pragma unroll
          for (int v = 0; v < (int)sizeof(HT); ++v)
            tc::cp_async16(hs + u * kBN + cq * 16 + v * (16 / sizeof(HT)), src + v * (16 / sizeof(HT)));
        }
      }
      tc::cp_async_arrive(&S.hready[s]);
    };
    // two cursors over (tile, K-block) in the producer's order: copies (cc,
    // flat index gc) run kAhead K-blocks ahead of the build (cb, flat index g)
    struct Cursor {
      int tile, kb, tn, k0, k1, nkb;
    };
    auto enter_tile = [&](Cursor& c) {
      if (c.tile < num_tiles) {
        const int tv = c.tile / a.tiles_n;
        c.tn = c.tile % a.tiles_n;
        c.k0 = __ldg(a.kstart + tv);
        c.k1 = __ldg(a.kstart + tv + 1);
        c.nkb = __ldg(a.kblocks + tv);
      }
    };
    auto advance = [&](Cursor& c) {
      if (++c.kb >= c.nkb) {
        c.tile += gridDim.x;
        c.kb = 0;
        enter_tile(c);
      }
    };
    Cursor cb{(int)blockIdx.x, 0, 0, 0, 0, 0};
    enter_tile(cb);
    Cursor cc = cb;
    uint32_t gc = 0, g = 0;
    bool ok = true;
    auto wait_records = [&]() {
      ok = tc::mbar_wait(&S.loaded[gc % NS], (gc / NS) & 1u, a.err, 23, kWait);
    };
    auto copy_next = [&]() {
      issue_copies((int)(gc % NS), cc.k0 + cc.kb * kBK2, cc.k1, cc.tn);
      advance(cc);
      ++gc;
    };
    for (int d = 0; d < St::kAhead && ok && cc.tile < num_tiles; ++d) {
      wait_records();
      if (ok) copy_next();
    }
    const int quad = bt & (kBN / 4 - 1);  // chains 4 quad .. 4 quad + 3
    const int chunk = bt / (kBN / 4);     // incidences 8 chunk .. 8 chunk + 7
    // slot r of a thread holds chain 4 quad + off[r]: the rotation by quad / 2
    // gives the 8 lanes of each store phase 8 different 16-byte bank groups
    int off[4];
    uint32_t sel[4];  // byte permutation that moves slot r's pattern to the low bits
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      off[r] = (r + (quad >> 1)) & 3;
      sel[r] = sizeof(HT) == 1 ? 0x4440u | (uint32_t)off[r] : 0x10u + 0x22u * (uint32_t)off[r];
    }
    while (ok && cb.tile < num_tiles) {
      // the copies of K-block g + kAhead are issued after this build's proxy
      // fence, so that the fence does not wait for them to land
      const bool more = cc.tile < num_tiles;
      if (more) {
        wait_records();
        if (!ok) break;
      } else if (g >= 2) {
        // no copies left to order it: wait for the MMA that last read this
        // G buffer (K-block g - 2)
        ok = tc::mbar_wait(&S.empty[(g - 2) % NS], ((g - 2) / NS) & 1u, a.err, 27, kWait);
        if (!ok) break;
      }
      // build the current K-block once every builder's copies have landed
      const int s = (int)(g % NS);
      ok = tc::mbar_wait(&S.hready[s], (g / NS) & 1u, a.err, 26, kWait);
      if (!ok) break;
      {
        const int jj0 = cb.k0 + cb.kb * kBK2, k1 = cb.k1;
        const int4* inc = stI(s);
        const HT* hs = stH(s) + 4 * quad;
        uint8_t* gt = stB(g);
        int e[4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
          e[r] = temp_of(C.g8_off * 8 + cb.tn * kBN + 4 * quad + off[r], T.n_temps, C.B_total,
                         C.inv_B_total);
        // the quad's chains of one temperature (all but at most E - 1 quads)
        const bool same_e = e[1] == e[0] && e[2] == e[0] && e[3] == e[0];
        const char* gqc = reinterpret_cast<const char*>(gq);
        uint32_t pk[4][4];
        // FULL: all 64 incidences of the K-block exist (every K-block but a
        // tile's last), so that the loads of different incidences carry no
        // branch between them and overlap. UNI: one temperature, so one table
        // row per incidence serves the four chains.
        auto lookups = [&](auto full, auto uni) {
#pragma unroll
          for (int u2 = 0; u2 < 4; ++u2) {
            uint32_t v0[4] = {0u, 0u, 0u, 0u}, v1[4] = {0u, 0u, 0u, 0u};  // 0 = +0.0
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
              const int u = chunk * 8 + u2 * 2 + hf;
              if (decltype(full)::value || jj0 + u < k1) {
                const int4 m = inc[u];
                const int b = m.y & 0x7FFFFFFF;
                const int z2 = 2 * m.z;  // bytes between hidden patterns
                uint32_t hw0, hw1 = 0;   // the 4 chains' hidden patterns
                if constexpr (sizeof(HT) == 1) {
                  hw0 = *reinterpret_cast<const uint32_t*>(hs + u * kBN);
                } else {
                  const uint2 t2 = *reinterpret_cast<const uint2*>(hs + u * kBN);
                  hw0 = t2.x;
                  hw1 = t2.y;
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                  uint32_t hp;
                  if constexpr (sizeof(HT) == 1)
                    hp = __byte_perm(hw0, 0u, sel[r]);
                  else
                    hp = __byte_perm(hw0, hw1, sel[r]) & 0xFFFFu;
                  const int row = decltype(uni)::value ? b + e[0] * m.w : b + e[r] * m.w;
                  const uint32_t v =
                      *reinterpret_cast<const uint16_t*>(gqc + 2 * row + (int)hp * z2);
                  if (hf == 0)
                    v0[r] = v;
                  else
                    v1[r] = v;
                }
              }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) pk[r][u2] = __byte_perm(v0[r], v1[r], 0x5410u);
          }
        };
        if (same_e) {
          if (jj0 + kBK2 <= k1)
            lookups(std::true_type{}, std::true_type{});
          else
            lookups(std::false_type{}, std::true_type{});
        } else {
          if (jj0 + kBK2 <= k1)
            lookups(std::true_type{}, std::false_type{});
          else
            lookups(std::false_type{}, std::false_type{});
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int chain = 4 * quad + off[r];
          *reinterpret_cast<uint4*>(gt + chain * 128 + ((chunk ^ (chain & 7)) << 4)) =
              make_uint4(pk[r][0], pk[r][1], pk[r][2], pk[r][3]);
        }
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&S.built[s]);
      }
      if (more) copy_next();
      ++g;
      advance(cb);
    }
    // the visible update of the CTA's last tile, shared with the epilogue
    // warps (worker kEpi2 / 4 + index among the quarter's builder warps)
    if (ok && (int)blockIdx.x < num_tiles) {
      const int nt = (num_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x;  // its local index
      const int lt = (int)blockIdx.x + nt * (int)gridDim.x;
      tc::mbar_wait(&S.tfull[nt & 1], (uint32_t)(nt >> 1) & 1u, a.err, 28, kWait);
      tc::fence_after_sync();
#pragma unroll 1
      for (int c = kEpi2 / 4 + (warp - 2) / 4; c < kBN / 8; c += kShare)
        visible8(lt / a.tiles_n, lt % a.tiles_n, nt & 1, c);
    }
  } else {
    // epilogue: row = variable. A tile's 32 groups of 8 chains go to the
    // epilogue warps of each lane quarter; the CTA's last tile is shared with
    // the builder warps, idle by then (kShare warps per quarter)
    const int ew = warp - 2 - kBld;  // 0 .. kEpi2 - 1
    const int cgrp = ew / 4;
    int li = 0;
    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++li) {
      const int tv = tile / a.tiles_n, tn = tile % a.tiles_n;
      const int buf = li & 1;
      {
        // the tile's state rows into L2 while its mainloop runs: thread =
        // one chain, its 128 variables (one line of x, four of nu; n_pad is
        // a multiple of 128)
        for (int ch = ew * 32 + lane; ch < kBN; ch += kEpi2 * 32) {
          const size_t row = (size_t)(tn * kBN + ch) * a.n_pad + (size_t)tv * kBM;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(a.X + row));
#pragma unroll
          for (int q = 0; q < 4; ++q)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.nu + row + 32 * q));
        }
      }
      tc::mbar_wait(&S.tfull[buf], (uint32_t)(li >> 1) & 1u, a.err, 25, kWait);
      tc::fence_after_sync();
      if (tile + (int)gridDim.x < num_tiles) {
#pragma unroll 1
        for (int c = cgrp; c < kBN / 8; c += kEpi2 / 4) visible8(tv, tn, buf, c);
      } else {
#pragma unroll 1
        for (int c = cgrp; c < kBN / 8; c += kShare) visible8(tv, tn, buf, c);
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&S.tempty[buf]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 2 * kBN);
  }
}

// ---------------------------------------------------------------- state
__global__ void k_init_dense(DevChains C, uint8_t* X, float* nu, uint8_t* best_x, int n,
                             int n_pad, uint8_t one, uint8_t minus_one) {
  const int g8 = blockIdx.x, b0 = g8 * 8;
  const int i = blockIdx.y * blockDim.x + threadIdx.x;
  if (i < n_pad) {
    uint4 r = make_uint4(0, 0, 0, 0);
    if (i < n)
      r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(g8 + C.g8_off), 0u, kPhaseInit), C.keys);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const size_t o = (size_t)(b0 + q) * n_pad + i;
      const bool bit = lane16(r, q) < 32768u;
      X[o] = i < n ? (bit ? one : minus_one) : 0;
      nu[o] = i < n ? 0.25f : 0.f;
      best_x[o] = i < n && bit ? 1 : 0;
    }
  }
  if (blockIdx.y == 0 && threadIdx.x < 8) {
    C.best[b0 + threadIdx.x] = INT64_MAX;
    C.improved[b0 + threadIdx.x] = 0;
  }
}

__global__ void k_keep_copy_dense(const DevChains C, const uint8_t* X, uint8_t* best_x, int n,
                                  int n_pad, uint8_t one) {
  const int b = blockIdx.y;
  if (!C.improved[b]) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const size_t o = (size_t)b * n_pad + i;
    best_x[o] = X[o] == one ? 1 : 0;
  }
}

template <bool SAMPLE, bool SM, typename HT>
cudaError_t g1_variant(int grid, int smem, cudaStream_t st, const CUtensorMap& tmA,
                       const CUtensorMap& tmB, const G1Args& a, const DevTables& T,
                       const DevChains& C) {
  // one-chunk records (L <= 3 everywhere): the sampling has no chunk loop
  auto kern = k_gemm1_step<SAMPLE, SM, HT, false>;
  if constexpr (SAMPLE && sizeof(HT) == 1)
    if (T.one_chunk) kern = k_gemm1_step<SAMPLE, SM, HT, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, 64 + 32 * kEpi1, smem, st>>>(tmA, tmB, a, T, C);
  return cudaGetLastError();
}

template <bool SM, typename HT>
cudaError_t g2_variant(int grid, int smem, cudaStream_t st, const CUtensorMap& tmA2,
                       const G2Args& a, const DevTables& T, const DevChains& C) {
  auto kern = k_gemm2<SM, HT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, 64 + 32 * (kBld + kEpi2), smem, st>>>(tmA2, a, T, C);
  return cudaGetLastError();
}

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 1;
  }
  return sms;
}

constexpr int kSmemMax = 227 * 1024;

}  // namespace

int dense_g1_table_bytes(const DevTables& T) {
  return align16(T.n_groups * (int)sizeof(GroupMeta)) + align16(T.rec_len * 4);
}

cudaError_t launch_gemm1_step(bool sample, const CUtensorMap& tmA, const CUtensorMap& tmB, int m,
                              int m_pad, int n_pad, int B, int Bp, bool e5m2,
                              const int32_t* row_len, const int64_t* row_w, const int32_t* cl_grp,
                              const uint8_t* grp_same, int64_t* cost_part, float* fe_part, void* H,
                              bool wide, const uint32_t* tdev, uint32_t t_rel, int* err,
                              const DevTables& T, const DevChains& C, cudaStream_t st) {
  G1Args a;
  a.m = m;
  a.num_kb = n_pad / kBK1;
  a.tiles_m = m_pad / kBM;
  a.tiles_n = Bp / kBN;
  a.B = B;
  a.Bp = Bp;
  const uint32_t fmt = e5m2 ? 1u : 0u;
  a.idesc = tc::instr_desc(kBM, kBN, fmt, fmt);
  a.row_len = row_len;
  a.row_w = row_w;
  a.cl_grp = cl_grp;
  a.grp_same = grp_same;
  a.cost_part = cost_part;
  a.fe_part = fe_part;
  a.H = H;
  a.tdev = tdev;
  a.t_rel = t_rel;
  a.err = err;
  const int base_smem = 1024 + kTabOff1;
  const int tb = dense_g1_table_bytes(T);
  const bool sm = base_smem + tb <= kSmemMax;
  const int smem = base_smem + (sm ? tb : 0);
  const int grid = std::min(sm_count(), a.tiles_m * a.tiles_n);
  if (sample) {
    if (sm) return wide ? g1_variant<true, true, uint16_t>(grid, smem, st, tmA, tmB, a, T, C)
                        : g1_variant<true, true, uint8_t>(grid, smem, st, tmA, tmB, a, T, C);
    return wide ? g1_variant<true, false, uint16_t>(grid, smem, st, tmA, tmB, a, T, C)
                : g1_variant<true, false, uint8_t>(grid, smem, st, tmA, tmB, a, T, C);
  }
  if (sm) return g1_variant<false, true, uint8_t>(grid, smem, st, tmA, tmB, a, T, C);
  return g1_variant<false, false, uint8_t>(grid, smem, st, tmA, tmB, a, T, C);
}

cudaError_t launch_keep_dense(const int64_t* cost_part, const float* fe_part, int tiles_m,
                              const DevChains& C, cudaStream_t st) {
  k_keep_dense<<<(C.Bp + 63) / 64, 64, 0, st>>>(cost_part, fe_part, tiles_m, C);
  return cudaGetLastError();
}

cudaError_t launch_gemm2(const CUtensorMap& tmA2, int n, int n_pad, int B, int Bp, int tiles_v,
                         const int32_t* kstart, const int32_t* kblocks, const int4* var_inc,
                         const uint16_t* gq16, const void* H, bool wide, uint8_t* X, float* nu,
                         uint8_t* best_x,
                         bool e5m2, bool bf16, float alpha, const uint32_t* tdev, uint32_t t_rel,
                         int* err, const DevTables& T, const DevChains& C, cudaStream_t st) {
  G2Args a;
  a.n = n;
  a.n_pad = n_pad;
  a.B = B;
  a.Bp = Bp;
  a.tiles_v = tiles_v;
  a.tiles_n = Bp / kBN;
  const uint32_t fmt = bf16 ? 1u : 0u;
  a.idesc = tc::instr_desc(kBM, kBN, fmt, fmt);
  a.kstart = kstart;
  a.kblocks = kblocks;
  a.var_inc = var_inc;
  a.gq16 = gq16;
  a.H = H;
  a.X = X;
  a.nu = nu;
  a.best_x = best_x;
  fp8_encode_int(1, e5m2, &a.one);
  fp8_encode_int(-1, e5m2, &a.minus_one);
  a.bf16 = bf16;
  a.alpha = alpha;
  a.tdev = tdev;
  a.t_rel = t_rel;
  a.err = err;
  const int tb = align16(T.gq_len * 4) + align16(T.pv_len * 4);
  const int grid = std::min(sm_count(), a.tiles_v * a.tiles_n);
  if (wide) {
    const int base_smem = 1024 + G2Stage<uint16_t>::kTabOff;
    const bool sm = base_smem + tb <= kSmemMax;
    return sm ? g2_variant<true, uint16_t>(grid, base_smem + tb, st, tmA2, a, T, C)
              : g2_variant<false, uint16_t>(grid, base_smem, st, tmA2, a, T, C);
  }
  const int base_smem = 1024 + G2Stage<uint8_t>::kTabOff;
  const bool sm = base_smem + tb <= kSmemMax;
  return sm ? g2_variant<true, uint8_t>(grid, base_smem + tb, st, tmA2, a, T, C)
            : g2_variant<false, uint8_t>(grid, base_smem, st, tmA2, a, T, C);
}

cudaError_t launch_init_dense(const DevChains& C, uint8_t* X, float* nu, uint8_t* best_x, int n,
                              int n_pad, bool e5m2, cudaStream_t st) {
  uint8_t one, minus_one;
  fp8_encode_int(1, e5m2, &one);
  fp8_encode_int(-1, e5m2, &minus_one);
  dim3 grid(C.Bp / 8, (n_pad + 127) / 128);
  k_init_dense<<<grid, 128, 0, st>>>(C, X, nu, best_x, n, n_pad, one, minus_one);
  return cudaGetLastError();
}

cudaError_t launch_keep_copy_dense(const DevChains& C, const uint8_t* X, uint8_t* best_x, int n,
                                   int n_pad, bool e5m2, cudaStream_t st) {
  uint8_t one;
  fp8_encode_int(1, e5m2, &one);
  dim3 grid((n + 255) / 256, C.Bp);
  k_keep_copy_dense<<<grid, 256, 0, st>>>(C, X, best_x, n, n_pad, one);
  return cudaGetLastError();
}

}  // namespace rbmsat
