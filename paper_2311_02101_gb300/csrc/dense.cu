// Dense tensor-core path: the clause gather of a Gibbs round as one FP8
// matrix product on the 5th-generation tensor cores.
//
// The paper evaluates clause inputs with a one-hot batched matrix product on
// the TPU's matrix unit (Sec. 4.3, "gather ... via batched matrix
// multiplication"). Here clause c's row of the m x n operand A holds
// lambda_ck 2^k at the variable of its k-th literal (lambda = +1 / -1 for a
// plain / negated literal). With the chain states as s = +1 / -1 (B operand,
// chains x variables), the product is
//   D_cb = sum_k 2^k lambda_ck s_{t_ck, b} = 2 p_cb - (2^K_c - 1),
// where p_cb = sum_k tau_ck(b) 2^k is the truth pattern of the clause's
// literals (tau = 1 when the literal is true). One MMA therefore yields the
// whole pattern: its count of true literals, satisfaction (p != 0) and the
// table row of the clause RBM. Entries are small signed sums of powers of two,
// exact in FP8 (E4M3 up to length 9, E5M2 beyond); the FP32 accumulator is
// exact for |D| < 2^24.
//
// Kernel structure (one 128-clause x 128-chain tile per CTA, 6 warps):
//   warp 0     TMA producer: 128-byte-swizzled K-blocks of A and B into a
//              4-stage shared-memory ring (mbarrier complete_tx);
//   warp 1     allocates 128 TMEM columns and issues tcgen05.mma
//              (kind::f8f6f4, M = 128, N = 128, K = 32) from one thread;
//              tcgen05.commit frees ring slots and signals the accumulator;
//   warps 2-5  epilogue: tcgen05.ld 32 columns at a time (one row = one
//              clause per thread), decode patterns, reduce weighted costs per
//              chain across the 128 rows, and (last tile of a chain column to
//              arrive) sum the per-tile partials in tile order.
// Every mbarrier wait is bounded; a timeout records an error code that the
// host reads after the launch, and the kernel still releases its TMEM.
#include <cuda.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace rbmsat {

namespace {

constexpr int kBM = 128;          // clauses per tile
constexpr int kBN = 128;          // chains per tile
constexpr int kBK = 128;          // FP8 elements (bytes) per K-block: one 128-byte swizzle row
constexpr int kStages = 4;
constexpr int kStageA = kBM * kBK;  // 16 KB
constexpr int kStageB = kBN * kBK;  // 16 KB
constexpr int kThreads = 192;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

struct Gemm1Smem {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t accum;
  uint32_t tmem_slot;
  int last;
  int64_t cost[4][kBN];
};

constexpr int kGemm1Smem = 1024 + kStages * (kStageA + kStageB) + (int)sizeof(Gemm1Smem);

__device__ __forceinline__ void epi_bar() {
  asm volatile("bar.sync 1, 128;" ::: "memory");
}

// EVAL: weighted unsatisfied cost per chain.
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm1_eval(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 int m, int num_kb, int B, int Bp, uint32_t idesc, const int32_t* __restrict__ row_len,
                 const int64_t* __restrict__ row_w, int64_t* __restrict__ part,
                 int32_t* __restrict__ tickets, int64_t* __restrict__ out, int* err) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint32_t base = (tc::smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t* tiles = smem_raw + (base - tc::smem_u32(smem_raw));
  uint8_t* sA = tiles;
  uint8_t* sB = tiles + kStages * kStageA;
  Gemm1Smem& S = *reinterpret_cast<Gemm1Smem*>(tiles + kStages * (kStageA + kStageB));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile_n = blockIdx.x, tile_m = blockIdx.y;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&S.full[s], 1);
      tc::mbar_init(&S.empty[s], 1);
    }
    tc::mbar_init(&S.accum, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  if (warp == 1) {
    tc::tmem_alloc(&S.tmem_slot, kBN);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = S.tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      for (int kb = 0; kb < num_kb; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
        if (!tc::mbar_wait(&S.empty[s], ph ^ 1u, err, 1, kWaitCycles)) break;
        tc::mbar_arrive_expect_tx(&S.full[s], kStageA + kStageB);
        tc::tma_load_2d(sA + s * kStageA, &tmA, &S.full[s], kb * kBK, tile_m * kBM);
        tc::tma_load_2d(sB + s * kStageB, &tmB, &S.full[s], kb * kBK, tile_n * kBN);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int kb = 0; kb < num_kb && ok; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
        ok = tc::mbar_wait(&S.full[s], ph, err, 2, kWaitCycles);
        if (!ok) break;
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(sA + s * kStageA), b0 = tc::smem_u32(sB + s * kStageB);
#pragma unroll
        for (int kk = 0; kk < kBK / 32; ++kk)
          tc::mma<true>(tmem, tc::sw128_desc(a0 + kk * 32), tc::sw128_desc(b0 + kk * 32), idesc,
                        (kb > 0 || kk > 0) ? 1u : 0u);
        tc::commit(&S.empty[s]);
      }
      tc::commit(&S.accum);
    }
    __syncwarp();
  } else {
    // epilogue warps 2..5: TMEM lane quarter = warp % 4
    const int quarter = warp & 3;
    const int ew = warp - 2;
    const int row = quarter * 32 + lane;
    const int c = tile_m * kBM + row;
    const int len = c < m ? __ldg(row_len + c) : 0;
    const int64_t w = c < m ? __ldg(row_w + c) : 0;
    const int bias = (1 << len) - 1;
    const uint32_t wlo = (uint32_t)(w & 0xFFFF), whi = (uint32_t)(w >> 16);
    const bool ok = tc::mbar_wait(&S.accum, 0, err, 3, kWaitCycles);
    tc::fence_after_sync();
    for (int j = 0; j < kBN / 32; ++j) {
      uint32_t r[32];
      tc::tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(j * 32), r);
      tc::tmem_ld_wait();
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int d = __float2int_rn(__uint_as_float(r[q]));
        const bool unsat = ok && ((d + bias) >> 1) == 0;
        const uint32_t lo = __reduce_add_sync(0xFFFFFFFFu, unsat ? wlo : 0u);
        const uint32_t hi = __reduce_add_sync(0xFFFFFFFFu, unsat ? whi : 0u);
        if (lane == 0) S.cost[ew][j * 32 + q] = (int64_t)lo + ((int64_t)hi << 16);
      }
    }
    tc::fence_before_sync();
    epi_bar();
    const int t = threadIdx.x - 64;  // 0..127
    const int64_t csum = S.cost[0][t] + S.cost[1][t] + S.cost[2][t] + S.cost[3][t];
    part[(size_t)tile_m * Bp + (size_t)tile_n * kBN + t] = csum;
    __threadfence();
    epi_bar();
    if (t == 0) S.last = atomicAdd(tickets + tile_n, 1) == (int)gridDim.y - 1;
    epi_bar();
    if (S.last) {
      __threadfence();
      const int b = tile_n * kBN + t;
      int64_t tot = 0;
      for (int k = 0; k < (int)gridDim.y; ++k) tot += __ldcg(part + (size_t)k * Bp + b);
      if (b < B) out[b] = tot;
      if (t == 0) tickets[tile_n] = 0;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kBN);
  }
}

// assign (B x n bytes, nonzero = true) -> X (Bp x n_pad FP8): +1 / -1 for
// variables, 0 for padding variables and padding chains.
__global__ void k_assign_fp8(const uint8_t* __restrict__ assign, int B, int n, int Bp, int n_pad,
                             uint8_t one, uint8_t minus_one, uint8_t* __restrict__ X) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)Bp * n_pad) return;
  const int b = (int)(idx / n_pad), i = (int)(idx % n_pad);
  uint8_t v = 0;
  if (b < B && i < n) v = assign[(size_t)b * n + i] ? one : minus_one;
  X[idx] = v;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

}  // namespace

// Exact FP8 encoding of a small integer, or false when it is not
// representable. E4M3: 4 exponent bits (bias 7), 3 mantissa bits, largest
// finite 448; E5M2: 5 exponent bits (bias 15), 2 mantissa bits.
bool fp8_encode_int(int v, bool e5m2, uint8_t* out) {
  if (v == 0) {
    *out = 0;
    return true;
  }
  const uint8_t sign = v < 0 ? 0x80 : 0;
  unsigned a = (unsigned)(v < 0 ? -v : v);
  int k = 31 - __builtin_clz(a);
  const int mbits = e5m2 ? 2 : 3;
  if (k > mbits && (a & ((1u << (k - mbits)) - 1u)) != 0) return false;
  const unsigned frac = k >= mbits ? (a >> (k - mbits)) & ((1u << mbits) - 1u)
                                   : (a << (mbits - k)) & ((1u << mbits) - 1u);
  if (e5m2) {
    if (k > 15) return false;
    *out = sign | (uint8_t)((k + 15) << 2) | (uint8_t)frac;
  } else {
    if (k > 8 || (k == 8 && frac > 6)) return false;
    *out = sign | (uint8_t)((k + 7) << 3) | (uint8_t)frac;
  }
  return true;
}

std::string make_tmap_2d(CUtensorMap* tm, const void* base, uint64_t inner, uint64_t rows,
                         uint64_t row_bytes, uint32_t box_inner, uint32_t box_rows, bool bf16) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return "cuTensorMapEncodeTiled is not available";
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
  return "";
}

std::string build_gather_matrix(int n, int m, const int64_t* off, const int32_t* lits,
                                bool* e5m2, int* n_pad, int* m_pad, std::vector<uint8_t>* A) {
  int maxlen = 0;
  for (int c = 0; c < m; ++c) maxlen = std::max(maxlen, (int)(off[c + 1] - off[c]));
  *e5m2 = maxlen > 9;
  *n_pad = (n + kBK - 1) / kBK * kBK;
  *m_pad = std::max(kBM, (m + kBM - 1) / kBM * kBM);
  A->assign((size_t)(*m_pad) * (*n_pad), 0);
  std::vector<int> acc;
  for (int c = 0; c < m; ++c) {
    const int len = (int)(off[c + 1] - off[c]);
    // sum of lambda 2^k per variable of the clause
    for (int k = 0; k < len; ++k) {
      const int32_t l = lits[off[c] + k];
      const int v = (l > 0 ? l : -l) - 1;
      int sum = 0;
      bool first = true;
      for (int k2 = 0; k2 < len; ++k2) {
        const int32_t l2 = lits[off[c] + k2];
        if ((l2 > 0 ? l2 : -l2) - 1 != v) continue;
        if (k2 < k) first = false;
        sum += (l2 > 0 ? 1 : -1) * (1 << k2);
      }
      if (!first) continue;
      uint8_t byte;
      if (!fp8_encode_int(sum, *e5m2, &byte))
        return "clause " + std::to_string(c) + " has a repeated variable whose coefficient " +
               std::to_string(sum) + " is not exact in FP8";
      (*A)[(size_t)c * (*n_pad) + v] = byte;
    }
  }
  return "";
}

cudaError_t launch_gemm1_eval(const CUtensorMap& tmA, const CUtensorMap& tmB, int m, int m_pad,
                              int n_pad, int B, int Bp, bool e5m2, const int32_t* row_len,
                              const int64_t* row_w, int64_t* part, int32_t* tickets,
                              int64_t* out, int* err, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm1_eval, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kGemm1Smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const uint32_t fmt = e5m2 ? 1u : 0u;
  const uint32_t idesc = tc::instr_desc(kBM, kBN, fmt, fmt);
  dim3 grid(Bp / kBN, m_pad / kBM);
  k_gemm1_eval<<<grid, kThreads, kGemm1Smem, st>>>(tmA, tmB, m, n_pad / kBK, B, Bp, idesc, row_len,
                                                   row_w, part, tickets, out, err);
  return cudaGetLastError();
}

cudaError_t launch_assign_fp8(const uint8_t* assign, int B, int n, int Bp, int n_pad, bool e5m2,
                              uint8_t* X, cudaStream_t st) {
  uint8_t one, minus_one;
  fp8_encode_int(1, e5m2, &one);
  fp8_encode_int(-1, e5m2, &minus_one);
  const size_t total = (size_t)Bp * n_pad;
  k_assign_fp8<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(assign, B, n, Bp, n_pad, one,
                                                                 minus_one, X);
  return cudaGetLastError();
}

}  // namespace rbmsat
