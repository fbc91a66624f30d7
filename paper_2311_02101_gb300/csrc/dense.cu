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
// Kernel structure (persistent: one CTA per SM walks 128-clause x 256-chain
// tiles, chain tile fastest; 18 warps):
//   warp 0     TMA producer: 128-byte-swizzled K-blocks of A and B into a
//              4-stage shared-memory ring (mbarrier complete_tx);
//   warp 1     allocates 2 x 256 TMEM columns (two accumulators, so the
//              epilogue of one tile overlaps the MMAs of the next) and issues
//              tcgen05.mma (kind::f8f6f4, M = 128, N = 256, K = 32) from one
//              thread; tcgen05.commit frees ring slots and signals the
//              accumulator;
//   warps 2-17 epilogue, four warps per TMEM lane quarter (one row = one
//              clause per thread, 64 columns per warp): tcgen05.ld 32 columns
//              at a time, test each entry against the all-false value, a
//              32 x 32 bit transpose turns rows into columns, the weighted
//              unsatisfied cost of every chain is summed over the tile's 128
//              rows and added to the chain's cost with a 64-bit atomic
//              (integers: exact in any order).
// An evaluation is two launches: k_assign_fp8 converts the assignments to
// the FP8 B operand and zeroes the costs; k_gemm1_eval is its programmatic
// dependent, so its setup (barriers, TMEM, tensor-map prefetch) overlaps the
// conversion and it waits (griddepcontrol.wait) only before touching them.
// Consecutive evaluations alternate between two state buffers, and each
// product lets the next conversion start at once: that conversion runs beside
// the product and waits for its end only before it zeroes the costs.
// Every mbarrier wait is bounded; a timeout records an error code that the
// host reads after the launch, and the kernel still releases its TMEM.
#include <cuda.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"
#include "dense_common.cuh"

namespace rbmsat {

namespace {

constexpr int kBM = 128;          // clauses per tile (TMEM lanes)
constexpr int kBN = 256;          // chains per tile (TMEM columns per accumulator)
constexpr int kBK = 128;          // FP8 elements (bytes) per K-block: one 128-byte swizzle row
constexpr int kStages = 4;
constexpr int kStageA = kBM * kBK;  // 16 KB
constexpr int kStageB = kBN * kBK;  // 32 KB
constexpr int kEpiWarps = 16;  // epilogue warps (four per TMEM lane quarter)
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

struct Gemm1Smem {
  uint64_t full[kStages];   // TMA -> MMA: stage loaded
  uint64_t empty[kStages];  // MMA -> TMA: stage consumed
  uint64_t tfull[2];        // MMA -> epilogue: accumulator buffer ready
  uint64_t tempty[2];       // epilogue -> MMA: accumulator buffer drained
  uint32_t tmem_slot;
  int64_t cost[2][4 * kBN];  // per tile parity and epilogue warp: its rows' column sums
  int64_t w[kEpiWarps][32];  // per epilogue warp: the weights of its 32 rows
};

constexpr int kGemm1Smem = 1024 + kStages * (kStageA + kStageB) + (int)sizeof(Gemm1Smem);

// Persistent gather GEMM: each CTA walks the tiles blockIdx.x, blockIdx.x +
// gridDim.x, ... (chain tile fastest). EVAL epilogue: weighted unsatisfied
// cost per chain. Two TMEM accumulators (2 x 256 columns) let the epilogue of
// one tile overlap the MMAs of the next.
template <int EPI>
__global__ void __launch_bounds__(64 + 32 * EPI, 1)
    k_gemm1_eval(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 int m, int num_kb, int tiles_m, int tiles_n, int B, int Bp, uint32_t idesc,
                 const int32_t* __restrict__ row_len, const int64_t* __restrict__ row_w,
                 const uint8_t* __restrict__ grp_small, int64_t* __restrict__ out, int* err) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint32_t base = (tc::smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t* tiles = smem_raw + (base - tc::smem_u32(smem_raw));
  uint8_t* sA = tiles;
  uint8_t* sB = tiles + kStages * kStageA;
  Gemm1Smem& S = *reinterpret_cast<Gemm1Smem*>(tiles + kStages * (kStageA + kStageB));

  static_assert(EPI == 4 || EPI == 8 || EPI == 16, "4, 8 or 16 epilogue warps");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_tiles = tiles_m * tiles_n;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&S.full[s], 1);
      tc::mbar_init(&S.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&S.tfull[b], 1);
      tc::mbar_init(&S.tempty[b], EPI);
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
  // the B operand and the zeroed costs come from the preceding conversion
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the next evaluation's conversion (into the other state buffer) may start
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  if (warp == 0) {
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
        const int tm = tile / tiles_n, tn = tile % tiles_n;
        for (int kb = 0; kb < num_kb; ++kb, ++g) {
          const int s = (int)(g % kStages);
          const uint32_t ph = (g / kStages) & 1u;
          ok = tc::mbar_wait(&S.empty[s], ph ^ 1u, err, 1, kWaitCycles);
          if (!ok) break;
          tc::mbar_arrive_expect_tx(&S.full[s], kStageA + kStageB);
          tc::tma_load_2d(sA + s * kStageA, &tmA, &S.full[s], kb * kBK, tm * kBM);
          tc::tma_load_2d(sB + s * kStageB, &tmB, &S.full[s], kb * kBK, tn * kBN);
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
        const uint32_t use = (uint32_t)(li >> 1);
        ok = tc::mbar_wait(&S.tempty[buf], (use & 1u) ^ 1u, err, 4, kWaitCycles);
        if (!ok) break;
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(buf * kBN);
        for (int kb = 0; kb < num_kb; ++kb, ++g) {
          const int s = (int)(g % kStages);
          const uint32_t ph = (g / kStages) & 1u;
          ok = tc::mbar_wait(&S.full[s], ph, err, 2, kWaitCycles);
          if (!ok) break;
          tc::fence_after_sync();
          const uint32_t a0 = tc::smem_u32(sA + s * kStageA), b0 = tc::smem_u32(sB + s * kStageB);
#pragma unroll
          for (int kk = 0; kk < kBK / 32; ++kk)
            tc::mma<true>(d, tc::sw128_desc(a0 + kk * 32), tc::sw128_desc(b0 + kk * 32), idesc,
                          (kb > 0 || kk > 0) ? 1u : 0u);
          tc::commit(&S.empty[s]);
        }
        tc::commit(&S.tfull[buf]);
      }
    }
    __syncwarp();
  } else {
    // epilogue warps: TMEM lane quarter = warp % 4; the EPI / 4 warps of a
    // quarter split the columns
    constexpr int kCols = kBN * 4 / EPI;  // columns per epilogue warp
    const int quarter = warp & 3;
    const int ew = warp - 2;
    const int half = ew / 4;              // which column slice of its quarter
    const int t = threadIdx.x - 64;       // 0 .. 32 EPI - 1
    int li = 0;
    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++li) {
      const int tm = tile / tiles_n, tn = tile % tiles_n;
      const int buf = li & 1;
      const int row = quarter * 32 + lane;
      const int c = tm * kBM + row;
      const int len = c < m ? __ldg(row_len + c) : 0;
      const int64_t w = c < m ? __ldg(row_w + c) : 0;
      const int bias = (1 << len) - 1;
      // rows of one warp that share a weight let a popcount replace the sum
      const bool uniform = __ldg(grp_small + tm * 4 + quarter) != 0;
      const float unsat_d = -(float)bias;  // D of a clause with no true literal
      S.w[ew][lane] = w;
      __syncwarp();
      const bool ok = tc::mbar_wait(&S.tfull[buf], (uint32_t)(li >> 1) & 1u, err, 3, kWaitCycles);
      tc::fence_after_sync();
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) +
                             (uint32_t)(buf * kBN + half * kCols);
      for (int j = 0; j < kCols / 32; ++j) {
        uint32_t r[32];
        tc::tmem_ld32(taddr + (uint32_t)(j * 32), r);
        tc::tmem_ld_wait();
        uint32_t unsat = 0;  // bit q: column q unsatisfied for this row
#pragma unroll
        for (int q = 0; q < 32; ++q) unsat |= (uint32_t)(__uint_as_float(r[q]) == unsat_d) << q;
        if (!ok) unsat = 0;
        uint32_t rows = tc::transpose32(unsat, lane);  // lane = column: its unsatisfied rows
        int64_t col;
        if (uniform) {
          col = (int64_t)__popc(rows) * S.w[ew][0];
        } else {
          col = 0;
          while (rows) {
            col += S.w[ew][__ffs(rows) - 1];
            rows &= rows - 1;
          }
        }
        S.cost[buf][ew * kCols + j * 32 + lane] = col;
      }
      // accumulator drained: hand the buffer back to the MMA warp
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&S.tempty[buf]))
                     : "memory");
      // one barrier per tile: the column sums are double-buffered by tile
      // parity, so the next tile writes the other buffer while this one is read
      tc::epi_bar<32 * EPI>();
      for (int col = t; col < kBN; col += 32 * EPI) {
        const int h = col / kCols, cc = col % kCols;  // which warp of each quarter
        int64_t csum = 0;
#pragma unroll
        for (int qd = 0; qd < 4; ++qd) csum += S.cost[buf][(h * 4 + qd) * kCols + cc];
        const int b = tn * kBN + col;
        if (b < B && csum != 0)
          atomicAdd(reinterpret_cast<unsigned long long*>(out + b), (unsigned long long)csum);
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

// 16 bytes of X (chain b, variables i0 .. i0 + 15) from the assignment
// bytes: +1 / -1 (nonzero / zero) as FP8, 0 past n; 8-byte loads when the
// row segment allows them, else byte loads.
__device__ __forceinline__ uint4 convert16(const uint8_t* __restrict__ assign, int n, int b,
                                           int i0, uint32_t minus_one4) {
  const uint8_t* p = assign + (size_t)b * n + i0;
  uint32_t w[4] = {0u, 0u, 0u, 0u}, valid[4] = {0u, 0u, 0u, 0u};
  if (i0 + 16 <= n && (reinterpret_cast<uintptr_t>(p) & 7u) == 0) {
    const uint2 lo = __ldg(reinterpret_cast<const uint2*>(p));
    const uint2 hi = __ldg(reinterpret_cast<const uint2*>(p) + 1);
    w[0] = lo.x;
    w[1] = lo.y;
    w[2] = hi.x;
    w[3] = hi.y;
#pragma unroll
    for (int q = 0; q < 4; ++q) valid[q] = 0xFFFFFFFFu;
  } else {
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (i0 + k < n) {
        w[k >> 2] |= (uint32_t)__ldg(p + k) << (8 * (k & 3));
        valid[k >> 2] |= 0xFFu << (8 * (k & 3));
      }
  }
  uint32_t o[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    // bit 7 of each byte: the byte is nonzero; flipping the sign of -1 gives +1
    const uint32_t nz = (((w[q] & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w[q]) & 0x80808080u;
    o[q] = (minus_one4 ^ nz) & valid[q];
  }
  return make_uint4(o[0], o[1], o[2], o[3]);
}

// assign (B x n bytes, nonzero = true) -> X (Bp x n_pad FP8): +1 / -1 for
// variables, 0 for padding variables and padding chains; 16 output bytes
// (one 16-byte store) per thread. Then zeroes the B costs the product
// accumulates into. It is the programmatic dependent of the launch before it
// on the stream: when that is the previous evaluation's product (which lets
// it start early, and reads the other state buffer), the conversion runs
// beside it, and only the zeroing of the costs, which that product may
// still be adding into, waits for its end.
__global__ void k_assign_fp8(const uint8_t* __restrict__ assign, int B, int n, int Bp, int n_pad,
                             uint32_t minus_one4, uint8_t* __restrict__ X,
                             int64_t* __restrict__ cost) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t first = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int chunks = n_pad / 16;
  for (size_t idx = first; idx < (size_t)Bp * chunks; idx += stride) {
    const int b = (int)(idx / chunks), i0 = (int)(idx % chunks) * 16;
    reinterpret_cast<uint4*>(X)[idx] =
        b < B ? convert16(assign, n, b, i0, minus_one4) : make_uint4(0u, 0u, 0u, 0u);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (size_t idx = first; idx < (size_t)B; idx += stride) cost[idx] = 0;
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
                              const int64_t* row_w, const uint8_t* grp_small, int64_t* out,
                              int* err, cudaStream_t st) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_gemm1_eval<kEpiWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kGemm1Smem);
    if (e != cudaSuccess) {
      sms = 0;
      return e;
    }
  }
  const uint32_t fmt = e5m2 ? 1u : 0u;
  const uint32_t idesc = tc::instr_desc(kBM, kBN, fmt, fmt);
  const int tiles_m = m_pad / kBM, tiles_n = Bp / kBN;
  const int grid = std::min(sms, tiles_m * tiles_n);
  // programmatic dependent of the conversion launched just before it
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(64 + 32 * kEpiWarps);
  cfg.dynamicSmemBytes = kGemm1Smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_gemm1_eval<kEpiWarps>, tmA, tmB, m, n_pad / kBK, tiles_m,
                            tiles_n, B, Bp, idesc, row_len, row_w, grp_small, out, err);
}

cudaError_t launch_assign_fp8(const uint8_t* assign, int B, int n, int Bp, int n_pad, bool e5m2,
                              uint8_t* X, int64_t* cost, cudaStream_t st) {
  uint8_t minus_one;
  fp8_encode_int(-1, e5m2, &minus_one);
  const size_t total = std::max((size_t)Bp * (n_pad / 16), (size_t)B);
  // at most 3 blocks per SM (30 registers a thread): all of them stay
  // resident beside the previous evaluation's product (one CTA of 576
  // threads at 61 registers per SM), so the conversion is done before that
  // product ends and only the zeroing waits for it
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 1;
  }
  const size_t blocks = std::min((total + 255) / 256, (size_t)3 * (size_t)sms);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_assign_fp8, assign, B, n, Bp, n_pad, 0x01010101u * minus_one,
                            X, cost);
}

}  // namespace rbmsat
