// Prioritized unit propagation (Sec. 4.4) and the B-of-2B merge on the GPU.
//
// The paper runs the heuristic on host cores while the accelerator keeps
// sampling. Here the same procedure runs as one warp per chain on a side
// stream (the Gibbs rounds keep running on the context's stream meanwhile),
// and the merge scores, ranks and permutes the candidates on the device.
//
// k_up_chains  one warp = one chain, its state in shared memory:
//   keys   n_pad u64: nu ranking keys, sorted by a warp bitonic sort
//          (nu descending, ties to the lower index; -0 == +0); once sorted,
//          compacted in place to n int32 variable indices (the ranking), and
//          the bytes after them hold the queue: n int32 literals (bit 31 =
//          negated), first in, first out;
//   val    n bytes: 0 / 1 assigned, 2 unassigned, 3 unassigned and queued.
// A clause's state is read from val directly (satisfied: a true literal;
// unit: no true literal and exactly one unassigned literal occurrence),
// which is what the host's incremental counters hold. Queue entries are
// appended in the host's order, but a variable is queued at most once: only
// the first entry of a variable can assign it (a later entry finds it
// assigned), so the dropped entries change nothing, and the queue holds at
// most n entries.
// k_up_rank    position of each of the 2B candidates in the stable sort by
//              cost descending (= satisfied weight ascending), by counting:
//              each block counts one slice of the compared candidates and
//              adds its counts to a zeroed rank array (integer atomics);
// k_up_place   candidates at positions B .. 2B - 1 become chains 0 .. B - 1.
// k_up_permute chain j takes the candidate at position B + j; nu of the
//              chain it came from.
#include <cstdint>

#include "internal.h"

namespace rbmsat {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kUpMaxWarps = 4;             // chains per block
constexpr int kUpSmemBudget = 200 * 1024;  // shared memory of one block (cap)

int up_npad(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

int up_warp_bytes(int n) { return (8 * up_npad(n) + n + 15) & ~15; }

// descending order of nu as an ascending u32 (-0 and +0 equal)
__device__ __forceinline__ uint32_t desc_key(float f) {
  uint32_t u = __float_as_uint(f);
  if ((u << 1) == 0u) u = 0u;
  const uint32_t asc = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ~asc;
}

// lit_var of clause c's only unassigned literal occurrence when the clause is
// not satisfied and exactly one occurrence is unassigned; val is indexed by a
// variable's index within its formula (global index - vb)
__device__ __forceinline__ bool unit_literal(const UpDev& U, const int8_t* val, int vb, int c,
                                             int32_t* lv_out) {
  const int o = __ldg(U.cl_off + c), e = __ldg(U.cl_off + c + 1);
  int nun = 0;
  int32_t first = 0;
  for (int j = o; j < e; ++j) {
    const int32_t lv = __ldg(U.lit_var + j);
    const int s = val[(lv & 0x7FFFFFFF) - vb];
    if (s >= 2) {
      if (nun == 0) first = lv;
      ++nun;
    } else if ((s == 1) != (lv < 0)) {
      return false;  // satisfied
    }
  }
  *lv_out = first;
  return nun == 1;
}

struct ChainState {
  int8_t* val;     // by index within the formula
  int32_t* queue;  // lit_var entries (global variable indices)
  int head, tail;
  int vb;          // the formula's first variable
};

// appends the literals of the lanes in `ballot`, in lane order, each
// variable at most once
__device__ __forceinline__ void append(uint32_t ballot, int32_t lv, ChainState& S, int lane) {
  while (ballot) {
    const int src = __ffs(ballot) - 1;
    ballot &= ballot - 1;
    const int32_t l = __shfl_sync(kFull, lv, src);
    const int v = (l & 0x7FFFFFFF) - S.vb;
    const bool fresh = S.val[v] == 2;
    __syncwarp();
    if (fresh && lane == 0) {
      S.val[v] = 3;
      S.queue[S.tail] = l;
    }
    __syncwarp();
    S.tail += fresh ? 1 : 0;
  }
}

// assigns v (index within the formula) and queues the open literal of every
// clause of v that became unit (v's occurrences in clause order)
__device__ __forceinline__ void set_check(const UpDev& U, ChainState& S, int v, int value,
                                          int lane) {
  if (lane == 0) S.val[v] = (int8_t)value;
  __syncwarp();
  const int k0 = __ldg(U.occ_off + S.vb + v), k1 = __ldg(U.occ_off + S.vb + v + 1);
  for (int k = k0; k < k1; k += 32) {
    int32_t lv = 0;
    bool unit = false;
    if (k + lane < k1) unit = unit_literal(U, S.val, S.vb, __ldg(U.occ + k + lane), &lv);
    append(__ballot_sync(kFull, unit), lv, S, lane);
  }
}

__device__ __forceinline__ void drain(const UpDev& U, ChainState& S, int lane) {
  while (S.head < S.tail) {
    const int32_t l = S.queue[S.head++];
    const int v = (l & 0x7FFFFFFF) - S.vb;
    if (S.val[v] >= 2) set_check(U, S, v, l >= 0 ? 1 : 0, lane);
  }
}

__global__ void __launch_bounds__(32 * kUpMaxWarps)
    k_up_chains(UpDev U, const uint8_t* __restrict__ xs, const float* __restrict__ nus, int Bp,
                int B, uint8_t* __restrict__ out, int Bp2, int col0, int n_pad, int wbytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // warp g: formula g / B, chain g % B (whole warps leave together)
  const int g = blockIdx.x * (blockDim.x >> 5) + warp;
  if (g >= U.n_inst * B) return;
  const int fk = g / B, b = g - fk * B;
  const int vb = __ldg(U.var_base + fk), n = __ldg(U.var_base + fk + 1) - vb;
  const int cb0 = __ldg(U.cl_base + fk), cb1 = __ldg(U.cl_base + fk + 1);
  int np = 1;  // this formula's sort size (n_pad: the largest formula's)
  while (np < n) np <<= 1;
  unsigned char* base = smem + (size_t)warp * wbytes;
  uint64_t* keys = reinterpret_cast<uint64_t*>(base);
  int32_t* order = reinterpret_cast<int32_t*>(base);  // after the sort
  ChainState S;
  S.queue = reinterpret_cast<int32_t*>(base + 4 * (size_t)n);  // after the sort
  S.val = reinterpret_cast<int8_t*>(base + 8 * (size_t)n_pad);
  S.head = S.tail = 0;
  S.vb = vb;

  // 1. rank the variables by nu (bitonic sort of unique keys, ascending)
  for (int v = lane; v < np; v += 32)
    keys[v] = v < n ? ((uint64_t)desc_key(nus[(size_t)(vb + v) * Bp + b]) << 32) | (uint32_t)v
                    : ~0ull;
  for (int v = lane; v < n; v += 32) S.val[v] = 2;
  __syncwarp();
  for (int k = 2; k <= np; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < np / 2; t += 32) {
        const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        const uint64_t a = keys[i], c = keys[i + j];
        if ((a > c) == ((i & k) == 0)) {
          keys[i] = c;
          keys[i + j] = a;
        }
      }
      __syncwarp();
    }
  // the ranking as int32 over the keys' first 4 n bytes: chunks in increasing
  // order, each chunk's reads before its writes; later chunks read past them
  for (int r0 = 0; r0 < n; r0 += 32) {
    const int r = r0 + lane;
    const int v = r < n ? (int)(uint32_t)keys[r] : 0;
    __syncwarp();
    if (r < n) order[r] = v;
    __syncwarp();
  }

  // 2. the floor(n / 2) highest-ranked variables keep their values
  const int half = n / 2;
  for (int r = lane; r < half; r += 32) {
    const int v = order[r];
    S.val[v] = xs[(size_t)(vb + v) * Bp + b] ? 1 : 0;
  }
  __syncwarp();

  // 3. the formula's unit clauses in clause order, then propagation
  for (int c0 = cb0; c0 < cb1; c0 += 32) {
    int32_t lv = 0;
    bool unit = false;
    if (c0 + lane < cb1) unit = unit_literal(U, S.val, vb, c0 + lane, &lv);
    append(__ballot_sync(kFull, unit), lv, S, lane);
  }
  drain(U, S, lane);

  // 4. the rest in rank order, each still unassigned one from x, propagated
  for (int r = half; r < n; ++r) {
    const int v = order[r];
    if (S.val[v] >= 2) {
      set_check(U, S, v, xs[(size_t)(vb + v) * Bp + b] ? 1 : 0, lane);
      drain(U, S, lane);
    }
  }
  for (int v = lane; v < n; v += 32)
    out[(size_t)(vb + v) * Bp2 + col0 + b] = (uint8_t)S.val[v];
}

constexpr int kRankSlice = 1024;  // compared candidates per block

// blockIdx.z: the formula (its 2B costs and ranks at offset 2B z)
__global__ void __launch_bounds__(256) k_up_rank(const int64_t* __restrict__ cost, int N,
                                                 int32_t* __restrict__ rank) {
  __shared__ int64_t s[kRankSlice];
  cost += (size_t)blockIdx.z * N;
  rank += (size_t)blockIdx.z * N;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int lo = blockIdx.y * kRankSlice, hi = min(N, lo + kRankSlice);
  for (int k = threadIdx.x; k < hi - lo; k += blockDim.x) s[k] = cost[lo + k];
  __syncthreads();
  if (a >= N) return;
  const int64_t ca = cost[a];
  int r = 0;
  for (int k = 0; k < hi - lo; ++k) {
    const int64_t cb = s[k];
    r += (cb > ca || (cb == ca && lo + k < a)) ? 1 : 0;
  }
  if (r) atomicAdd(rank + a, r);
}

__global__ void __launch_bounds__(256) k_up_place(const int32_t* __restrict__ rank, int N, int B,
                                                  int32_t* __restrict__ perm) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= N) return;
  const int r = rank[(size_t)blockIdx.y * N + a];
  if (r >= B) perm[(size_t)blockIdx.y * B + r - B] = a;
}

// variable i of formula k (var_inst[i].x; 0 without var_inst) takes the
// candidate perm[k B + j] in chain j
__global__ void __launch_bounds__(256) k_up_permute(const uint8_t* __restrict__ cand, int Bp2,
                                                    const int32_t* __restrict__ perm, int B,
                                                    uint8_t* __restrict__ xt,
                                                    const float* __restrict__ nu,
                                                    float* __restrict__ nu_out, int Bp, int n,
                                                    const int2* __restrict__ var_inst) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= B) return;
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    const int k = var_inst ? __ldg(var_inst + i).x : 0;
    const int a = perm[(size_t)k * B + j];
    xt[(size_t)i * Bp + j] = cand[(size_t)i * Bp2 + a];
    nu_out[(size_t)i * Bp + j] = nu[(size_t)i * Bp + a % B];
  }
}

// proposal columns B..2B-1 of cand: chain b's state with every variable of
// code 0 / 1 set to it (code 2: kept)
__global__ void __launch_bounds__(256) k_flip_candidates(const uint8_t* __restrict__ xt, int Bp,
                                                         const uint8_t* __restrict__ code, int n,
                                                         int B, uint8_t* __restrict__ cand,
                                                         int Bp2) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    const uint8_t k = code[i];
    cand[(size_t)i * Bp2 + B + b] = k < 2 ? k : xt[(size_t)i * Bp + b];
  }
}

}  // namespace

cudaError_t launch_flip_candidates(const uint8_t* xt, int Bp, const uint8_t* code, int n, int B,
                                   uint8_t* cand, int Bp2, cudaStream_t st) {
  const dim3 grid((B + 255) / 256, n < 4096 ? n : 4096);
  k_flip_candidates<<<grid, 256, 0, st>>>(xt, Bp, code, n, B, cand, Bp2);
  return cudaGetLastError();
}

int up_gpu_chains_per_block(int n_max) {
  if (n_max < 1) return 0;
  const int w = up_warp_bytes(n_max);
  const int k = kUpSmemBudget / w;
  return k < 1 ? 0 : (k < kUpMaxWarps ? k : kUpMaxWarps);
}

cudaError_t launch_up_chains(const UpDev& U, const uint8_t* xs, const float* nus, int Bp, int B,
                             uint8_t* out, int Bp2, int col0, cudaStream_t st) {
  const int W = up_gpu_chains_per_block(U.n_max);
  if (W < 1 || B < 1 || U.n_inst < 1) return cudaErrorInvalidValue;
  const int wbytes = up_warp_bytes(U.n_max);
  const int smem = W * wbytes;
  {
    const cudaError_t e = allow_dynamic_smem(k_up_chains, smem);
    if (e != cudaSuccess) return e;
  }
  // three quarters of the unified memory as shared memory: as many chains per
  // SM as fit, with some L1 left for the formula's clause and occurrence lists
  // (measured: 6 % faster than the whole as shared memory; a larger L1 with
  // fewer chains is slower)
  const cudaError_t ce =
      cudaFuncSetAttribute(k_up_chains, cudaFuncAttributePreferredSharedMemoryCarveout, 75);
  if (ce != cudaSuccess) return ce;
  const int64_t warps = (int64_t)U.n_inst * B;
  if (warps > INT32_MAX - W) return cudaErrorInvalidValue;
  k_up_chains<<<(unsigned)((warps + W - 1) / W), 32 * W, smem, st>>>(
      U, xs, nus, Bp, B, out, Bp2, col0, up_npad(U.n_max), wbytes);
  return cudaGetLastError();
}

cudaError_t launch_up_merge(const int64_t* cost, int n_inst, int B, int32_t* rank, int32_t* perm,
                            const uint8_t* cand, int Bp2, uint8_t* xt, const float* nu,
                            float* nu_out, int Bp, int n, const int2* var_inst,
                            cudaStream_t st) {
  const int N = 2 * B;
  if (n_inst < 1 || n_inst > 65535) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(rank, 0, sizeof(int32_t) * (size_t)N * n_inst, st);
  if (e != cudaSuccess) return e;
  const dim3 rgrid((N + 255) / 256, (N + kRankSlice - 1) / kRankSlice, n_inst);
  if (rgrid.y > 65535) return cudaErrorInvalidValue;
  k_up_rank<<<rgrid, 256, 0, st>>>(cost, N, rank);
  k_up_place<<<dim3((N + 255) / 256, n_inst), 256, 0, st>>>(rank, N, B, perm);
  const dim3 grid((B + 255) / 256, n < 4096 ? n : 4096);
  k_up_permute<<<grid, 256, 0, st>>>(cand, Bp2, perm, B, xt, nu, nu_out, Bp, n, var_inst);
  return cudaGetLastError();
}

}  // namespace rbmsat
