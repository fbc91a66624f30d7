// Allocation-free cost evaluation: maxsat_eval_noalloc.
//
// Some callers cannot call cudaMalloc: frameworks whose own caching allocator
// owns the device memory budget (an allocation behind its back can fail or
// fragment its pool), and latency-critical loops that cannot take the implicit
// device synchronisation that cudaMalloc or cudaFree may cause. This entry
// point scores assignments of a formula that already lives in the caller's
// device memory and uses no memory beyond the caller's inputs and outputs
// except one file-scope device array, g_scratch, of
// MAXSAT_NOALLOC_SCRATCH_BYTES bytes that every GPU that loads the library
// holds until the process exits.
//
// It is a variant of the sparse evaluation pipeline of sparse.cu (transpose
// the assignments to variable-major, gather the literal truths of every clause
// for 8 chains per thread, reduce the per-block weighted costs), reading the
// DIMACS clause lists directly instead of the context's converted copy.
//
// Scratch layout: [transposed assignments: n x Bp bytes][cost partials:
// blocks x Bp int64], Bp = B rounded up to 256. Every call overwrites all of
// the scratch it reads, so nothing has to start at zero; calls that overlap on
// the GPU (on different streams, or from different host threads) share the
// array and race.
#include <cstdint>
#include <mutex>
#include <string>

#include "internal.h"

namespace rbmsat {

namespace {

static __device__ __align__(256) unsigned char g_scratch[MAXSAT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};  // device address of g_scratch per device
int noalloc_fail(int code, const std::string& msg) {
  set_context_free_error(msg);  // read back with maxsat_last_error(NULL)
  return code;
}

// assign (B x n, chain-major, nonzero = true) -> xt (n x Bp, 0/1); chains B..Bp-1
// read as all-false.
// by0: the first 32-chain tile of this launch (grids have at most 65535 tiles
// in y; more chains take several launches).
__global__ void k_na_transpose(const uint8_t* __restrict__ assign, int B, int n,
                               uint8_t* __restrict__ xt, int Bp, int by0) {
  __shared__ uint8_t tile[32][33];
  const int i0 = blockIdx.x * 32, b0 = (by0 + blockIdx.y) * 32;
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

// One thread = one clause x 8 chains, as the sparse gather; literals are read
// as DIMACS (signed, 1-based) from the caller's arrays. Offsets are clamped to
// [0, n_lits] and literals outside [-n, n] \ {0} are skipped, so no access
// leaves the caller's buffers.
__global__ void __launch_bounds__(256) k_na_gather(int m, int n, int64_t n_lits,
                                                   const int64_t* __restrict__ off,
                                                   const int32_t* __restrict__ lits,
                                                   const int64_t* __restrict__ w,
                                                   const uint8_t* __restrict__ xt, int Bp,
                                                   int cblock, int64_t* __restrict__ part) {
  __shared__ int64_t s_cost[8][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b0 = (blockIdx.x * 32 + lane) * 8;
  const int c_begin = blockIdx.y * cblock;
  const int c_end = min(c_begin + cblock, m);
  int64_t cost[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int c = c_begin + warp; c < c_end; c += 8) {
    const int64_t o0 = min(max(__ldg(off + c), (int64_t)0), n_lits);
    const int64_t o1 = min(max(__ldg(off + c + 1), o0), n_lits);
    uint64_t sat = 0;  // byte q = 1 when some literal is true for chain q
    for (int64_t j = o0; j < o1; ++j) {
      const int32_t l = __ldg(lits + j);
      // the variable index in 64-bit arithmetic: |INT32_MIN| does not fit an int
      const int64_t v = (l > 0 ? (int64_t)l : -(int64_t)l) - 1;
      if (l == 0 || v < 0 || v >= n) continue;
      uint64_t x8 = __ldg(reinterpret_cast<const unsigned long long*>(xt + (size_t)v * Bp + b0));
      if (l < 0) x8 ^= 0x0101010101010101ull;
      sat |= x8;
    }
    const int64_t wc = w ? __ldg(w + c) : 1;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (((sat >> (8 * q)) & 1u) == 0) cost[q] += wc;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) s_cost[warp][lane * 8 + q] = cost[q];
  __syncthreads();
  int64_t tc = 0;
#pragma unroll
  for (int wi = 0; wi < 8; ++wi) tc += s_cost[wi][threadIdx.x];
  part[(size_t)blockIdx.y * Bp + (size_t)blockIdx.x * 256 + threadIdx.x] = tc;
}

__global__ void k_na_reduce(const int64_t* __restrict__ part, int nblk, int Bp, int B,
                            int64_t* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  int64_t c = 0;
  for (int k = 0; k < nblk; ++k) c += part[(size_t)k * Bp + b];
  out[b] = c;
}

// Once per device, with that device current: the device address of g_scratch.
int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(MAXSAT_ENODEV, std::string("no CUDA device: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(MAXSAT_ENODEV, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    cudaDeviceProp prop{};
    e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return noalloc_fail(MAXSAT_ENODEV, cudaGetErrorString(e));
    if (prop.major != 10 || prop.minor != 3)
      return noalloc_fail(MAXSAT_ENODEV, "libmaxsat is built for sm_103 (GB300)");
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return noalloc_fail(MAXSAT_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return MAXSAT_OK;
}

}  // namespace

}  // namespace rbmsat

extern "C" int maxsat_eval_noalloc(int32_t n, int64_t m, int64_t n_lits,
                                   const int64_t* off_dev, const int32_t* lits_dev,
                                   const int64_t* w_dev, const uint8_t* assign_dev, int32_t B,
                                   int64_t* cost_dev, void* cuda_stream) {
  using namespace rbmsat;
  set_context_free_error("");
  if (n < 1 || m < 0 || m > (int64_t)INT32_MAX / 2 || n_lits < 0 || B < 0)
    return noalloc_fail(MAXSAT_EINVAL, "bad sizes");
  if (B == 0) return MAXSAT_OK;
  if (!off_dev || (n_lits > 0 && !lits_dev) || !assign_dev || !cost_dev)
    return noalloc_fail(MAXSAT_EINVAL, "NULL device pointer");
  const int64_t Bp64 = ((int64_t)B + kChainTile - 1) / kChainTile * kChainTile;
  const int cblock = clause_block_for((int)m);
  const int nblk = clause_blocks_for((int)m);
  const size_t xt_bytes = ((size_t)n * (size_t)Bp64 + 255) / 256 * 256;
  const size_t need = xt_bytes + (size_t)nblk * (size_t)Bp64 * sizeof(int64_t);
  if (need > (size_t)MAXSAT_NOALLOC_SCRATCH_BYTES)
    return noalloc_fail(MAXSAT_EINVAL,
                        "maxsat_eval_noalloc needs " + std::to_string(need) +
                            " bytes of scratch for n_vars = " + std::to_string(n) + ", B = " +
                            std::to_string(B) + "; the limit is MAXSAT_NOALLOC_SCRATCH_BYTES = " +
                            std::to_string((size_t)MAXSAT_NOALLOC_SCRATCH_BYTES));
  // the scratch bound keeps Bp below 2^25, so it is an int from here on
  const int Bp = (int)Bp64;
  unsigned char* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != MAXSAT_OK) return rc;
  uint8_t* xt = scratch;
  int64_t* part = reinterpret_cast<int64_t*>(scratch + xt_bytes);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // every launch is checked before the next one is issued, so a failed
  // transpose never lets the gather and the reduce write costs from stale
  // scratch
  auto launched = [](const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return MAXSAT_OK;
    return noalloc_fail(MAXSAT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  const int tiles = Bp / 32;
  for (int by0 = 0; by0 < tiles; by0 += 65535) {
    const int ny = tiles - by0 < 65535 ? tiles - by0 : 65535;
    k_na_transpose<<<dim3((n + 31) / 32, ny), dim3(32, 8), 0, st>>>(assign_dev, B, n, xt, Bp, by0);
    if ((rc = launched("transpose launch")) != MAXSAT_OK) return rc;
  }
  k_na_gather<<<dim3(Bp / kChainTile, nblk), 256, 0, st>>>((int)m, n, n_lits, off_dev, lits_dev,
                                                            w_dev, xt, Bp, cblock, part);
  if ((rc = launched("gather launch")) != MAXSAT_OK) return rc;
  k_na_reduce<<<(B + 255) / 256, 256, 0, st>>>(part, nblk, Bp, B, cost_dev);
  return launched("reduce launch");
}
