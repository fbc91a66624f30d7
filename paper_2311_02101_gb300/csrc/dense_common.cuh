// Device helpers shared by the dense (tensor-core) kernels.
#pragma once

#include <cstdint>

#include "tc_ptx.cuh"

namespace rbmsat {
namespace tc {

template <int EPI_THREADS>
__device__ __forceinline__ void epi_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");
}

// 32 x 32 bit-matrix transpose across a warp: lane i holds row i (bit q =
// column q); afterwards lane q holds column q (bit i = row i). Five stages
// swap the off-diagonal blocks of size 16, 8, 4, 2, 1.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int j = 16 >> st;
    const uint32_t mk = masks[st];
    const uint32_t other = __shfl_xor_sync(0xFFFFFFFFu, x, j);
    x = (lane & j) ? ((x & ~mk) | ((other >> j) & mk)) : ((x & mk) | ((other & mk) << j));
  }
  return x;
}

// Warp transpose-reduce: lane l holds v[0..31] (one value per column of its
// row); afterwards v[0] of lane l is the sum over the 32 lanes of column l.
// Five halving levels, 31 shuffles in total.
template <typename T>
__device__ __forceinline__ T column_sums32(T (&v)[32], int lane) {
#pragma unroll
  for (int level = 0; level < 5; ++level) {
    const int half = 16 >> level;
    const bool upper = (lane & half) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const T send = upper ? v[i] : v[i + half];
      const T keep = upper ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, half);
    }
  }
  return v[0];
}


// Sum over the 32 lanes of 8 per-lane column values: afterwards every lane
// holds the total of column (lane & 7). Three halving levels and two plain
// ones, 9 shuffles.
template <typename T>
__device__ __forceinline__ T column_sums8(T (&v)[8], int lane) {
#pragma unroll
  for (int level = 0; level < 3; ++level) {
    const int half = 4 >> level;
    const bool upper = (lane & half) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const T send = upper ? v[i] : v[i + half];
      const T keep = upper ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, half);
    }
  }
  T x = v[0];
  x += __shfl_xor_sync(0xFFFFFFFFu, x, 8);
  x += __shfl_xor_sync(0xFFFFFFFFu, x, 16);
  return x;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (tensor core / TMA) reads.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace tc
}  // namespace rbmsat
