// Learned proposal: a message-passing network over the variable-clause
// incidence of a formula, trained on the solver's own best assignments, that
// supplies the chains' initial assignments (the paper names learned initial
// assignments as complementary to RbmSAT, Sec. 2).
//
//   f_v = [pos_v / deg_v - 1/2, log(1 + deg_v) / 4, 1],  g_c = [log(w_c) / 8, len_c / 4, 1]
//   h_v^0 = relu(Wf f_v),  h_c^0 = relu(Wg g_c)                      (H = 64)
//   layer l: m_c = mean_{(v,s) in c} s h_v^{l-1}
//            h_c^l = relu(Wc_l [m_c ; h_c^{l-1}] + bc_l)
//            a_v = mean_{(c,s) : v in c} s h_c^l
//            h_v^l = relu(Wv_l [a_v ; h_v^{l-1}] + bv_l)
//   z_v = wo . h_v^L + bo,  p_v = sigmoid(z_v),  loss = mean_v softplus(z_v) - y_v z_v
//
// Weight matrices are used in BF16 (rounded from FP32 master weights after
// every Adam step); activations, biases and all sums are FP32. Every kernel is
// hand-written: the signed-mean aggregations walk the same clause and
// variable incidence lists as the Gibbs round (one warp per clause or
// variable, two features per lane), the dense layers stage the weights in
// shared memory, and weight gradients are reduced in two deterministic
// stages (per-block partials, then a fixed-order sum). No atomics.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"
#include "philox.cuh"

namespace rbmsat {

namespace {

constexpr int kH = 64;
constexpr int kRowsW = 256;  // rows per block of the weight-gradient partials

__device__ __forceinline__ float relu(float x) { return x > 0.f ? x : 0.f; }

// ---------------------------------------------------------------- features
__global__ void k_mp_var_features(DevFormula F, float* f, float* inv_deg) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= F.n) return;
  const int j0 = F.var_off[v], j1 = F.var_off[v + 1];
  int pos = 0;
  for (int j = j0; j < j1; ++j) pos += F.var_inc[j].y >= 0 ? 1 : 0;
  const int deg = j1 - j0;
  f[3 * v + 0] = deg > 0 ? (float)pos / (float)deg - 0.5f : 0.f;
  f[3 * v + 1] = log1pf((float)deg) * 0.25f;
  f[3 * v + 2] = 1.f;
  inv_deg[v] = deg > 0 ? 1.f / (float)deg : 0.f;
}

__global__ void k_mp_clause_features(DevFormula F, float* g, float* inv_len) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= F.m) return;
  const int len = F.cl_off[c + 1] - F.cl_off[c];
  g[3 * c + 0] = logf((float)F.cl_w[c]) * 0.125f;
  g[3 * c + 1] = (float)len * 0.25f;
  g[3 * c + 2] = 1.f;
  inv_len[c] = len > 0 ? 1.f / (float)len : 0.f;
}

// out[r][j] = relu(sum_k W[j][k] in[r][k]), K = 3
__global__ void k_mp_proj(const float* in, int rows, const __nv_bfloat16* W, float* out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * kH) return;
  const int r = (int)(e / kH), j = (int)(e % kH);
  const float* x = in + 3 * (size_t)r;
  float acc = __bfloat162float(W[3 * j]) * x[0];
  acc = fmaf(__bfloat162float(W[3 * j + 1]), x[1], acc);
  acc = fmaf(__bfloat162float(W[3 * j + 2]), x[2], acc);
  out[e] = relu(acc);
}

// ------------------------------------------------------------- aggregation
// Per clause c (one warp, two features per lane):
//   out[c] (+)= cscale[c] * sum_{(v, s) in c} s * vscale[v] * h[v]
// (scales NULL = 1).
__global__ void k_mp_clause_agg(DevFormula F, const float* h, const float* cscale,
                                const float* vscale, float* out, int accumulate) {
  const int c = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= F.m) return;
  float2 acc = make_float2(0.f, 0.f);
  for (int j = F.cl_off[c]; j < F.cl_off[c + 1]; ++j) {
    const int32_t lv = __ldg(F.lit_var + j);
    const int v = lv & 0x7FFFFFFF;
    float s = lv < 0 ? -1.f : 1.f;
    if (vscale) s *= __ldg(vscale + v);
    const float2 x = __ldg(reinterpret_cast<const float2*>(h + (size_t)v * kH) + lane);
    acc.x = fmaf(s, x.x, acc.x);
    acc.y = fmaf(s, x.y, acc.y);
  }
  const float cs = cscale ? cscale[c] : 1.f;
  float2* o = reinterpret_cast<float2*>(out + (size_t)c * kH) + lane;
  float2 r = make_float2(cs * acc.x, cs * acc.y);
  if (accumulate) {
    const float2 p = *o;
    r.x += p.x;
    r.y += p.y;
  }
  *o = r;
}

// Per variable v (one warp): out[v] (+)= vscale[v] * sum_{(c, s) : v in c}
// s * cscale[c] * h[c].
__global__ void k_mp_var_agg(DevFormula F, const float* h, const float* cscale,
                             const float* vscale, float* out, int accumulate) {
  const int v = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (v >= F.n) return;
  float2 acc = make_float2(0.f, 0.f);
  for (int j = F.var_off[v]; j < F.var_off[v + 1]; ++j) {
    const int4 inc = __ldg(F.var_inc + j);
    float s = inc.y < 0 ? -1.f : 1.f;
    if (cscale) s *= __ldg(cscale + inc.x);
    const float2 x = __ldg(reinterpret_cast<const float2*>(h + (size_t)inc.x * kH) + lane);
    acc.x = fmaf(s, x.x, acc.x);
    acc.y = fmaf(s, x.y, acc.y);
  }
  const float vs = vscale ? vscale[v] : 1.f;
  float2* o = reinterpret_cast<float2*>(out + (size_t)v * kH) + lane;
  float2 r = make_float2(vs * acc.x, vs * acc.y);
  if (accumulate) {
    const float2 p = *o;
    r.x += p.x;
    r.y += p.y;
  }
  *o = r;
}

// ------------------------------------------------------------ dense layers
// out[r] = relu(W [A[r] ; B[r]] + b), W 64 x 128 (BF16), 256 threads, 32 rows
// per block (4 rows at a time, one output feature per thread).
__global__ void __launch_bounds__(256) k_mp_dense_fwd(const float* A, const float* Bm, int rows,
                                                      const __nv_bfloat16* W, const float* b,
                                                      float* out) {
  __shared__ float Wt[2 * kH][kH];  // transposed: Wt[k][j]
  __shared__ float x[4][2 * kH];
  for (int e = threadIdx.x; e < kH * 2 * kH; e += 256) {
    const int j = e / (2 * kH), k = e % (2 * kH);
    Wt[k][j] = __bfloat162float(W[e]);
  }
  const int ri = threadIdx.x >> 6, j = threadIdx.x & 63;
  const float bj = b[j];
  for (int g = 0; g < 8; ++g) {
    const int r0 = blockIdx.x * 32 + g * 4;
    __syncthreads();
    for (int e = threadIdx.x; e < 4 * 2 * kH; e += 256) {
      const int rr = e / (2 * kH), k = e % (2 * kH), r = r0 + rr;
      x[rr][k] = r < rows ? (k < kH ? A[(size_t)r * kH + k] : Bm[(size_t)r * kH + k - kH]) : 0.f;
    }
    __syncthreads();
    const int r = r0 + ri;
    float acc = bj;
#pragma unroll 16
    for (int k = 0; k < 2 * kH; ++k) acc = fmaf(Wt[k][j], x[ri][k], acc);
    if (r < rows) out[(size_t)r * kH + j] = relu(acc);
  }
}

// dX = (dout * [out > 0]) W: dA[r] = first 64 columns, dB[r] = last 64 (written).
__global__ void __launch_bounds__(256) k_mp_dense_bwd_x(const float* dout, const float* out,
                                                        int rows, const __nv_bfloat16* W,
                                                        float* dA, float* dB) {
  __shared__ float Ws[kH][2 * kH];
  __shared__ float d[2][kH];
  for (int e = threadIdx.x; e < kH * 2 * kH; e += 256) Ws[e / (2 * kH)][e % (2 * kH)] = __bfloat162float(W[e]);
  const int ri = threadIdx.x >> 7, k = threadIdx.x & 127;
  for (int g = 0; g < 16; ++g) {
    const int r0 = blockIdx.x * 32 + g * 2;
    __syncthreads();
    if (threadIdx.x < 2 * kH) {
      const int rr = threadIdx.x / kH, jj = threadIdx.x % kH, r = r0 + rr;
      d[rr][jj] = r < rows && out[(size_t)r * kH + jj] > 0.f ? dout[(size_t)r * kH + jj] : 0.f;
    }
    __syncthreads();
    const int r = r0 + ri;
    float acc = 0.f;
#pragma unroll 16
    for (int j = 0; j < kH; ++j) acc = fmaf(d[ri][j], Ws[j][k], acc);
    if (r < rows) {
      if (k < kH) dA[(size_t)r * kH + k] = acc;
      else dB[(size_t)r * kH + k - kH] = acc;
    }
  }
}

// Per-block partial weight gradients of a dense layer over kRowsW rows:
// part[blk] = [sum_r delta[r][j] x[r][k] (64 x K) ; sum_r delta[r][j] (64)],
// delta = dout * [out > 0], x = [A ; B] (K = 128) or A alone (K = 3).
template <int K>
__global__ void __launch_bounds__(256) k_mp_wgrad_parts(const float* dout, const float* out,
                                                        const float* A, const float* Bm, int rows,
                                                        float* part) {
  constexpr int E = kH * K;
  constexpr int PER = (E + 255) / 256;
  __shared__ float d[16][kH];
  __shared__ float x[16][K];
  float acc[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) acc[i] = 0.f;
  float accb = 0.f;
  const int rbase = blockIdx.x * kRowsW;
  for (int r0 = rbase; r0 < rbase + kRowsW; r0 += 16) {
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * kH; e += 256) {
      const int rr = e / kH, j = e % kH, r = r0 + rr;
      d[rr][j] = r < rows && out[(size_t)r * kH + j] > 0.f ? dout[(size_t)r * kH + j] : 0.f;
    }
    for (int e = threadIdx.x; e < 16 * K; e += 256) {
      const int rr = e / K, k = e % K, r = r0 + rr;
      float v = 0.f;
      if (r < rows) {
        if (K == 2 * kH) v = k < kH ? A[(size_t)r * kH + k] : Bm[(size_t)r * kH + k - kH];
        else v = A[(size_t)r * K + k];
      }
      x[rr][k] = v;
    }
    __syncthreads();
    for (int rr = 0; rr < 16; ++rr) {
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        const int e = threadIdx.x + 256 * i;
        if (e < E) acc[i] = fmaf(d[rr][e / K], x[rr][e % K], acc[i]);
      }
      if (threadIdx.x < kH) accb += d[rr][threadIdx.x];
    }
  }
  float* p = part + (size_t)blockIdx.x * (E + kH);
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + 256 * i;
    if (e < E) p[e] = acc[i];
  }
  if (threadIdx.x < kH) p[E + threadIdx.x] = accb;
}

// grad[e] = sum over blocks of part[blk][e] (fixed order), e < count; rows of
// part are `stride` apart
__global__ void k_mp_sum_parts(const float* part, int nblk, int stride, int count, float* grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * stride + e];
  grad[e] = s;
}

// ---------------------------------------------------------------- read-out
// z = wo . h + bo, p = sigmoid(z); with labels: dz = (p - y) / n and the loss
// terms softplus(z) - y z (per-block partial sums, 8 rows per block).
__global__ void k_mp_out(const float* h, int n, const float* wo, const float* bo,
                         const uint8_t* y, float* prob, float* dz, double* loss_part) {
  __shared__ double lp[8];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * 8 + w;
  double term = 0.0;
  if (r < n) {
    const float2 x = reinterpret_cast<const float2*>(h + (size_t)r * kH)[lane];
    const float2 o = reinterpret_cast<const float2*>(wo)[lane];
    float acc = fmaf(x.x, o.x, x.y * o.y);
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, s);
    const float z = acc + bo[0];
    const float p = 1.f / (1.f + expf(-z));
    if (lane == 0) {
      if (prob) prob[r] = p;
      if (y) {
        const float yy = y[r] ? 1.f : 0.f;
        dz[r] = (p - yy) / (float)n;
        term = (double)(z > 0.f ? z + log1pf(expf(-z)) : log1pf(expf(z))) - (double)(yy * z);
      }
    }
  }
  if (lane == 0) lp[w] = term;
  __syncthreads();
  if (threadIdx.x == 0 && loss_part) {
    double s = 0.0;
    for (int i = 0; i < 8; ++i) s += lp[i];
    loss_part[blockIdx.x] = s;
  }
}

// dh[r][k] = dz[r] wo[k]; per-block partials of [sum_r dz[r] h[r][k] (64) ; sum_r dz[r]]
__global__ void k_mp_out_bwd(const float* h, const float* dz, int n, const float* wo, float* dh,
                             float* part) {
  __shared__ float sh[kH + 1];
  const int k = threadIdx.x;  // 64 threads
  float acc = 0.f, accb = 0.f;
  const int r0 = blockIdx.x * kRowsW;
  for (int r = r0; r < min(r0 + kRowsW, n); ++r) {
    const float d = dz[r];
    dh[(size_t)r * kH + k] = d * wo[k];
    acc = fmaf(d, h[(size_t)r * kH + k], acc);
    accb += d;
  }
  sh[k] = acc;
  if (k == 0) sh[kH] = accb;
  __syncthreads();
  float* p = part + (size_t)blockIdx.x * (kH + 1);
  p[k] = sh[k];
  if (k == 0) p[kH] = sh[kH];
}

// --------------------------------------------------------------- optimiser
__global__ void k_mp_adam(float* P, const float* G, float* M, float* V, int count, float lr,
                          float b1, float b2, float eps, float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float g = G[e];
  const float m = b1 * M[e] + (1.f - b1) * g;
  const float v = b2 * V[e] + (1.f - b2) * g * g;
  M[e] = m;
  V[e] = v;
  P[e] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__global__ void k_mp_to_bf16(const float* P, __nv_bfloat16* Pb, int count) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) Pb[e] = __float2bfloat16_rn(P[e]);
}

// ------------------------------------------------ biased initial states
// x = [u < P_v] with the initial-draw Philox counter (variable, chain octet,
// 0, init phase | instance << 8): P_v = 32768 everywhere gives exactly the
// states of maxsat_reset. Sparse layout (variable-major) and dense layout.
__global__ void k_init_probs_sparse(DevFormula F, DevChains C, const uint32_t* P, int vg0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g8 = blockIdx.x * 32 + lane, b0 = g8 * 8;
  const int i = (vg0 + blockIdx.y) * 8 + warp;
  if (i >= F.n) return;
  const int2 vi = F.var_inst ? F.var_inst[i] : make_int2(0, i);
  const uint4 r = philox4x32_10(make_uint4((uint32_t)vi.y, (uint32_t)(g8 + C.g8_off), 0u,
                                           kPhaseInit | ((uint32_t)vi.x << 8)),
                                C.keys);
  const uint32_t Pi = P[i];
  uint64_t x = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) x |= (uint64_t)(lane16(r, q) < Pi) << (8 * q);
  const size_t o = (size_t)i * C.Bp + b0;
  *reinterpret_cast<uint64_t*>(C.xt + o) = x;
  *reinterpret_cast<uint64_t*>(C.best_xt + o) = x;
}

__global__ void k_init_probs_dense(int n, int n_pad, DevChains C, const uint32_t* P, uint8_t* X,
                                   uint8_t* best_x, uint8_t one, uint8_t minus_one, int vg0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g8 = blockIdx.x * 32 + lane, b0 = g8 * 8;
  const int i = (vg0 + blockIdx.y) * 8 + warp;
  if (i >= n) return;
  const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(g8 + C.g8_off), 0u, kPhaseInit),
                                C.keys);
  const uint32_t Pi = P[i];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const bool bit = lane16(r, q) < Pi;
    const size_t o = (size_t)(b0 + q) * n_pad + i;
    X[o] = bit ? one : minus_one;
    best_x[o] = bit ? 1 : 0;
  }
}

}  // namespace

// ====================================================================== host
int mp_layout(int L, MpLayout* out) {
  if (L < 1 || L > kMpMaxLayers) return -1;
  int o = 0;
  out->L = L;
  out->Wf = o, o += kH * 3;
  out->Wg = o, o += kH * 3;
  for (int l = 0; l < L; ++l) {
    out->Wc[l] = o, o += kH * 2 * kH;
    out->bc[l] = o, o += kH;
    out->Wv[l] = o, o += kH * 2 * kH;
    out->bv[l] = o, o += kH;
  }
  out->wo = o, o += kH;
  out->bo = o, o += 1;
  out->total = o;
  return 0;
}

namespace {
inline int blocks(long long count, int per) { return (int)((count + per - 1) / per); }
}  // namespace

cudaError_t mp_launch_features(const DevFormula& F, float* f, float* g, float* inv_len,
                               float* inv_deg, cudaStream_t st) {
  if (F.n > 0) k_mp_var_features<<<blocks(F.n, 256), 256, 0, st>>>(F, f, inv_deg);
  if (F.m > 0) k_mp_clause_features<<<blocks(F.m, 256), 256, 0, st>>>(F, g, inv_len);
  return cudaGetLastError();
}

cudaError_t mp_launch_proj(const float* in, int rows, const __nv_bfloat16* W, float* out,
                           cudaStream_t st) {
  if (rows > 0) k_mp_proj<<<blocks((long long)rows * kH, 256), 256, 0, st>>>(in, rows, W, out);
  return cudaGetLastError();
}

cudaError_t mp_launch_clause_agg(const DevFormula& F, const float* h, const float* cscale,
                                 const float* vscale, float* out, bool acc, cudaStream_t st) {
  if (F.m > 0)
    k_mp_clause_agg<<<blocks(F.m, 8), 256, 0, st>>>(F, h, cscale, vscale, out, acc ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t mp_launch_var_agg(const DevFormula& F, const float* h, const float* cscale,
                              const float* vscale, float* out, bool acc, cudaStream_t st) {
  if (F.n > 0)
    k_mp_var_agg<<<blocks(F.n, 8), 256, 0, st>>>(F, h, cscale, vscale, out, acc ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t mp_launch_dense_fwd(const float* A, const float* Bm, int rows, const __nv_bfloat16* W,
                                const float* b, float* out, cudaStream_t st) {
  if (rows > 0) k_mp_dense_fwd<<<blocks(rows, 32), 256, 0, st>>>(A, Bm, rows, W, b, out);
  return cudaGetLastError();
}

cudaError_t mp_launch_dense_bwd(const float* dout, const float* out, const float* A,
                                const float* Bm, int rows, const __nv_bfloat16* W, float* dA,
                                float* dB, float* part, float* gW, cudaStream_t st) {
  if (rows <= 0) return cudaMemsetAsync(gW, 0, sizeof(float) * (kH * 2 * kH + kH), st);
  k_mp_dense_bwd_x<<<blocks(rows, 32), 256, 0, st>>>(dout, out, rows, W, dA, dB);
  const int nb = blocks(rows, kRowsW);
  k_mp_wgrad_parts<2 * kH><<<nb, 256, 0, st>>>(dout, out, A, Bm, rows, part);
  const int width = kH * 2 * kH + kH;
  k_mp_sum_parts<<<blocks(width, 256), 256, 0, st>>>(part, nb, width, width, gW);
  return cudaGetLastError();
}

cudaError_t mp_launch_proj_bwd(const float* dout, const float* out, const float* in, int rows,
                               float* part, float* gW, cudaStream_t st) {
  if (rows <= 0) return cudaMemsetAsync(gW, 0, sizeof(float) * kH * 3, st);
  const int nb = blocks(rows, kRowsW);
  k_mp_wgrad_parts<3><<<nb, 256, 0, st>>>(dout, out, in, nullptr, rows, part);
  // the projection has no bias: only the first 64 x 3 entries of each part
  k_mp_sum_parts<<<1, 256, 0, st>>>(part, nb, kH * 3 + kH, kH * 3, gW);
  return cudaGetLastError();
}

cudaError_t mp_launch_out(const float* h, int n, const float* wo, const float* bo,
                          const uint8_t* y, float* prob, float* dz, double* loss_part,
                          cudaStream_t st) {
  if (n > 0) k_mp_out<<<blocks(n, 8), 256, 0, st>>>(h, n, wo, bo, y, prob, dz, loss_part);
  return cudaGetLastError();
}

cudaError_t mp_launch_out_bwd(const float* h, const float* dz, int n, const float* wo, float* dh,
                              float* part, float* g_wo, cudaStream_t st) {
  const int nb = blocks(n, kRowsW);
  k_mp_out_bwd<<<nb, kH, 0, st>>>(h, dz, n, wo, dh, part);
  k_mp_sum_parts<<<1, kH + 1, 0, st>>>(part, nb, kH + 1, kH + 1, g_wo);  // wo then bo
  return cudaGetLastError();
}

cudaError_t mp_launch_adam(float* P, const float* G, float* M, float* V, int count, float lr,
                           float b1, float b2, float eps, int step, __nv_bfloat16* Pb,
                           cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_mp_adam<<<blocks(count, 256), 256, 0, st>>>(P, G, M, V, count, lr, b1, b2, eps, c1, c2);
  k_mp_to_bf16<<<blocks(count, 256), 256, 0, st>>>(P, Pb, count);
  return cudaGetLastError();
}

cudaError_t mp_launch_to_bf16(const float* P, __nv_bfloat16* Pb, int count, cudaStream_t st) {
  k_mp_to_bf16<<<blocks(count, 256), 256, 0, st>>>(P, Pb, count);
  return cudaGetLastError();
}

cudaError_t launch_init_probs_sparse(const DevFormula& F, const DevChains& C, const uint32_t* P,
                                     cudaStream_t st) {
  const int groups = (F.n + 7) / 8;
  for (int vg0 = 0; vg0 < groups; vg0 += 65535) {
    dim3 grid(C.Bp / kChainTile, std::min(65535, groups - vg0));
    k_init_probs_sparse<<<grid, 256, 0, st>>>(F, C, P, vg0);
  }
  return cudaGetLastError();
}

cudaError_t launch_init_probs_dense(int n, int n_pad, const DevChains& C, const uint32_t* P,
                                    uint8_t* X, uint8_t* best_x, uint8_t one, uint8_t minus_one,
                                    cudaStream_t st) {
  const int groups = (n + 7) / 8;
  for (int vg0 = 0; vg0 < groups; vg0 += 65535) {
    dim3 grid(C.Bp / kChainTile, std::min(65535, groups - vg0));
    k_init_probs_dense<<<grid, 256, 0, st>>>(n, n_pad, C, P, X, best_x, one, minus_one, vg0);
  }
  return cudaGetLastError();
}

}  // namespace rbmsat
