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
// variable, two features per lane), the 64 x 128 dense layers run on the
// tensor cores (mma.sync BF16, activations as three BF16 terms), and weight
// gradients are reduced in two deterministic stages (per-block partials,
// then a fixed-order sum). No atomics.
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
constexpr int kRowsW = 256;    // rows per block of the projections' weight-gradient partials
constexpr int kRowsTc = 256;   // rows per block of the dense layers' weight-gradient partials

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
// The three 64 x 128 contractions of a dense layer (forward, input gradient,
// weight gradient) run on the tensor cores: mma.sync m16n8k16 with BF16
// operands and FP32 accumulation. The weights are BF16 already; an FP32
// activation or gradient v enters as three BF16 terms hi + mid + lo (hi =
// bf16(v), mid = bf16(v - hi), lo = bf16(v - hi - mid)), so that products
// with BF16 weights sum to FP32 accuracy; the weight gradient, a product of
// two FP32 operands, keeps the three leading cross terms (hi x hi, hi x mid,
// mid x hi).

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
  return *reinterpret_cast<const uint32_t*>(&v);
}

// the three BF16 terms of a pair of FP32 values, packed as BF16 pairs
__device__ __forceinline__ void split3(float x0, float x1, uint32_t& t0, uint32_t& t1,
                                       uint32_t& t2) {
  const float h0 = __bfloat162float(__float2bfloat16_rn(x0));
  const float h1 = __bfloat162float(__float2bfloat16_rn(x1));
  const float r0 = x0 - h0, r1 = x1 - h1;  // exact
  const float m0 = __bfloat162float(__float2bfloat16_rn(r0));
  const float m1 = __bfloat162float(__float2bfloat16_rn(r1));
  t0 = pack_bf16(h0, h1);
  t1 = pack_bf16(m0, m1);
  t2 = pack_bf16(r0 - m0, r1 - m1);
}

__device__ __forceinline__ float2 ld2(const float* base, int rows, int r, int k) {
  return r < rows ? *reinterpret_cast<const float2*>(base + (size_t)r * kH + k)
                  : make_float2(0.f, 0.f);
}

// out[r] = relu(W [A[r] ; B[r]] + b), W 64 x 128 (BF16): one warp = 16 rows
// x 64 outputs, 8 warps per block.
__global__ void __launch_bounds__(256) k_mp_dense_fwd(const float* A, const float* Bm, int rows,
                                                      const __nv_bfloat16* W, const float* b,
                                                      float* out) {
  __shared__ uint32_t Ws[kH][kH + 4];  // W as BF16 pairs along k: Ws[j][k / 2]
  const uint32_t* W2 = reinterpret_cast<const uint32_t*>(W);
  for (int e = threadIdx.x; e < kH * kH; e += 256) Ws[e / kH][e % kH] = W2[e];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = (blockIdx.x * 8 + warp) * 16;
  if (r0 >= rows) return;
  const int ra = r0 + g, rb = r0 + g + 8;
  float acc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;
#pragma unroll 1
  for (int s = 0; s < 8; ++s) {  // k-steps of 16: [A ; B]
    const float* src = s < 4 ? A : Bm;
    const int kc = (s & 3) * 16 + 2 * t;
    const float2 x0 = ld2(src, rows, ra, kc), x1 = ld2(src, rows, rb, kc);
    const float2 x2 = ld2(src, rows, ra, kc + 8), x3 = ld2(src, rows, rb, kc + 8);
    uint32_t ah[4], am[4], al[4];
    split3(x0.x, x0.y, ah[0], am[0], al[0]);
    split3(x1.x, x1.y, ah[1], am[1], al[1]);
    split3(x2.x, x2.y, ah[2], am[2], al[2]);
    split3(x3.x, x3.y, ah[3], am[3], al[3]);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int j = nt * 8 + g;
      const uint32_t b0 = Ws[j][8 * s + t], b1 = Ws[j][8 * s + 4 + t];
      mma_bf16(acc[nt], ah, b0, b1);
      mma_bf16(acc[nt], am, b0, b1);
      mma_bf16(acc[nt], al, b0, b1);
    }
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int j = nt * 8 + 2 * t;
    const float b0 = b[j], b1 = b[j + 1];
    if (ra < rows)
      *reinterpret_cast<float2*>(out + (size_t)ra * kH + j) =
          make_float2(relu(acc[nt][0] + b0), relu(acc[nt][1] + b1));
    if (rb < rows)
      *reinterpret_cast<float2*>(out + (size_t)rb * kH + j) =
          make_float2(relu(acc[nt][2] + b0), relu(acc[nt][3] + b1));
  }
}

__device__ __forceinline__ float2 ld_delta(const float* dout, const float* out, int rows, int r,
                                           int j) {
  if (r >= rows) return make_float2(0.f, 0.f);
  const float2 d = *reinterpret_cast<const float2*>(dout + (size_t)r * kH + j);
  const float2 o = *reinterpret_cast<const float2*>(out + (size_t)r * kH + j);
  return make_float2(o.x > 0.f ? d.x : 0.f, o.y > 0.f ? d.y : 0.f);
}

// dX = (dout * [out > 0]) W: dA[r] = its first 64 columns, dB[r] the last
// 64 (written). One warp = 16 rows x 128 columns.
__global__ void __launch_bounds__(256) k_mp_dense_bwd_x(const float* dout, const float* out,
                                                        int rows, const __nv_bfloat16* W,
                                                        float* dA, float* dB) {
  __shared__ uint32_t WT[2 * kH][kH / 2 + 4];  // W^T as BF16 pairs along j: WT[k][j / 2]
  for (int e = threadIdx.x; e < 2 * kH * (kH / 2); e += 256) {
    const int k = e / (kH / 2), jp = e % (kH / 2);
    const __nv_bfloat16 lo = W[(2 * jp) * 2 * kH + k], hi = W[(2 * jp + 1) * 2 * kH + k];
    WT[k][jp] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = (blockIdx.x * 8 + warp) * 16;
  if (r0 >= rows) return;
  const int ra = r0 + g, rb = r0 + g + 8;
  float acc[16][4];
#pragma unroll
  for (int nt = 0; nt < 16; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;
#pragma unroll 1
  for (int s = 0; s < 4; ++s) {  // k-steps of 16 over the 64 outputs j
    const int jc = s * 16 + 2 * t;
    const float2 d0 = ld_delta(dout, out, rows, ra, jc), d1 = ld_delta(dout, out, rows, rb, jc);
    const float2 d2 = ld_delta(dout, out, rows, ra, jc + 8);
    const float2 d3 = ld_delta(dout, out, rows, rb, jc + 8);
    uint32_t ah[4], am[4], al[4];
    split3(d0.x, d0.y, ah[0], am[0], al[0]);
    split3(d1.x, d1.y, ah[1], am[1], al[1]);
    split3(d2.x, d2.y, ah[2], am[2], al[2]);
    split3(d3.x, d3.y, ah[3], am[3], al[3]);
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      const int k = nt * 8 + g;
      const uint32_t b0 = WT[k][8 * s + t], b1 = WT[k][8 * s + 4 + t];
      mma_bf16(acc[nt], ah, b0, b1);
      mma_bf16(acc[nt], am, b0, b1);
      mma_bf16(acc[nt], al, b0, b1);
    }
  }
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
    float* dst = nt < 8 ? dA : dB;
    const int k = (nt & 7) * 8 + 2 * t;
    if (ra < rows)
      *reinterpret_cast<float2*>(dst + (size_t)ra * kH + k) = make_float2(acc[nt][0], acc[nt][1]);
    if (rb < rows)
      *reinterpret_cast<float2*>(dst + (size_t)rb * kH + k) = make_float2(acc[nt][2], acc[nt][3]);
  }
}

// Per-block partial weight gradients of a 64 x 128 dense layer over kRowsTc
// rows: part[blk] = [sum_r delta[r][j] x[r][k] (64 x 128) ; sum_r delta[r][j]
// (64)], delta = dout * [out > 0], x = [A ; B]. Rows pass through shared
// memory 32 at a time as BF16 terms, transposed so that a fragment's row pair
// is one 32-bit word; warp w owns outputs j of tile w % 4 and columns k of
// half w / 4. Each output's bias sum is split over the four threads that
// stage it and combined in a fixed order.
__global__ void __launch_bounds__(256) k_mp_wgrad_tc(const float* dout, const float* out,
                                                     const float* A, const float* Bm, int rows,
                                                     float* part) {
  constexpr int R = 32;              // rows per pass
  __shared__ uint32_t dT[2][kH][R / 2 + 4];       // hi, mid terms of delta: [j][row pair]
  __shared__ uint32_t xT[2][2 * kH][R / 2 + 4];   // hi, mid terms of x: [k][row pair]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int mi = warp & 3, nh = warp >> 2;
  float acc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;
  float accb = 0.f;
  const int rbase = blockIdx.x * kRowsTc;
  for (int c0 = rbase; c0 < rbase + kRowsTc && c0 < rows; c0 += R) {
    __syncthreads();
    // thread t always stages output j = t % 64 (row pairs t / 64, + 4, ...)
    // and keeps its share of the bias sum
    for (int e = threadIdx.x; e < (R / 2) * kH; e += 256) {
      const int rp = e / kH, j = e % kH, r = c0 + 2 * rp;
      float v0 = 0.f, v1 = 0.f;
      if (r < rows && out[(size_t)r * kH + j] > 0.f) v0 = dout[(size_t)r * kH + j];
      if (r + 1 < rows && out[(size_t)(r + 1) * kH + j] > 0.f) v1 = dout[(size_t)(r + 1) * kH + j];
      accb += v0;
      accb += v1;
      uint32_t th, tm, tl;
      split3(v0, v1, th, tm, tl);
      dT[0][j][rp] = th;
      dT[1][j][rp] = tm;
    }
    for (int e = threadIdx.x; e < (R / 2) * 2 * kH; e += 256) {
      const int rp = e / (2 * kH), k = e % (2 * kH), r = c0 + 2 * rp;
      const float* src = k < kH ? A : Bm;
      const int kk = k < kH ? k : k - kH;
      const float v0 = r < rows ? src[(size_t)r * kH + kk] : 0.f;
      const float v1 = r + 1 < rows ? src[(size_t)(r + 1) * kH + kk] : 0.f;
      uint32_t th, tm, tl;
      split3(v0, v1, th, tm, tl);
      xT[0][k][rp] = th;
      xT[1][k][rp] = tm;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < R / 16; ++ks) {
      const int j = mi * 16 + g;
      uint32_t a[2][4];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        a[p][0] = dT[p][j][8 * ks + t];
        a[p][1] = dT[p][j + 8][8 * ks + t];
        a[p][2] = dT[p][j][8 * ks + 4 + t];
        a[p][3] = dT[p][j + 8][8 * ks + 4 + t];
      }
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int k = nh * 64 + nt * 8 + g;
        const uint32_t bh0 = xT[0][k][8 * ks + t], bh1 = xT[0][k][8 * ks + 4 + t];
        const uint32_t bm0 = xT[1][k][8 * ks + t], bm1 = xT[1][k][8 * ks + 4 + t];
        mma_bf16(acc[nt], a[0], bh0, bh1);
        mma_bf16(acc[nt], a[0], bm0, bm1);
        mma_bf16(acc[nt], a[1], bh0, bh1);
      }
    }
  }
  float* p = part + (size_t)blockIdx.x * (kH * 2 * kH + kH);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int j = mi * 16 + g, k = nh * 64 + nt * 8 + 2 * t;
    p[j * 2 * kH + k] = acc[nt][0];
    p[j * 2 * kH + k + 1] = acc[nt][1];
    p[(j + 8) * 2 * kH + k] = acc[nt][2];
    p[(j + 8) * 2 * kH + k + 1] = acc[nt][3];
  }
  // the four threads of output j combine their bias shares in a fixed order
  __syncthreads();
  float* sb = reinterpret_cast<float*>(&dT[0][0][0]);
  sb[threadIdx.x] = accb;
  __syncthreads();
  if (threadIdx.x < kH)
    p[kH * 2 * kH + threadIdx.x] = ((sb[threadIdx.x] + sb[threadIdx.x + kH]) +
                                    sb[threadIdx.x + 2 * kH]) + sb[threadIdx.x + 3 * kH];
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

// grad[e] = sum over blocks of part[blk][e], e < count; rows of part are
// `stride` apart. One warp per entry: lane l sums blocks l, l + 32, ... in
// order, then a fixed shuffle tree (the same order on every run).
__global__ void k_mp_sum_parts(const float* part, int nblk, int stride, int count, float* grad) {
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (e >= count) return;
  float s = 0.f;
  for (int b = lane; b < nblk; b += 32) s += part[(size_t)b * stride + e];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) grad[e] = s;
}

cudaError_t launch_sum_parts(const float* part, int nblk, int stride, int count, float* grad,
                             cudaStream_t st) {
  k_mp_sum_parts<<<(count + 7) / 8, 256, 0, st>>>(part, nblk, stride, count, grad);
  return cudaGetLastError();
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
  if (rows > 0) k_mp_dense_fwd<<<blocks(rows, 128), 256, 0, st>>>(A, Bm, rows, W, b, out);
  return cudaGetLastError();
}

cudaError_t mp_launch_dense_bwd_x(const float* dout, const float* out, int rows,
                                  const __nv_bfloat16* W, float* dA, float* dB, cudaStream_t st) {
  if (rows > 0) k_mp_dense_bwd_x<<<blocks(rows, 128), 256, 0, st>>>(dout, out, rows, W, dA, dB);
  return cudaGetLastError();
}

cudaError_t mp_launch_dense_wgrad(const float* dout, const float* out, const float* A,
                                  const float* Bm, int rows, float* part, float* gW,
                                  cudaStream_t st) {
  if (rows <= 0) return cudaMemsetAsync(gW, 0, sizeof(float) * (kH * 2 * kH + kH), st);
  k_mp_wgrad_tc<<<blocks(rows, kRowsTc), 256, 0, st>>>(dout, out, A, Bm, rows, part);
  return cudaGetLastError();
}

// sums the weight-gradient partials of mp_launch_dense_wgrad over `rows` rows
cudaError_t mp_launch_dense_wsum(const float* part, int rows, float* gW, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const int width = kH * 2 * kH + kH;
  return launch_sum_parts(part, blocks(rows, kRowsTc), width, width, gW, st);
}

cudaError_t mp_launch_proj_bwd(const float* dout, const float* out, const float* in, int rows,
                               float* part, float* gW, cudaStream_t st) {
  if (rows <= 0) return cudaMemsetAsync(gW, 0, sizeof(float) * kH * 3, st);
  const int nb = blocks(rows, kRowsW);
  k_mp_wgrad_parts<3><<<nb, 256, 0, st>>>(dout, out, in, nullptr, rows, part);
  // the projection has no bias: only the first 64 x 3 entries of each part
  return launch_sum_parts(part, nb, kH * 3 + kH, kH * 3, gW, st);
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
  return launch_sum_parts(part, nb, kH + 1, kH + 1, g_wo, st);  // wo then bo
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
