// Internal declarations shared by the host core and the kernels of
// libmaxsat.so. Not part of the public ABI (include/maxsat.h is).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "maxsat.h"

namespace rbmsat {

// Phase word of the randomness contract: draw (phase, t, a, h, b) is the
// 16-bit lane (b & 7) of Philox4x32-10 at counter (a, (b >> 3) | (h << 24), t,
// phase) under key = seed. a is the variable (initial / visible draws) or the
// clause (hidden draws); h the hidden unit.
enum : uint32_t { kPhaseInit = 1, kPhaseHidden = 2, kPhaseVisible = 3 };

constexpr int kChainTile = 256;   // chains per block of the sparse kernels
constexpr int kClauseBlock = 64;  // clauses per block of the sparse gather

// ---------------------------------------------------------------------------
// Device views passed to kernels by value.
// ---------------------------------------------------------------------------
struct DevFormula {
  int32_t n, m, nnz;
  const int32_t* cl_off;   // m + 1 literal offsets
  const int32_t* lit_var;  // nnz: 0-based variable, bit 31 set when negated
  const int32_t* cl_grp;   // m: clause group (length, bucket); -1 = empty clause
  const int64_t* cl_w;     // m weights
  const int32_t* var_off;  // n + 1 offsets into var_lit
  const int32_t* var_lit;  // nnz: literal index, bit 31 set when negated
};

struct DevTables {
  int32_t n_temps;     // E
  int32_t qmax;        // visible logits clamp to [-qmax, qmax] (units 2^-Q)
  const int32_t* grp_nh;    // per group: hidden units L
  const int32_t* phid_off;  // per set s = g * E + e: offset into phid
  const int32_t* fe_off;    // per set: offset into fe
  const int32_t* gq_off;    // per set: offset into gq
  const uint32_t* phid;     // [pattern][h]: 65536 sigma(b_h + sum_k W_kh tau_k), rint
  const float* fe;          // [pattern]: clause free energy (Eq. 1)
  const int16_t* gq;        // [hidden pattern][k]: 2^Q sum_h W_kh h_h
  const uint32_t* pv;       // [q + qmax]: 65536 sigma(q 2^-Q), rint
};

struct DevChains {
  int32_t B;      // chains reported
  int32_t Bp;     // chains allocated (multiple of kChainTile)
  uint32_t key0, key1;
  uint8_t* xt;        // sparse layout: n x Bp, 0/1
  float* nu;          // n x Bp
  int64_t* best;      // Bp
  uint8_t* best_xt;   // n x Bp
  int64_t* cost;      // Bp (last scored)
  float* fe;          // Bp (last scored)
  uint8_t* improved;  // Bp flags of the last best-keep
  int64_t* cost_part; // [clause block][Bp]
  float* fe_part;     // [clause block][Bp]
  int16_t* G;         // nnz x Bp: 2^Q G per literal and chain
};

// ---------------------------------------------------------------------------
// Host-side parameter sets and tables
// ---------------------------------------------------------------------------
struct RbmSet {
  int32_t len = 0, bucket = 0, temp = 0, nh = 0;
  std::vector<double> W;  // len x nh
  std::vector<double> b;  // nh
};

struct HostTables {
  int32_t n_groups = 0, n_temps = 0, qmax = 0, quant_bits = 0;
  std::vector<int32_t> grp_len, grp_bucket, grp_nh;
  std::vector<int32_t> phid_off, fe_off, gq_off;
  std::vector<uint32_t> phid;
  std::vector<float> fe;
  std::vector<int16_t> gq;
  std::vector<uint32_t> pv;
  int32_t gq_absmax = 0;  // largest |2^Q G|
};

// fit.cpp
int fit_or_rbm(int len, int nh, double fstar, int quant_bits, int iters, double* W,
               double* b);
int hidden_units_for(int len);

// tables.cpp: builds the per-set tables; returns "" or an error message.
std::string build_tables(const std::vector<RbmSet>& sets, int n_temps, int quant_bits,
                         const std::vector<int32_t>& grp_len,
                         const std::vector<int32_t>& grp_bucket, HostTables* out);

// message returned by maxsat_last_error(NULL) (context-free calls)
void set_context_free_error(const std::string& msg);

// clause blocking of the sparse gather: clauses per block and block count
int clause_block_for(int m);
int clause_blocks_for(int m);

// sparse.cu launchers (all asynchronous on `st`)
cudaError_t launch_init_sparse(const DevChains& C, int n, cudaStream_t st);
cudaError_t launch_gather(const DevFormula& F, const DevTables& T, const DevChains& C,
                          const uint8_t* xt, int Bp, bool sample, bool free_energy,
                          const uint32_t* tdev, uint32_t t_rel, int64_t* cost_part,
                          float* fe_part, cudaStream_t st);
cudaError_t launch_best_keep(const DevFormula& F, const DevChains& C, cudaStream_t st);
cudaError_t launch_visible(const DevFormula& F, const DevTables& T, const DevChains& C,
                           float alpha, const uint32_t* tdev, uint32_t t_rel,
                           cudaStream_t st);
cudaError_t launch_keep_copy(const DevChains& C, int n, cudaStream_t st);
cudaError_t launch_advance(uint32_t* tdev, uint32_t by, cudaStream_t st);
cudaError_t launch_set_u32(uint32_t* dst, uint32_t value, cudaStream_t st);
cudaError_t launch_transpose_in(const uint8_t* assign, int B, int n, uint8_t* xt, int Bp,
                                cudaStream_t st);
cudaError_t launch_reduce_cost(const int64_t* cost_part, int nblk, int Bp, int B,
                               int64_t* cost_out, cudaStream_t st);

}  // namespace rbmsat
