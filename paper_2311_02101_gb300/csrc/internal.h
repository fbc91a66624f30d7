// Internal declarations shared by the host core and the kernels of
// libmaxsat.so. Not part of the public ABI (include/maxsat.h is).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "maxsat.h"

namespace rbmsat {

// Phase word of the randomness contract: draw (phase, t, a, h, b) is the
// 16-bit lane (b & 7) of Philox4x32-10 at counter (a, (b >> 3) | (h << 24), t,
// phase) under key = seed. a is the variable (initial / visible draws) or the
// clause (hidden draws); h the hidden unit.
enum : uint32_t { kPhaseInit = 1, kPhaseHidden = 2, kPhaseVisible = 3, kPhaseSwap = 4 };

constexpr int kChainTile = 256;   // chains per block of the sparse kernels
constexpr int kClauseBlock = 64;  // clauses per block of the sparse gather

// ---------------------------------------------------------------------------
// Per clause group (length, weight bucket): its table offsets.
// ---------------------------------------------------------------------------
struct GroupMeta {
  int32_t len = 0;      // clause length K
  int32_t nh = 0;       // hidden units L
  int32_t rec_off = 0;  // into rec (u32, a multiple of 4): + (e 2^K + p) stride
  int32_t stride = 0;   // u32 words per pattern record: 4 ceil((L + 1) / 4)
  int32_t gq_off = 0;   // into gq (int16): + (e 2^L + hp) K + k
  int32_t sat = 0;      // 1 when some hidden probability of the group is 65536 / 65536
  int32_t feq_off = 0;  // into feq (int32): + e 2^K + p
  int32_t pad1 = 0;
};

// ---------------------------------------------------------------------------
// Device views passed to kernels by value.
// ---------------------------------------------------------------------------
struct DevFormula {
  int32_t n, m, nnz;
  const int32_t* cl_off;   // m + 1 literal offsets
  const int32_t* lit_var;  // nnz: 0-based variable, bit 31 set when negated
  const int32_t* cl_grp;   // m: clause group (length, bucket); -1 = empty clause
  const int64_t* cl_w;     // m weights
  const int32_t* var_off;  // n + 1 offsets into var_inc
  int32_t n_inst;          // formulas in the batch (1 for a single formula)
  const int2* var_inst;    // n: {instance, index within it}; NULL for one formula
  const int4* var_inc;     // incidence of a variable: {clause, gq_off + position
                           // (+ gq_len and bit 31 set when negated: the
                           // table's negated half), clause length K,
                           // per-temperature stride 2^L K of gq}
  const int4* cl4;         // m clause records {0-based variable of literals
                           // 0..2 (0 when absent), group << 8 | negated << 2 |
                           // length}, bit k of `negated` set when literal k is
                           // negated, when every clause has at most 3
                           // literals (one-chunk tables); else NULL
  const int32_t* var_order;  // n: the visible update's order: variables by
                             // degree, highest first (ties to the lower index),
                             // within windows of 512 variables of one formula
};

// Work list of the clause gather: blocks of consecutive clauses that never
// straddle two formulas of a batch.
struct GatherPlan {
  const int4* blk;          // per block: {instance, first clause, end clause,
                            //             the instance's first clause}
  const int32_t* inst_blk;  // n_inst + 1: first block of each instance
  int32_t n_blk;
};

struct DevTables {
  int32_t n_temps;     // E
  int32_t qmax;        // visible logits clamp to [-qmax, qmax] (units 2^-Q)
  int32_t n_groups;
  int32_t rec_len, gq_len, pv_len;  // element counts
  int32_t one_chunk;   // every group's pattern record is 16 bytes (L <= 3)
  int32_t plain3;      // every clause has exactly 3 literals and no hidden
                       // probability is 65536 / 65536
  const int32_t* feq;  // fixed-point clause free energies (parallel tempering)
  int32_t smem_bytes;  // bytes to stage all tables in shared memory, 0 = too big
  const GroupMeta* meta;
  const uint32_t* rec;
  // one-chunk tables only: the records of group g at temperature e as a
  // 256-byte block at word (g E + e) 64: the 2^K records of 4 words, then at
  // word 32 the group's flags (bit 8: some hidden probability is 65536); NULL
  // when not built (too large)
  const uint32_t* rec3;
  int32_t rec3_words;
  const int16_t* gq;   // 2 gq_len entries: 2^Q G, then -2^Q G (a negated
                       // literal's incidence reads the second half)
  const uint32_t* pv;
};

// Lets kernel `kern` launch with `dyn` bytes of dynamic shared memory: when
// dynamic plus the kernel's static shared memory exceed the default 48 KB per
// block, the launch needs the opt-in attribute.
template <typename K>
cudaError_t allow_dynamic_smem(K kern, int dyn) {
  cudaFuncAttributes fa;
  const cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  if ((size_t)dyn + fa.sharedSizeBytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
}

// Philox round keys of one seed (computed on the host, read by the kernels
// from parameter space).
struct RoundKeys {
  uint32_t k0[10], k1[10];
};

struct DevChains {
  int32_t B;      // chains reported
  int32_t Bp;     // chains allocated (multiple of kChainTile)
  int32_t g8_off;   // global index of local chain 0, divided by 8 (chain shards)
  int32_t B_total;  // chains of the whole ensemble (temperature blocks)
  float inv_B_total;  // 1 / B_total (first guess of the temperature index)
  int32_t cost32;     // sparse gather: every clause block's weight sum < 2^31
  int32_t cost16;     // one-chunk gather: a thread's clauses of one block (its
                      // eighth of the block) weigh less than 2^16 in total
  int32_t n_inst;     // formulas: best / cost / fe / improved are n_inst x Bp,
                      // tickets n_inst x (Bp / kChainTile)
  uint32_t key0, key1;
  RoundKeys keys;
  uint8_t* xt;        // sparse layout: n x Bp, 0/1
  float* nu;          // n x Bp
  int64_t* best;      // Bp
  uint8_t* best_xt;   // n x Bp
  int64_t* cost;      // Bp (last scored)
  float* fe;          // Bp (last scored)
  uint8_t* improved;  // Bp flags of the last best-keep
  int64_t* cost_part; // [clause block][Bp]
  float* fe_part;     // [clause block][Bp]
  void* H;            // m x Bp hidden patterns (uint8_t, or uint16_t when L > 8)
  int32_t* tickets;   // Bp / kChainTile arrival counters of the gather blocks
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
  int32_t n_groups = 0, n_temps = 0, qmax = 0, quant_bits = 0, max_nh = 0;
  std::vector<int32_t> grp_len, grp_bucket, grp_nh;
  std::vector<GroupMeta> meta;
  std::vector<uint32_t> rec;
  std::vector<int32_t> feq;  // rint(2^20 F) per (group, temperature, pattern)
  bool feq_ok = true;        // every entry fits int32
  std::vector<int16_t> gq;
  std::vector<uint32_t> pv;
  int32_t gq_absmax = 0;  // largest |2^Q G|
};

// up.cpp: prioritized unit propagation on the host (Sec. 4.4)
struct UpFormula {
  int32_t n = 0, m = 0;
  std::vector<int64_t> cl_off;   // m + 1
  std::vector<int32_t> lit;      // DIMACS literals
  std::vector<int64_t> occ_off;  // n + 1
  std::vector<int32_t> occ;      // per variable, clause order: clause | sign bit 31
};
void up_prepare(int32_t n, int64_t m, const int64_t* off, const int32_t* lits, UpFormula* F);
// out (B x n) = unit propagation of every row of x (B x n) ranked by nu (B x n)
void up_chains(const UpFormula& F, int32_t B, const uint8_t* x, const float* nu, uint8_t* out,
               int threads);

// up_gpu.cu: unit propagation and the B-of-2B merge on the GPU (sparse path)
struct UpDev {
  int32_t n, m;            // all formulas of the context
  const int32_t* cl_off;   // m + 1
  const int32_t* lit_var;  // nnz (global variable indices)
  const int32_t* occ_off;  // n + 1
  const int32_t* occ;      // per variable, its clauses in clause order
  int32_t n_inst;          // formulas; each has its own B chains
  const int32_t* var_base; // n_inst + 1: first variable of each formula
  const int32_t* cl_base;  // n_inst + 1: first clause of each formula
  int32_t n_max;           // variables of the largest formula
};
// chains per block of the propagation kernel for formulas of at most n_max
// variables (0: a chain's state does not fit in shared memory)
int up_gpu_chains_per_block(int n_max);
// out[v * Bp2 + col0 + b] = unit propagation of chain b of the snapshot, for
// every formula (xs: n x Bp states, nus: n x Bp nu; one warp per formula and
// chain)
cudaError_t launch_up_chains(const UpDev& U, const uint8_t* xs, const float* nus, int Bp, int B,
                             uint8_t* out, int Bp2, int col0, cudaStream_t st);
// cand columns B..2B-1 = xt columns 0..B-1 with variable i set to code[i]
// where code[i] < 2
cudaError_t launch_flip_candidates(const uint8_t* xt, int Bp, const uint8_t* code, int n, int B,
                                   uint8_t* cand, int Bp2, cudaStream_t st);
// cost: per formula k its 2B candidate costs at cost + 2B k (cand columns
// 0..2B-1, n x Bp2); in every formula chain j of xt takes the candidate at
// position B + j of the formula's stable sort by cost descending, and
// nu_out gets nu of the chain it came from. var_inst: NULL for one formula.
cudaError_t launch_up_merge(const int64_t* cost, int n_inst, int B, int32_t* rank, int32_t* perm,
                            const uint8_t* cand, int Bp2, uint8_t* xt, const float* nu,
                            float* nu_out, int Bp, int n, const int2* var_inst,
                            cudaStream_t st);

// mp.cu: the learned proposal's kernels (message passing, hidden size 64)
constexpr int kMpHidden = 64;
constexpr int kMpMaxLayers = 8;
struct MpLayout {  // offsets into the flat FP32 parameter vector
  int L = 0, Wf = 0, Wg = 0, Wc[kMpMaxLayers] = {}, bc[kMpMaxLayers] = {},
      Wv[kMpMaxLayers] = {}, bv[kMpMaxLayers] = {}, wo = 0, bo = 0, total = 0;
};
int mp_layout(int L, MpLayout* out);
}  // namespace rbmsat
#include <cuda_bf16.h>
namespace rbmsat {
cudaError_t mp_launch_features(const DevFormula& F, float* f, float* g, float* inv_len,
                               float* inv_deg, cudaStream_t st);
cudaError_t mp_launch_proj(const float* in, int rows, const __nv_bfloat16* W, float* out,
                           cudaStream_t st);
cudaError_t mp_launch_clause_agg(const DevFormula& F, const float* h, const float* cscale,
                                 const float* vscale, float* out, bool acc, cudaStream_t st);
cudaError_t mp_launch_var_agg(const DevFormula& F, const float* h, const float* cscale,
                              const float* vscale, float* out, bool acc, cudaStream_t st);
cudaError_t mp_launch_dense_fwd(const float* A, const float* Bm, int rows, const __nv_bfloat16* W,
                                const float* b, float* out, cudaStream_t st);
// gW receives 64 x 128 weight gradients followed by the 64 bias gradients
cudaError_t mp_launch_dense_bwd_x(const float* dout, const float* out, int rows,
                                  const __nv_bfloat16* W, float* dA, float* dB, cudaStream_t st);
cudaError_t mp_launch_dense_wgrad(const float* dout, const float* out, const float* A,
                                  const float* Bm, int rows, float* part, float* gW,
                                  cudaStream_t st);
cudaError_t mp_launch_dense_wsum(const float* part, int rows, float* gW, cudaStream_t st);
cudaError_t mp_launch_proj_bwd(const float* dout, const float* out, const float* in, int rows,
                               float* part, float* gW, cudaStream_t st);
cudaError_t mp_launch_out(const float* h, int n, const float* wo, const float* bo,
                          const uint8_t* y, float* prob, float* dz, double* loss_part,
                          cudaStream_t st);
cudaError_t mp_launch_out_bwd(const float* h, const float* dz, int n, const float* wo, float* dh,
                              float* part, float* g_wo, cudaStream_t st);
cudaError_t mp_launch_adam(float* P, const float* G, float* M, float* V, int count, float lr,
                           float b1, float b2, float eps, int step, __nv_bfloat16* Pb,
                           cudaStream_t st);
cudaError_t mp_launch_to_bf16(const float* P, __nv_bfloat16* Pb, int count, cudaStream_t st);
cudaError_t launch_init_probs_sparse(const DevFormula& F, const DevChains& C, const uint32_t* P,
                                     cudaStream_t st);
cudaError_t launch_init_probs_dense(int n, int n_pad, const DevChains& C, const uint32_t* P,
                                    uint8_t* X, uint8_t* best_x, uint8_t one, uint8_t minus_one,
                                    cudaStream_t st);

// pt.cu: parallel-tempering swap rounds (sparse layout)
cudaError_t launch_pt_round(const DevFormula& F, const DevTables& T, const DevChains& C, int S,
                            int E, int parity, uint32_t t, const long long* Tc, long long* Fown,
                            long long* Foth, uint8_t* flag, int* n_acc, cudaStream_t st);

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
// clauses per block for the step / score gathers over `tiles` chain tiles:
// the block count tiles * ceil(m / cb) is fitted to whole waves of `slots`
// resident blocks (SMs x blocks per SM)
int gather_clause_block(int m, int tiles, int slots);
// resident gather blocks per SM for the tables' shared-memory footprint
int gather_blocks_per_sm(const DevTables& T, bool wide_h);

// sparse.cu launchers (all asynchronous on `st`)
enum GatherMode { kStep = 0, kScore = 1, kEval = 2 };
cudaError_t launch_init_sparse(const DevFormula& F, const DevChains& C, int n, cudaStream_t st);
// kStep: cost, free energy, hidden draws, then (last block of each instance
// and chain tile) best-keep; kScore: the same without draws; kEval: cost only,
// written to eval_out (n_inst x B). xt / Bp / B / tickets / partials may
// differ from C's (eval). Grid: chain tiles x P.n_blk.
cudaError_t launch_gather(GatherMode mode, const DevFormula& F, const DevTables& T,
                          const DevChains& C, const uint8_t* xt, int B, int Bp,
                          const GatherPlan& P, const uint32_t* tdev, uint32_t t_rel,
                          int64_t* cost_part, float* fe_part, int32_t* tickets,
                          int64_t* eval_out, bool wide_h, cudaStream_t st);
// batch: incidences per thread whose hidden-pattern loads are in flight
// together (2, 4 or 8)
cudaError_t launch_visible(const DevFormula& F, const DevTables& T, const DevChains& C,
                           float alpha, const uint32_t* tdev, uint32_t t_rel, bool wide_h,
                           cudaStream_t st, int batch = 4);
// the persistent round (one cooperative launch of `rounds` Gibbs rounds,
// grid barriers between the phases) covers this context's sparse round:
// clauses of at most 3 literals, single-temperature octets, byte patterns
bool persistent_round_supported(const DevTables& T, const DevChains& C, const DevFormula& F,
                                bool wide_h);
constexpr int kMaxPersistentRounds = 1 << 16;
// rounds t0 .. t0 + rounds - 1 (absolute indices); bar: 2 device words,
// zeroed on st before the launch; err: device error code (16 = a grid
// barrier wait gave up after about 2 s)
cudaError_t launch_round_persistent(const DevFormula& F, const DevTables& T, const DevChains& C,
                                    const GatherPlan& P, uint32_t t0, int rounds, float alpha,
                                    uint32_t* bar, int* err, cudaStream_t st);
cudaError_t launch_keep_copy(const DevFormula& F, const DevChains& C, int n, cudaStream_t st);
cudaError_t launch_advance(uint32_t* tdev, uint32_t by, cudaStream_t st);
cudaError_t launch_set_u32(uint32_t* dst, uint32_t value, cudaStream_t st);
cudaError_t launch_transpose_in(const uint8_t* assign, int B, int n, uint8_t* xt, int Bp,
                                cudaStream_t st);

// dense.cu: tensor-core path
bool fp8_encode_int(int v, bool e5m2, uint8_t* out);
std::string build_gather_matrix(int n, int m, const int64_t* off, const int32_t* lits,
                                bool* e5m2, int* n_pad, int* m_pad, std::vector<uint8_t>* A);
std::string make_tmap_2d(CUtensorMap* tm, const void* base, uint64_t inner, uint64_t rows,
                         uint64_t row_bytes, uint32_t box_inner, uint32_t box_rows, bool bf16);
// adds every chain's weighted unsatisfied cost into out (B, zeroed by
// launch_assign_fp8, which must be the launch just before it on st); lets
// the next launch on st start early (the next evaluation's conversion, into
// the other state buffer)
cudaError_t launch_gemm1_eval(const CUtensorMap& tmA, const CUtensorMap& tmB, int m, int m_pad,
                              int n_pad, int B, int Bp, bool e5m2, const int32_t* row_len,
                              const int64_t* row_w, const uint8_t* grp_small, int64_t* out,
                              int* err, cudaStream_t st);
// assignments -> FP8 B operand X; zeroes cost (B)
cudaError_t launch_assign_fp8(const uint8_t* assign, int B, int n, int Bp, int n_pad, bool e5m2,
                              uint8_t* X, int64_t* cost, cudaStream_t st);

// dense_step.cu: the dense Gibbs round
cudaError_t launch_gemm1_step(bool sample, const CUtensorMap& tmA, const CUtensorMap& tmB, int m,
                              int m_pad, int n_pad, int B, int Bp, bool e5m2,
                              const int32_t* row_len, const int64_t* row_w, const int32_t* cl_grp,
                              const uint8_t* grp_same, int64_t* cost_part, float* fe_part, void* H,
                              bool wide, const uint32_t* tdev, uint32_t t_rel, int* err,
                              const DevTables& T, const DevChains& C, cudaStream_t st);
cudaError_t launch_keep_dense(const int64_t* cost_part, const float* fe_part, int tiles_m,
                              const DevChains& C, cudaStream_t st);
cudaError_t launch_gemm2(const CUtensorMap& tmA2, int n, int n_pad, int B, int Bp, int tiles_v,
                         const int32_t* kstart, const int32_t* kblocks, const int4* var_inc,
                         const uint16_t* gq16, const void* H, bool wide, uint8_t* X, float* nu,
                         uint8_t* best_x,
                         bool e5m2, bool bf16, float alpha, const uint32_t* tdev, uint32_t t_rel,
                         int* err, const DevTables& T, const DevChains& C, cudaStream_t st);
cudaError_t launch_init_dense(const DevChains& C, uint8_t* X, float* nu, uint8_t* best_x, int n,
                              int n_pad, bool e5m2, cudaStream_t st);
cudaError_t launch_keep_copy_dense(const DevChains& C, const uint8_t* X, uint8_t* best_x, int n,
                                   int n_pad, bool e5m2, cudaStream_t st);

#ifdef __CUDACC__
// Temperature of global chain b among E contiguous blocks of B chains:
// floor(b E / B) (capped at E - 1). A float product gives the quotient to
// within one; exact 64-bit products correct it.
__device__ __forceinline__ int temp_of(int b, int E, int B, float inv_B) {
  int e = __float2int_rz((float)b * (float)E * inv_B);
  const long long num = (long long)b * E;
  if ((long long)(e + 1) * B <= num) ++e;
  else if ((long long)e * B > num) --e;
  return e < E - 1 ? e : E - 1;
}
#endif

}  // namespace rbmsat
