// Host core of libmaxsat.so: the C ABI of include/maxsat.h.
//
// maxsat_create ingests the signed-literal formula (the index table T of
// Sec. 4.3), assigns every clause to a group (length, weight bucket), fits or
// accepts the OR-gate clause RBMs (Sec. 4.1), builds the probability and
// free-energy tables and copies everything to the device. The Gibbs rounds
// (Sec. 4.2-4.4) then run entirely in the kernels of sparse.cu / dense.cu,
// launched on the caller's stream, optionally replayed from a CUDA graph of
// `steps_per_graph` rounds (the paper dispatches 500 rounds at a time,
// appendix "Batching operations").
#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>
#include <numeric>

#include "internal.h"
#include "philox.cuh"

using namespace rbmsat;

namespace {

thread_local std::string g_create_error;

// An NVTX range over a scope (entry points and kernel launches), so that a
// profiler's timeline (ncu --nvtx, Nsight Systems) groups the work by call;
// without an attached tool each push and pop is a no-op call.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device blocks freed by contexts, kept per device for later contexts:
// cudaMalloc and cudaFree take tens of microseconds each (and cudaFree waits
// for the device), which dominates short solves that create and destroy a
// context around a few Gibbs rounds. A request takes the smallest cached
// block of at least its size and at most twice it; blocks beyond 4 GiB of
// cache per device go back to the driver.
class BlockCache {
 public:
  static constexpr int kMaxDevices = 64;
  static constexpr size_t kCap = size_t(4) << 30;
  void* get(int dev, size_t bytes, size_t* got) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(mu_);
    auto& f = free_[dev];
    auto it = f.lower_bound(bytes);
    if (it == f.end() || it->first > 2 * bytes) return nullptr;
    void* p = it->second;
    *got = it->first;
    cached_[dev] -= it->first;
    f.erase(it);
    return p;
  }
  // the caller guarantees that no device work still uses p
  void put(int dev, void* p, size_t bytes) {
    if (dev >= 0 && dev < kMaxDevices) {
      std::lock_guard<std::mutex> lock(mu_);
      if (cached_[dev] + bytes <= kCap) {
        free_[dev].emplace(bytes, p);
        cached_[dev] += bytes;
        return;
      }
    }
    cudaFree(p);
  }

 private:
  std::mutex mu_;
  std::multimap<size_t, void*> free_[kMaxDevices];
  size_t cached_[kMaxDevices] = {};
};

BlockCache& block_cache() {
  static BlockCache* c = new BlockCache();  // kept until exit: no teardown order issues
  return *c;
}

struct DevAllocs {
  struct Block {
    void* p;
    size_t bytes;
    int dev;
  };
  std::vector<Block> blocks;
  ~DevAllocs() { release(); }
  // returns the blocks to the cache once the device is idle (as cudaFree would
  // wait): work still queued on any stream may use them
  void release() {
    if (blocks.empty()) return;
    cudaDeviceSynchronize();
    for (const Block& b : blocks) block_cache().put(b.dev, b.p, b.bytes);
    blocks.clear();
  }
  template <class T>
  cudaError_t alloc(T** out, size_t count) {
    const size_t bytes = (std::max<size_t>(count, 1) * sizeof(T) + 511) / 512 * 512;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    size_t got = bytes;
    void* p = block_cache().get(dev, bytes, &got);
    if (!p) {
      e = cudaMalloc(&p, bytes);
      if (e != cudaSuccess) return e;
    }
    blocks.push_back(Block{p, got, dev});
    *out = static_cast<T*>(p);
    return cudaSuccess;
  }
};

}  // namespace

namespace rbmsat {
void set_context_free_error(const std::string& msg) { g_create_error = msg; }
}  // namespace rbmsat

struct maxsat_ctx {
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
  int path = MAXSAT_PATH_SPARSE;
  int32_t n = 0, m = 0, nnz = 0;
  maxsat_params prm{};
  std::vector<double> fstar;
  HostTables tabs;
  int max_degree = 0;

  DevAllocs formula_mem;  // formula + tables (lifetime of the context)
  DevAllocs chain_mem;    // chain state (re-made when B changes)
  DevAllocs eval_mem;     // eval scratch (grown on demand)
  DevAllocs dense_eval_mem;  // dense eval scratch (grown on demand)
  DevFormula F{};
  DevTables T{};
  DevChains C{};
  bool have_chains = false;
  uint32_t t = 0;
  uint64_t seed = 0;
  uint32_t* d_t = nullptr;  // round index read by graph-replayed kernels
  bool d_t_synced = false;

  uint8_t* ev_xt = nullptr;
  int64_t* ev_part = nullptr;
  int32_t* ev_tickets = nullptr;
  int ev_Bp = 0;
  std::vector<int64_t> h_w;  // clause weights (host copy)
  // parallel tempering: Metropolis thresholds and per-round scratch
  DevAllocs pt_mem;
  long long *d_Tc = nullptr, *d_Fown = nullptr, *d_Foth = nullptr;
  uint8_t* d_swap = nullptr;
  int* d_nacc = nullptr;
  int pt_Bp = 0;
  // unit-propagation heuristic (Sec. 4.4): host formula, worker, results
  UpFormula upf;
  std::thread up_worker;
  bool up_pending = false;
  int up_B = 0;
  std::vector<uint8_t> up_x0, up_out;  // snapshot of the states, propagated states
  std::vector<float> up_nu0;           // snapshot of nu (the ranking keys)
  DevAllocs up_mem;                    // device candidates and their costs
  uint8_t* d_up_cand = nullptr;
  int64_t* d_up_cost = nullptr;
  size_t up_cap = 0;
  // unit propagation on the GPU (sparse path): occurrence lists, snapshot,
  // candidates (n x Bp2: current states, then propagated ones), their costs
  // and the merge permutation; a side stream with its events
  bool up_on_gpu = false;  // the pending round runs on the GPU
  DevAllocs upg_formula;
  int32_t* d_occ_off = nullptr;
  int32_t* d_occ = nullptr;
  int32_t* d_inst_var_base = nullptr;  // n_inst + 1 (device copies of the batch layout)
  int32_t* d_inst_cl_base = nullptr;
  DevAllocs upg_mem;
  int upg_Bp = 0;
  uint8_t* d_upg_xs = nullptr;
  float* d_upg_nus = nullptr;
  uint8_t* d_upg_cand = nullptr;
  int64_t* d_upg_cost = nullptr;
  int32_t* d_upg_perm = nullptr;
  int32_t* d_upg_rank = nullptr;
  uint8_t* d_flip_code = nullptr;  // flip proposals: per variable 0 / 1 / 2 = keep
  cudaStream_t up_stream = nullptr;
  cudaEvent_t up_ev_snap = nullptr, up_ev_done = nullptr;
  int n_inst = 1;                      // formulas in the batch
  std::vector<int32_t> inst_var_base;  // n_inst + 1 first variable of each formula
  std::vector<int32_t> inst_cl_base;   // n_inst + 1 first clause of each formula
  GatherPlan plan{};                   // clause blocks of the step / score gathers
  GatherPlan ev_plan{};                // clause blocks of the sparse eval
  int gather_slots = 0;  // SMs x resident gather blocks per SM
  int gather_cb = 0;     // clauses per gather block for the chains' Bp
  int cb_force = 0;      // clause block used instead of the wave-fitted one (0 = none)
  int vis_batch = 4;     // visible update: incidences whose loads are in flight together
  int tuned_B = 0;       // B of the last measured clause-block choice
  std::vector<std::pair<int, float>> tune_ms;  // measured (clause block, ms per round)
  std::vector<std::pair<int, float>> tune_vis_ms;  // measured (visible batch, ms per round)
  bool wide_h = false;  // hidden patterns need 16 bits (some group has L > 8)

  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;

  // dense tensor-core path (built when requested or for the measured choice)
  DevAllocs dense_mem;
  bool dense_built = false;  // dense operands exist
  // MAXSAT_PATH_AUTO builds the dense operands only when its measurement
  // needs them; until then it keeps the host inputs of that build
  bool dense_pending = false;
  std::vector<int64_t> lazy_off;
  std::vector<int32_t> lazy_lits, lazy_var_off;
  std::vector<int4> lazy_var_inc;
  bool dense = false;        // Gibbs rounds run on the dense path
  bool chains_dense = false; // layout of the allocated chain state
  int auto_B = 0;            // B of the last measured choice (AUTO)
  float auto_ms[2] = {0, 0}; // measured ms per round: sparse, dense
  bool e5m2 = false;
  int n_pad = 0, m_pad = 0;
  uint8_t* dA = nullptr;          // m_pad x n_pad FP8 pattern-encoding gather matrix
  int32_t* d_row_len = nullptr;   // m_pad clause lengths (0 for padding rows)
  int64_t* d_row_w = nullptr;     // m_pad weights (0 for padding rows)
  uint8_t* d_grp_small = nullptr; // per 32-row group: 1 when its rows share one weight
  CUtensorMap tmA{};
  uint8_t* dXe[2] = {nullptr, nullptr};  // eval scratch: two Bp x n_pad FP8 state buffers
  int dev_Bp = 0;
  CUtensorMap tmXe[2] = {};
  int ev_buf = 0;                 // state buffer of the next evaluation
  int* d_err = nullptr;           // device wait-timeout code (0 = none)
  uint32_t* d_bar = nullptr;      // persistent round: grid-barrier arrivals and give-up flag
  bool persist_ran = false;       // some maxsat_step ran persistent launches (read d_err)
  // dense scatter-add (GEMM2): block-diagonal variable x incidence matrix
  int tiles_v = 0, kmax = 0;
  bool g_bf16 = true;             // G operand BF16 (else FP16)
  int32_t* d_kstart = nullptr;    // tiles_v + 1
  int32_t* d_kblocks = nullptr;   // tiles_v
  uint16_t* d_gq16 = nullptr;     // contribution table as BF16 / FP16 bits
  CUtensorMap tmA2{};
  // dense chain state
  uint8_t* dX = nullptr;          // Bp x n_pad FP8 +-1
  float* dnu = nullptr;           // Bp x n_pad
  uint8_t* dbest_x = nullptr;     // Bp x n_pad 0/1
  int64_t* dcost_part = nullptr;  // tiles_m x Bp
  float* dfe_part = nullptr;      // tiles_m x Bp
  CUtensorMap tmX{};

  // per-kernel CUDA-event timing of plain launches
  bool profiling = false;
  struct Mark {
    int kernel;  // index into prof_names
    cudaEvent_t start, stop;
  };
  std::vector<Mark> marks;
  std::vector<std::string> prof_names;
  std::vector<double> prof_ms;
  std::vector<int64_t> prof_count;

  std::string err;
};

namespace {

int fail(maxsat_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(maxsat_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? MAXSAT_ENOMEM : MAXSAT_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(ctx, call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

int check_device(maxsat_ctx* ctx) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(ctx, MAXSAT_ENODEV, std::string("no CUDA device: ") + cudaGetErrorString(e));
  cudaDeviceProp prop{};
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return fail(ctx, MAXSAT_ENODEV, cudaGetErrorString(e));
  if (prop.major != 10 || prop.minor != 3)
    return fail(ctx, MAXSAT_ENODEV,
                "libmaxsat is built for sm_103 (GB300); device is sm_" +
                    std::to_string(prop.major) + std::to_string(prop.minor));
  return MAXSAT_OK;
}

void destroy_graph(maxsat_ctx* ctx) {
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  ctx->graph = nullptr;
  ctx->graph_steps = 0;
}

int32_t weight_bucket(int64_t w, int64_t wmin, int32_t J) {
  int32_t j = 0;
  while (j + 1 < J && wmin <= (INT64_MAX >> (j + 1)) && (wmin << (j + 1)) <= w) ++j;
  return j;
}

// Launches `body` on `st`, bracketed by CUDA events when profiling.
template <class Fn>
int timed(maxsat_ctx* ctx, cudaStream_t st, const char* name, Fn body) {
  NvtxRange range(name);
  if (!ctx->profiling) {
    const cudaError_t e = body();
    if (e != cudaSuccess) return cuda_fail(ctx, e, name);
    return MAXSAT_OK;
  }
  int k = 0;
  while (k < (int)ctx->prof_names.size() && ctx->prof_names[k] != name) ++k;
  if (k == (int)ctx->prof_names.size()) {
    ctx->prof_names.push_back(name);
    ctx->prof_ms.push_back(0.0);
    ctx->prof_count.push_back(0);
  }
  maxsat_ctx::Mark mk{k, nullptr, nullptr};
  CK(ctx, cudaEventCreate(&mk.start));
  CK(ctx, cudaEventCreate(&mk.stop));
  ctx->marks.push_back(mk);
  CK(ctx, cudaEventRecord(mk.start, st));
  const cudaError_t e = body();
  if (e != cudaSuccess) return cuda_fail(ctx, e, name);
  CK(ctx, cudaEventRecord(mk.stop, st));
  return MAXSAT_OK;
}

#define TIMED(ctx, st, name, expr)                                   \
  do {                                                               \
    int rc_ = timed(ctx, st, name, [&]() { return (expr); });        \
    if (rc_ != MAXSAT_OK) return rc_;                                \
  } while (0)

// One Gibbs round: absolute index t = (tdev ? *tdev : 0) + t_rel.
int launch_round(maxsat_ctx* ctx, cudaStream_t st, const uint32_t* tdev, uint32_t t_rel) {
  const DevChains& C = ctx->C;
  if (ctx->dense) {
    TIMED(ctx, st, "gemm1_step",
          launch_gemm1_step(true, ctx->tmA, ctx->tmX, ctx->m, ctx->m_pad, ctx->n_pad, C.B, C.Bp,
                            ctx->e5m2, ctx->d_row_len, ctx->d_row_w, ctx->F.cl_grp,
                            ctx->d_grp_small, ctx->dcost_part, ctx->dfe_part, C.H, ctx->wide_h,
                            tdev, t_rel, ctx->d_err, ctx->T, C, st));
    TIMED(ctx, st, "keep", launch_keep_dense(ctx->dcost_part, ctx->dfe_part, ctx->m_pad / 128, C, st));
    TIMED(ctx, st, "gemm2",
          launch_gemm2(ctx->tmA2, ctx->n, ctx->n_pad, C.B, C.Bp, ctx->tiles_v, ctx->d_kstart,
                       ctx->d_kblocks, ctx->F.var_inc, ctx->d_gq16, C.H, ctx->wide_h, ctx->dX, ctx->dnu,
                       ctx->dbest_x, ctx->e5m2, ctx->g_bf16, (float)ctx->prm.alpha, tdev, t_rel,
                       ctx->d_err, ctx->T, C, st));
    return MAXSAT_OK;
  }
  TIMED(ctx, st, "gather_hidden",
        launch_gather(kStep, ctx->F, ctx->T, C, C.xt, C.B, C.Bp, ctx->plan, tdev, t_rel,
                      C.cost_part, C.fe_part, C.tickets, nullptr, ctx->wide_h, st));
  TIMED(ctx, st, "visible",
        launch_visible(ctx->F, ctx->T, C, (float)ctx->prm.alpha, tdev, t_rel, ctx->wide_h, st,
                       ctx->vis_batch));
  return MAXSAT_OK;
}

int capture_graph(maxsat_ctx* ctx, int S) {
  destroy_graph(ctx);
  if (!ctx->cap_stream) CK(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  CK(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = MAXSAT_OK;
  for (int s = 0; s < S && rc == MAXSAT_OK; ++s) rc = launch_round(ctx, ctx->cap_stream, ctx->d_t, (uint32_t)s);
  if (rc == MAXSAT_OK) {
    cudaError_t e = launch_advance(ctx->d_t, (uint32_t)S, ctx->cap_stream);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "launch_advance");
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
  if (rc != MAXSAT_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&ctx->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
  ctx->graph_steps = S;
  return MAXSAT_OK;
}

// Clause blocks of at most cb clauses that never straddle two formulas of
// the batch (a formula without clauses still gets one empty block, so its
// costs are written); uploaded into A. *wmax receives the largest weight sum
// of a block.
// Clause blocks of one formula of mk clauses for the nominal size cb: as many
// as cb gives, but no more than its groups of 8 clauses.
static int64_t blocks_of(int64_t mk, int cb) {
  return std::max<int64_t>(1, std::min<int64_t>((mk + cb - 1) / cb, (mk + 7) / 8));
}

int plan_blocks(const maxsat_ctx* ctx, int cb) {
  int64_t nb = 0;
  for (int in = 0; in < ctx->n_inst; ++in)
    nb += blocks_of(ctx->inst_cl_base[in + 1] - ctx->inst_cl_base[in], cb);
  return (int)std::min<int64_t>(nb, INT32_MAX);
}

// Clause blocks of about cb clauses per instance. *wmax: the largest weight
// sum of a block; *wmax8 (optional): the largest weight sum of the clauses
// one warp of the one-chunk gather takes (every eighth clause of a block).
int upload_plan(maxsat_ctx* ctx, DevAllocs& A, int cb, GatherPlan* P, int64_t* wmax,
                int64_t* wmax8 = nullptr) {
  // one grid row per block: at most 65535 blocks
  while (plan_blocks(ctx, cb) > 65535 && cb < (1 << 29)) cb *= 2;
  if (plan_blocks(ctx, cb) > 65535) return fail(ctx, MAXSAT_EINVAL, "too many clause blocks");
  std::vector<int4> blk;
  std::vector<int32_t> ib(1, 0);
  *wmax = 0;
  if (wmax8) *wmax8 = 0;
  for (int in = 0; in < ctx->n_inst; ++in) {
    const int c0 = ctx->inst_cl_base[in], c1 = ctx->inst_cl_base[in + 1];
    // block sizes in whole groups of 8 clauses (a block's 8 warps then take
    // equal counts), as even as possible, the larger ones first
    const int64_t nb = blocks_of(c1 - c0, cb);
    const int64_t groups = (c1 - c0 + 7) / 8;
    int c = c0;
    for (int64_t k = 0; k < nb; ++k) {
      const int64_t g = groups / nb + (k < groups % nb ? 1 : 0);
      const int e = (int)std::min<int64_t>(c1, c + 8 * g);
      blk.push_back(make_int4(in, c, e, c0));
      int64_t sum = 0, part[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int q = c; q < e; ++q) {
        sum += ctx->h_w[q];
        part[(q - c) & 7] += ctx->h_w[q];
      }
      *wmax = std::max(*wmax, sum);
      if (wmax8)
        for (int64_t v : part) *wmax8 = std::max(*wmax8, v);
      c = e;
    }
    ib.push_back((int32_t)blk.size());
  }
  int4* dblk = nullptr;
  int32_t* dib = nullptr;
  CK(ctx, A.alloc(&dblk, blk.size()));
  CK(ctx, A.alloc(&dib, ib.size()));
  CK(ctx, cudaMemcpy(dblk, blk.data(), sizeof(int4) * blk.size(), cudaMemcpyHostToDevice));
  CK(ctx, cudaMemcpy(dib, ib.data(), sizeof(int32_t) * ib.size(), cudaMemcpyHostToDevice));
  P->blk = dblk;
  P->inst_blk = dib;
  P->n_blk = (int32_t)blk.size();
  return MAXSAT_OK;
}

int alloc_chains(maxsat_ctx* ctx, int32_t B) {
  if (ctx->have_chains && ctx->C.B == B && ctx->chains_dense == ctx->dense) return MAXSAT_OK;
  destroy_graph(ctx);
  ctx->chain_mem.release();
  ctx->have_chains = false;
  const int Bp = (B + kChainTile - 1) / kChainTile * kChainTile;
  const size_t nB = (size_t)ctx->n * Bp;
  if (ctx->gather_slots == 0) {
    int dev = 0, sms = 0;
    CK(ctx, cudaGetDevice(&dev));
    CK(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ctx->gather_slots = std::max(sms, 1) * gather_blocks_per_sm(ctx->T, ctx->wide_h);
  }
  ctx->gather_cb = ctx->cb_force > 0 ? ctx->cb_force
                                     : gather_clause_block(ctx->m, Bp / kChainTile, ctx->gather_slots);
  DevAllocs& A = ctx->chain_mem;
  int64_t wmax_block = 0, wmax_warp = 0;
  int rcp = upload_plan(ctx, A, ctx->gather_cb, &ctx->plan, &wmax_block, &wmax_warp);
  if (rcp != MAXSAT_OK) return rcp;
  const int nblk = ctx->plan.n_blk;
  const size_t nI = (size_t)ctx->n_inst * Bp;
  DevChains& C = ctx->C;
  C = DevChains{};
  // 32-bit per-block cost rows when no clause block's weight sum reaches 2^31
  C.cost32 = wmax_block < ((int64_t)1 << 31) ? 1 : 0;
  // two chains' costs share a 32-bit register in the one-chunk gather when
  // every warp's weight sum fits 16 bits
  C.cost16 = wmax_warp < 65536 ? 1 : 0;
  C.n_inst = ctx->n_inst;
  C.B = B;
  C.Bp = Bp;
  ctx->chains_dense = ctx->dense;
  if (ctx->dense) {
    const size_t nP = (size_t)ctx->n_pad * Bp;
    const int tiles_m = ctx->m_pad / 128;
    CK(ctx, A.alloc(&ctx->dX, nP));
    CK(ctx, A.alloc(&ctx->dnu, nP));
    CK(ctx, A.alloc(&ctx->dbest_x, nP));
    CK(ctx, A.alloc(&ctx->dcost_part, (size_t)tiles_m * Bp));
    CK(ctx, A.alloc(&ctx->dfe_part, (size_t)tiles_m * Bp));
    CK(ctx, A.alloc(&C.best, Bp));
    CK(ctx, A.alloc(&C.cost, Bp));
    CK(ctx, A.alloc(&C.fe, Bp));
    CK(ctx, A.alloc(&C.improved, Bp));
    uint8_t* H = nullptr;
    CK(ctx, A.alloc(&H, (size_t)std::max(ctx->m, 1) * Bp * (ctx->wide_h ? 2 : 1)));
    C.H = H;
    std::string e = make_tmap_2d(&ctx->tmX, ctx->dX, ctx->n_pad, Bp, ctx->n_pad, 128, 256, false);
    if (!e.empty()) return fail(ctx, MAXSAT_ECUDA, e);
    return MAXSAT_OK;
  }
  CK(ctx, A.alloc(&C.xt, nB));
  CK(ctx, A.alloc(&C.nu, nB));
  CK(ctx, A.alloc(&C.best, nI));
  CK(ctx, A.alloc(&C.best_xt, nB));
  CK(ctx, A.alloc(&C.cost, nI));
  CK(ctx, A.alloc(&C.fe, nI));
  CK(ctx, A.alloc(&C.improved, nI));
  CK(ctx, A.alloc(&C.cost_part, (size_t)nblk * Bp));
  CK(ctx, A.alloc(&C.fe_part, (size_t)nblk * Bp));
  CK(ctx, A.alloc(&C.tickets, (size_t)ctx->n_inst * (Bp / kChainTile)));
  uint8_t* H = nullptr;
  CK(ctx, A.alloc(&H, (size_t)ctx->m * Bp * (ctx->wide_h ? 2 : 1)));
  C.H = H;
  return MAXSAT_OK;
}

// Copies h to a new device buffer padded with zeros to a multiple of 16 bytes
// (kernels stage tables into shared memory 16 bytes at a time).
// Reads the kernels' wait-timeout code (call after synchronising the stream).
int check_device_error(maxsat_ctx* ctx) {
  int code = 0;
  CK(ctx, cudaMemcpy(&code, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (code != 0)
    return fail(ctx, MAXSAT_ECUDA,
                std::string(code == 16 ? "a grid barrier of the persistent round"
                                       : "a tensor-core pipeline wait") +
                    " timed out (code " + std::to_string(code) + "); results are invalid");
  return MAXSAT_OK;
}

template <class T>
int upload(maxsat_ctx* ctx, DevAllocs& A, std::vector<T> h, const T** out) {
  while ((h.size() * sizeof(T)) % 16 != 0 || h.empty()) h.push_back(T{});
  T* d = nullptr;
  CK(ctx, A.alloc(&d, h.size()));
  CK(ctx, cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = d;
  return MAXSAT_OK;
}

}  // namespace

int build_dense(maxsat_ctx* ctx, int32_t n, int64_t m, const int64_t* off, const int32_t* lits,
                const int64_t* weights, const std::vector<int32_t>& var_off,
                const std::vector<int4>& var_inc, std::string* why);

// Lower bound (ms) of one dense Gibbs round of B chains: its two tensor-core
// products alone (the FP8 gather C x states, 2 m_pad n_pad Bp FLOPs, and the
// block-diagonal BF16 scatter-add, 2 Bp x 128 x each 128-variable tile's
// incidence range padded to 64) at the GB300's nominal dense peaks (4.5
// PFLOP/s FP8, 2.25 PFLOP/s BF16 on 152 SMs), scaled to this device's SMs.
double dense_round_lower_bound_ms(const maxsat_ctx* ctx, int32_t B) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 152;
  const double Bp = (double)((B + 255) / 256 * 256);
  const int n = ctx->n;
  const double n_pad = (double)((n + 127) / 128 * 128), m_pad = (double)((ctx->m + 127) / 128 * 128);
  const std::vector<int32_t>& vo = ctx->lazy_var_off;
  double scatter = 0.0;
  for (int v0 = 0; v0 < n; v0 += 128) {
    const int k = vo[std::min(v0 + 128, n)] - vo[v0];
    scatter += 128.0 * 64.0 * std::max(1, (k + 63) / 64);
  }
  const double scale = (double)sms / 152.0;
  return 1e3 * (2.0 * m_pad * n_pad * Bp / (4.5e15 * scale) + 2.0 * Bp * scatter / (2.25e15 * scale));
}

// Measured path choice (MAXSAT_PATH_AUTO): times a few Gibbs rounds of B
// chains on the sparse path, then on the dense path unless its tensor-core
// products alone (at nominal peaks) would take longer than the measured
// sparse round, and keeps the faster. The dense operands are built here, the
// first time the dense path is measured.
int choose_path(maxsat_ctx* ctx, int32_t B) {
  cudaEvent_t e0, e1;
  CK(ctx, cudaEventCreate(&e0));
  CK(ctx, cudaEventCreate(&e1));
  const bool prof = ctx->profiling;
  ctx->profiling = false;
  int rc = MAXSAT_OK;
  ctx->auto_ms[1] = -1.f;  // not measured
  for (int d = 0; d <= 1 && rc == MAXSAT_OK; ++d) {
    if (d == 1) {
      if (ctx->dense_pending &&
          dense_round_lower_bound_ms(ctx, B) >= (double)ctx->auto_ms[0])
        break;  // the dense path cannot win: neither build nor measure it
      if (ctx->dense_pending) {
        std::string why;
        const int drc =
            build_dense(ctx, ctx->n, ctx->m, ctx->lazy_off.data(), ctx->lazy_lits.data(),
                        ctx->h_w.data(), ctx->lazy_var_off, ctx->lazy_var_inc, &why);
        ctx->dense_pending = false;
        std::vector<int64_t>().swap(ctx->lazy_off);
        std::vector<int32_t>().swap(ctx->lazy_lits);
        std::vector<int32_t>().swap(ctx->lazy_var_off);
        std::vector<int4>().swap(ctx->lazy_var_inc);
        if (drc != MAXSAT_OK) {
          ctx->dense_mem.release();  // not exact or too large: sparse only
          break;
        }
        ctx->dense_built = true;
      }
      if (!ctx->dense_built) break;
    }
    ctx->dense = d == 1;
    rc = alloc_chains(ctx, B);
    if (rc != MAXSAT_OK) break;
    ctx->C.keys = philox_keys(0x5EEDu, 0u);
    ctx->C.g8_off = 0;
    ctx->C.B_total = B;
    ctx->C.inv_B_total = 1.0f / (float)B;
    cudaError_t e = ctx->dense ? launch_init_dense(ctx->C, ctx->dX, ctx->dnu, ctx->dbest_x, ctx->n,
                                                   ctx->n_pad, ctx->e5m2, ctx->stream)
                               : launch_init_sparse(ctx->F, ctx->C, ctx->n, ctx->stream);
    if (e != cudaSuccess) {
      rc = cuda_fail(ctx, e, "init");
      break;
    }
    constexpr int kRounds = 3;
    for (int r = 0; r <= kRounds && rc == MAXSAT_OK; ++r) {
      if (r == 1) cudaEventRecord(e0, ctx->stream);
      rc = launch_round(ctx, ctx->stream, nullptr, (uint32_t)r);
    }
    if (rc != MAXSAT_OK) break;
    cudaEventRecord(e1, ctx->stream);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      rc = cuda_fail(ctx, e, "cudaEventSynchronize");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ctx->auto_ms[d] = ms / kRounds;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->profiling = prof;
  if (rc != MAXSAT_OK) return rc;
  ctx->dense = ctx->auto_ms[1] >= 0.f && ctx->auto_ms[1] < ctx->auto_ms[0];
  ctx->auto_B = B;
  // the timing runs left no valid states (the caller, maxsat_reset, initialises
  // them next); the sparse layout's memory stays allocated when it won
  ctx->have_chains = !ctx->dense && !ctx->chains_dense && ctx->C.B == B;
  return MAXSAT_OK;
}

// Measured launch shapes of the sparse round (params.tune_blocks): times 6
// Gibbs rounds for each candidate with CUDA events, in two passes, and keeps
// the fastest minimum. First the gather's clause-block size (the
// wave-fitted size, half and twice it, and the plain m / 256 rule), then,
// with that size, the visible update's load batch (2, 4 or 8 incidences in
// flight per thread). A candidate replaces the default (wave-fitted size,
// batch 4) only for a gain above 2 %.
int tune_blocks(maxsat_ctx* ctx, int32_t B) {
  const int Bp = (B + kChainTile - 1) / kChainTile * kChainTile;
  ctx->cb_force = 0;
  const int vis_fixed = ctx->prm.visible_batch;  // 0: measured below
  ctx->vis_batch = vis_fixed ? vis_fixed : 4;
  if (ctx->gather_slots == 0) {
    int rc0 = alloc_chains(ctx, B);  // sets gather_slots
    if (rc0 != MAXSAT_OK) return rc0;
  }
  const int fit = gather_clause_block(ctx->m, Bp / kChainTile, ctx->gather_slots);
  std::vector<int> cand = {fit, std::max(16, fit / 2), fit * 2, clause_block_for(ctx->m)};
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  cudaEvent_t e0, e1;
  CK(ctx, cudaEventCreate(&e0));
  CK(ctx, cudaEventCreate(&e1));
  const bool prof = ctx->profiling;
  ctx->profiling = false;
  ctx->tune_ms.clear();
  ctx->tune_vis_ms.clear();
  // ms per round of the current shape (fresh chains, 2 warm-up rounds)
  auto time_rounds = [&](float* ms_out) -> int {
    ctx->have_chains = false;
    int r0 = alloc_chains(ctx, B);
    if (r0 != MAXSAT_OK) return r0;
    ctx->C.keys = philox_keys(0x5EEDu, 0u);
    ctx->C.g8_off = 0;
    ctx->C.B_total = B;
    ctx->C.inv_B_total = 1.0f / (float)B;
    cudaError_t e = launch_init_sparse(ctx->F, ctx->C, ctx->n, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "init");
    constexpr int kWarm = 2, kRounds = 6;
    for (int r = 0; r < kWarm + kRounds; ++r) {
      if (r == kWarm) cudaEventRecord(e0, ctx->stream);
      r0 = launch_round(ctx, ctx->stream, nullptr, (uint32_t)r);
      if (r0 != MAXSAT_OK) return r0;
    }
    cudaEventRecord(e1, ctx->stream);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventSynchronize");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_out = ms / kRounds;
    return MAXSAT_OK;
  };
  std::map<int, float> best_of;  // clause block actually used -> fastest ms per round
  int rc = MAXSAT_OK;
  for (int pass = 0; pass < 2 && rc == MAXSAT_OK; ++pass)
    for (int cb : cand) {
      ctx->cb_force = cb;
      float ms = 0.f;
      rc = time_rounds(&ms);
      if (rc != MAXSAT_OK) break;
      ctx->tune_ms.emplace_back(ctx->gather_cb, ms);
      auto it = best_of.find(ctx->gather_cb);
      if (it == best_of.end() || ms < it->second) best_of[ctx->gather_cb] = ms;
    }
  int best = fit;
  if (rc == MAXSAT_OK) {
    float best_ms = best_of.count(fit) ? best_of[fit] : 1e30f;
    for (const auto& kv : best_of)
      if (kv.second < 0.98f * best_ms) {
        best_ms = kv.second;
        best = kv.first;
      }
  }
  ctx->cb_force = best;
  std::map<int, float> vis_of;  // visible batch -> fastest ms per round
  for (int pass = 0; pass < 2 && rc == MAXSAT_OK && !vis_fixed; ++pass)
    for (int vb : {2, 4, 8}) {
      ctx->vis_batch = vb;
      float ms = 0.f;
      rc = time_rounds(&ms);
      if (rc != MAXSAT_OK) break;
      ctx->tune_vis_ms.emplace_back(vb, ms);
      auto it = vis_of.find(vb);
      if (it == vis_of.end() || ms < it->second) vis_of[vb] = ms;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->profiling = prof;
  ctx->vis_batch = vis_fixed ? vis_fixed : 4;
  if (rc != MAXSAT_OK) return rc;
  float vis_ms = vis_of.count(4) ? vis_of[4] : 1e30f;
  for (const auto& kv : vis_of)
    if (kv.second < 0.98f * vis_ms) {
      vis_ms = kv.second;
      ctx->vis_batch = kv.first;
    }
  ctx->cb_force = best;
  ctx->tuned_B = B;
  ctx->have_chains = false;  // the timing runs left no valid chains
  return MAXSAT_OK;
}

// Builds the dense (tensor-core) operands: the FP8 pattern-encoding gather
// matrix, the block-diagonal variable x incidence matrix and their TMA maps.
// Returns MAXSAT_OK, or an error code with *why (the context stays usable on
// the sparse path).
int build_dense(maxsat_ctx* ctx, int32_t n, int64_t m, const int64_t* off, const int32_t* lits,
                const int64_t* weights, const std::vector<int32_t>& var_off,
                const std::vector<int4>& var_inc, std::string* why) {
  DevAllocs& A = ctx->dense_mem;
#define UPD(vec, dst)                                  \
  do {                                                 \
    int rc_ = upload(ctx, A, vec, &(dst));             \
    if (rc_ != MAXSAT_OK) {                            \
      *why = ctx->err;                                 \
      return rc_;                                      \
    }                                                  \
  } while (0)
  const int64_t cells = (int64_t)((n + 127) / 128 * 128) * (int64_t)((m + 127) / 128 * 128);
  if (cells > ((int64_t)1 << 33)) {
    *why = "the dense gather matrix would exceed 8 GB";
    return MAXSAT_EINVAL;
  }
  int64_t wmax = 0;
  for (int64_t c = 0; c < m; ++c) wmax = std::max<int64_t>(wmax, weights ? weights[c] : 1);
  if (wmax >= ((int64_t)1 << 43)) {
    *why = "the dense path needs weights below 2^43";
    return MAXSAT_EINVAL;
  }
  std::vector<uint8_t> Ah;
  std::string derr = build_gather_matrix(n, (int)m, off, lits, &ctx->e5m2, &ctx->n_pad,
                                         &ctx->m_pad, &Ah);
  if (!derr.empty()) {
    *why = derr;
    return MAXSAT_EINVAL;
  }
  std::vector<int32_t> rl(ctx->m_pad, 0);
  std::vector<int64_t> rw(ctx->m_pad, 0);
  for (int64_t c = 0; c < m; ++c) {
    rl[c] = (int32_t)(off[c + 1] - off[c]);
    rw[c] = weights ? weights[c] : 1;
  }
  // per 32-row group: 1 when all its rows carry the same weight
  std::vector<uint8_t> small(ctx->m_pad / 32, 0);
  for (int g = 0; g < ctx->m_pad / 32; ++g) {
    bool same = true;
    for (int r = 1; r < 32; ++r) same = same && rw[g * 32 + r] == rw[g * 32];
    small[g] = same ? 1 : 0;
  }
  const uint8_t* dA = nullptr;
  const int32_t* drl = nullptr;
  const int64_t* drw = nullptr;
  const uint8_t* dsm = nullptr;
  UPD(Ah, dA);
  UPD(rl, drl);
  UPD(rw, drw);
  UPD(small, dsm);
  ctx->d_grp_small = const_cast<uint8_t*>(dsm);
  ctx->dA = const_cast<uint8_t*>(dA);
  ctx->d_row_len = const_cast<int32_t*>(drl);
  ctx->d_row_w = const_cast<int64_t*>(drw);
  derr = make_tmap_2d(&ctx->tmA, ctx->dA, ctx->n_pad, ctx->m_pad, ctx->n_pad, 128, 128, false);
  if (!derr.empty()) {
    *why = derr;
    return MAXSAT_ECUDA;
  }
  // scatter-add operands: G values exact in BF16 up to 256, in FP16 up to
  // 2048; the FP32 accumulator exact while |2^Q z| < 2^24
  const int gmax = ctx->tabs.gq_absmax;
  if (gmax > 2048 || (int64_t)ctx->max_degree * gmax >= ((int64_t)1 << 24)) {
    *why = "scatter-add contributions are not exact in FP16 / FP32";
    return MAXSAT_EINVAL;
  }
  ctx->g_bf16 = gmax <= 256;
  ctx->tiles_v = ctx->n_pad / 128;
  std::vector<int32_t> kst(ctx->tiles_v + 1), kbl(ctx->tiles_v);
  for (int tv = 0; tv <= ctx->tiles_v; ++tv) kst[tv] = var_off[std::min(tv * 128, n)];
  int kbmax = 1;
  for (int tv = 0; tv < ctx->tiles_v; ++tv) {
    kbl[tv] = std::max(1, (kst[tv + 1] - kst[tv] + 63) / 64);
    kbmax = std::max(kbmax, kbl[tv]);
  }
  ctx->kmax = kbmax * 64;
  const uint16_t plus = ctx->g_bf16 ? 0x3F80 : 0x3C00, minus = ctx->g_bf16 ? 0xBF80 : 0xBC00;
  std::vector<uint16_t> A2((size_t)ctx->tiles_v * 128 * ctx->kmax, 0);
  for (int i = 0; i < n; ++i) {
    const int tv = i / 128;
    for (int jj = var_off[i]; jj < var_off[i + 1]; ++jj)
      A2[(size_t)i * ctx->kmax + (jj - kst[tv])] = var_inc[jj].y < 0 ? minus : plus;
  }
  // contributions as 16-bit floating-point bit patterns (exact: integers
  // below 2^8 in BF16, below 2^11 in FP16)
  // (both halves hold the positive values: the sign is in A2)
  const size_t gq_len = ctx->tabs.gq.size();
  std::vector<uint16_t> gq16(2 * gq_len);
  for (size_t k = 0; k < gq16.size(); ++k) {
    const int v = ctx->tabs.gq[k % gq_len];
    uint16_t bits = 0;
    if (v != 0) {
      const unsigned av = (unsigned)(v < 0 ? -v : v);
      const int e2 = 31 - __builtin_clz(av);
      const int mb = ctx->g_bf16 ? 7 : 10;  // mantissa bits
      const unsigned mant = (e2 <= mb ? (av << (mb - e2)) : (av >> (e2 - mb))) & ((1u << mb) - 1u);
      bits = (uint16_t)(((unsigned)(e2 + (ctx->g_bf16 ? 127 : 15)) << mb) | mant);
      if (v < 0) bits |= 0x8000;
    }
    gq16[k] = bits;
  }
  const uint16_t* dA2 = nullptr;
  const int32_t* dks = nullptr;
  const int32_t* dkb = nullptr;
  const uint16_t* dg16 = nullptr;
  UPD(A2, dA2);
  UPD(kst, dks);
  UPD(kbl, dkb);
  UPD(gq16, dg16);
  ctx->d_gq16 = const_cast<uint16_t*>(dg16);
  ctx->d_kstart = const_cast<int32_t*>(dks);
  ctx->d_kblocks = const_cast<int32_t*>(dkb);
  derr = make_tmap_2d(&ctx->tmA2, dA2, ctx->kmax, (uint64_t)ctx->tiles_v * 128,
                      (uint64_t)ctx->kmax * 2, 64, 128, true);
  if (!derr.empty()) {
    *why = derr;
    return MAXSAT_ECUDA;
  }
  return MAXSAT_OK;
#undef UPD
}

extern "C" {

void maxsat_default_params(maxsat_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->n_temps = 2;
  p->fstar = nullptr;
  p->n_buckets = 4;
  p->bucket_gamma = 0.5;
  p->alpha = 0.01;
  p->quant_bits = 4;
  p->path = MAXSAT_PATH_AUTO;
  p->fit_iters = 50000;
  p->n_sets = 0;
  p->sets = nullptr;
  p->steps_per_graph = 100;
  p->tune_blocks = 0;
  p->up_device = 1;
  p->visible_batch = 0;
  p->persistent_round = 0;
}

const char* maxsat_last_error(const maxsat_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int maxsat_get_path(const maxsat_ctx* ctx) {
  if (!ctx) return MAXSAT_EINVAL;
  return ctx->dense ? MAXSAT_PATH_DENSE : ctx->path;
}

// Creates a context for the disjoint union of formulas: formula k owns
// variables var_base[k] .. var_base[k + 1] - 1 and clauses cl_base[k] ..
// cl_base[k + 1] - 1 (one formula: {0, n} and {0, m}); lits use the union's
// variable numbering.
static int create_impl(maxsat_ctx** out, int32_t n, int64_t m, const int64_t* off,
                       const int32_t* lits, const int64_t* weights, const maxsat_params* params,
                       void* cuda_stream, const std::vector<int32_t>& var_base,
                       const std::vector<int32_t>& cl_base) {
  const int n_inst = (int)var_base.size() - 1;
  if (!out) return fail(nullptr, MAXSAT_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1) return fail(nullptr, MAXSAT_EINVAL, "n_vars must be >= 1");
  if (m < 0 || m > (int64_t)INT32_MAX / 2) return fail(nullptr, MAXSAT_EINVAL, "n_clauses out of range");
  if (!off) return fail(nullptr, MAXSAT_EINVAL, "clause_off is NULL");
  if (off[0] != 0) return fail(nullptr, MAXSAT_EINVAL, "clause_off[0] must be 0");
  for (int64_t c = 0; c < m; ++c) {
    const int64_t len = off[c + 1] - off[c];
    if (len < 0) return fail(nullptr, MAXSAT_EINVAL, "clause_off must be non-decreasing");
    if (len > MAXSAT_MAX_LEN)
      return fail(nullptr, MAXSAT_EINVAL, "clause " + std::to_string(c) + " is longer than MAXSAT_MAX_LEN");
  }
  const int64_t nnz = off[m];
  if (nnz > (int64_t)INT32_MAX / 2) return fail(nullptr, MAXSAT_EINVAL, "too many literals");
  if (nnz > 0 && !lits) return fail(nullptr, MAXSAT_EINVAL, "lits is NULL");
  for (int64_t j = 0; j < nnz; ++j)
    if (lits[j] == 0 || lits[j] > n || lits[j] < -n)
      return fail(nullptr, MAXSAT_EINVAL, "literal " + std::to_string(j) + " out of range");
  // weight buckets are relative to the lightest clause of each formula
  std::vector<int64_t> wmin(n_inst, INT64_MAX);
  for (int k = 0; k < n_inst; ++k) {
    int64_t wsum = 0;
    for (int64_t c = cl_base[k]; c < cl_base[k + 1]; ++c) {
      const int64_t w = weights ? weights[c] : 1;
      if (w < 1) return fail(nullptr, MAXSAT_EINVAL, "weights must be >= 1");
      if (w > ((int64_t)1 << 62) - wsum) return fail(nullptr, MAXSAT_EINVAL, "total weight exceeds 2^62");
      wsum += w;
      wmin[k] = std::min(wmin[k], w);
    }
  }
  maxsat_params prm;
  if (params) prm = *params;
  else maxsat_default_params(&prm);
  if (prm.n_temps < 1 || prm.n_temps > 64) return fail(nullptr, MAXSAT_EINVAL, "n_temps must be in 1..64");
  if (prm.n_buckets < 1 || prm.n_buckets > 16) return fail(nullptr, MAXSAT_EINVAL, "n_buckets must be in 1..16");
  if (!(prm.alpha >= 0.0 && prm.alpha <= 1.0)) return fail(nullptr, MAXSAT_EINVAL, "alpha must be in [0, 1]");
  if (prm.quant_bits < 0 || prm.quant_bits > 8) return fail(nullptr, MAXSAT_EINVAL, "quant_bits must be in 0..8");
  if (prm.path < 0 || prm.path > 2) return fail(nullptr, MAXSAT_EINVAL, "unknown path");
  if (prm.steps_per_graph < 0 || prm.steps_per_graph > 100000)
    return fail(nullptr, MAXSAT_EINVAL, "steps_per_graph out of range");
  if (prm.visible_batch != 0 && prm.visible_batch != 2 && prm.visible_batch != 4 &&
      prm.visible_batch != 8)
    return fail(nullptr, MAXSAT_EINVAL, "visible_batch must be 0, 2, 4 or 8");
  if (prm.persistent_round != 0 && prm.persistent_round != 1)
    return fail(nullptr, MAXSAT_EINVAL, "persistent_round must be 0 or 1");
  if (prm.n_sets < 0 || (prm.n_sets > 0 && !prm.sets)) return fail(nullptr, MAXSAT_EINVAL, "sets is NULL");

  if (n_inst > 1 && prm.path == MAXSAT_PATH_DENSE)
    return fail(nullptr, MAXSAT_EINVAL, "a batch of formulas runs on the sparse path only");

  int rc = check_device(nullptr);
  if (rc != MAXSAT_OK) return rc;

  maxsat_ctx* ctx = new maxsat_ctx();
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->n_inst = n_inst;
  ctx->inst_var_base = var_base;
  ctx->inst_cl_base = cl_base;
  ctx->n = n;
  ctx->m = (int32_t)m;
  ctx->nnz = (int32_t)nnz;
  ctx->prm = prm;
  ctx->vis_batch = prm.visible_batch ? prm.visible_batch : 4;
  static const double kDefaultFstar[2] = {0.068, 0.528};
  for (int e = 0; e < prm.n_temps; ++e) {
    double f = prm.fstar ? prm.fstar[e] : (prm.n_temps == 2 ? kDefaultFstar[e] : 0.068 + (0.528 - 0.068) * e / std::max(1, prm.n_temps - 1));
    ctx->fstar.push_back(f);
  }
  ctx->prm.fstar = nullptr;
  ctx->prm.sets = nullptr;
  ctx->path = MAXSAT_PATH_SPARSE;

  // groups (length, bucket) in order of first appearance
  std::vector<int32_t> cl_grp(m, -1), grp_len, grp_bucket;
  std::map<std::pair<int, int>, int> gidx;
  int inst_of_c = 0;
  for (int64_t c = 0; c < m; ++c) {
    while (c >= cl_base[inst_of_c + 1]) ++inst_of_c;
    const int len = (int)(off[c + 1] - off[c]);
    if (len == 0) continue;
    const int j = weight_bucket(weights ? weights[c] : 1, wmin[inst_of_c], prm.n_buckets);
    auto key = std::make_pair(len, j);
    auto it = gidx.find(key);
    if (it == gidx.end()) {
      it = gidx.emplace(key, (int)grp_len.size()).first;
      grp_len.push_back(len);
      grp_bucket.push_back(j);
    }
    cl_grp[c] = it->second;
  }

  // clause RBM parameter sets: given, or fitted (Sec. 4.1)
  std::vector<RbmSet> sets;
  if (params && params->n_sets > 0) {
    for (int s = 0; s < params->n_sets; ++s) {
      const maxsat_rbm_set& u = params->sets[s];
      if (u.len < 1 || u.len > MAXSAT_MAX_LEN || u.n_hidden < 1 || u.n_hidden > MAXSAT_MAX_HIDDEN ||
          !u.W || !u.b) {
        delete ctx;
        return fail(nullptr, MAXSAT_EINVAL, "malformed RBM set " + std::to_string(s));
      }
      RbmSet r;
      r.len = u.len;
      r.bucket = u.bucket;
      r.temp = u.temp;
      r.nh = u.n_hidden;
      r.W.assign(u.W, u.W + (size_t)u.len * u.n_hidden);
      r.b.assign(u.b, u.b + u.n_hidden);
      sets.push_back(std::move(r));
    }
  } else {
    for (size_t g = 0; g < grp_len.size(); ++g)
      for (int e = 0; e < prm.n_temps; ++e) {
        RbmSet r;
        r.len = grp_len[g];
        r.bucket = grp_bucket[g];
        r.temp = e;
        r.nh = hidden_units_for(r.len);
        r.W.resize((size_t)r.len * r.nh);
        r.b.resize(r.nh);
        sets.push_back(std::move(r));
      }
    // fitting cost grows as 2^len; beyond the paper's K <= 7 the iterations
    // are scaled down by 2^(len - 7) (at least 2000)
    std::vector<std::thread> pool;
    std::vector<int> status(sets.size(), MAXSAT_OK);
    const unsigned hw = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::atomic<size_t> next{0};
    for (unsigned w = 0; w < hw; ++w)
      pool.emplace_back([&]() {
        for (size_t i; (i = next.fetch_add(1)) < sets.size();) {
          RbmSet& r = sets[i];
          int iters = prm.fit_iters;
          if (r.len > 7) iters = std::max(std::min(2000, iters), iters >> (r.len - 7));
          const double target = ctx->fstar[r.temp] * (1.0 + r.bucket * prm.bucket_gamma);
          status[i] = fit_or_rbm(r.len, r.nh, target, prm.quant_bits, iters, r.W.data(), r.b.data());
        }
      });
    for (auto& th : pool) th.join();
    for (int s : status)
      if (s != MAXSAT_OK) {
        delete ctx;
        return fail(nullptr, s, "OR-gate RBM fit failed");
      }
  }
  std::string terr = build_tables(sets, prm.n_temps, prm.quant_bits, grp_len, grp_bucket, &ctx->tabs);
  if (!terr.empty()) {
    delete ctx;
    return fail(nullptr, MAXSAT_EINVAL, terr);
  }

  // host CSR in device form
  std::vector<int32_t> cl_off(m + 1), lit_var(nnz), var_off(n + 1, 0);
  std::vector<int4> var_inc(nnz);
  std::vector<int64_t> cl_w(m);
  for (int64_t c = 0; c <= m; ++c) cl_off[c] = (int32_t)off[c];
  for (int64_t c = 0; c < m; ++c) cl_w[c] = weights ? weights[c] : 1;
  ctx->h_w = cl_w;
  up_prepare(n, m, off, lits, &ctx->upf);
  for (int64_t j = 0; j < nnz; ++j) {
    const int32_t l = lits[j];
    const int32_t v = (l > 0 ? l : -l) - 1;
    lit_var[j] = v | (l < 0 ? (int32_t)0x80000000 : 0);
    var_off[v + 1]++;
  }
  for (int i = 0; i < n; ++i) var_off[i + 1] += var_off[i];
  {
    std::vector<int32_t> fill(var_off.begin(), var_off.end() - 1);
    for (int64_t c = 0; c < m; ++c) {
      if (cl_grp[c] < 0) continue;
      const GroupMeta& gm = ctx->tabs.meta[cl_grp[c]];
      for (int64_t j = off[c]; j < off[c + 1]; ++j) {
        const int32_t l = lits[j];
        const int32_t v = (l > 0 ? l : -l) - 1;
        const int32_t k = (int32_t)(j - off[c]);
        // a negated literal points into the table's negated half
        const int32_t gq_len = (int32_t)ctx->tabs.gq.size();
        var_inc[fill[v]++] =
            make_int4((int32_t)c,
                      l < 0 ? (gm.gq_off + gq_len + k) | (int32_t)0x80000000 : gm.gq_off + k,
                      gm.len, (1 << gm.nh) * gm.len);
      }
    }
  }
  for (int i = 0; i < n; ++i) ctx->max_degree = std::max(ctx->max_degree, var_off[i + 1] - var_off[i]);
  // exactness of the integer scatter-sum: |2^Q z| <= degree * max |2^Q G|
  if ((int64_t)ctx->max_degree * ctx->tabs.gq_absmax >= ((int64_t)1 << 31)) {
    delete ctx;
    return fail(nullptr, MAXSAT_EINVAL, "visible logits could overflow int32");
  }

  DevAllocs& A = ctx->formula_mem;
  DevFormula& F = ctx->F;
  F.n = n;
  F.m = (int32_t)m;
  F.nnz = (int32_t)nnz;
  DevTables& T = ctx->T;
  T.n_temps = prm.n_temps;
  T.qmax = ctx->tabs.qmax;
  T.n_groups = ctx->tabs.n_groups;
  T.rec_len = (int32_t)ctx->tabs.rec.size();
  T.one_chunk = ctx->tabs.max_nh <= 3 ? 1 : 0;
  T.gq_len = (int32_t)ctx->tabs.gq.size();
  T.pv_len = (int32_t)ctx->tabs.pv.size();
  ctx->wide_h = ctx->tabs.max_nh > 8;
#define UP(vec, dst)                                          \
  do {                                                        \
    int rc_ = upload(ctx, A, vec, &(dst));                    \
    if (rc_ != MAXSAT_OK) {                                   \
      std::string e_ = ctx->err;                              \
      delete ctx;                                             \
      return fail(nullptr, rc_, e_);                          \
    }                                                         \
  } while (0)
  UP(cl_off, F.cl_off);
  UP(lit_var, F.lit_var);
  UP(cl_grp, F.cl_grp);
  UP(cl_w, F.cl_w);
  UP(var_off, F.var_off);
  UP(var_inc, F.var_inc);
  {
    // by degree within windows of 512 variables of one formula: a block's 8
    // variables carry similar work, and neighbouring blocks stay in one
    // region of the hidden patterns (a global sort scatters a batch's
    // accesses over every formula)
    std::vector<int32_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    constexpr int kOrderWindow = 512;
    for (int k = 0; k < n_inst; ++k)
      for (int w0 = var_base[k]; w0 < var_base[k + 1]; w0 += kOrderWindow) {
        const int w1 = std::min(w0 + kOrderWindow, (int)var_base[k + 1]);
        std::stable_sort(order.begin() + w0, order.begin() + w1, [&](int32_t a, int32_t b) {
          return var_off[a + 1] - var_off[a] > var_off[b + 1] - var_off[b];
        });
      }
    UP(order, F.var_order);
  }
  F.cl4 = nullptr;
  if (T.one_chunk) {
    // one 16-byte record per clause for the one-chunk gather
    std::vector<int4> cl4(m);
    for (int64_t c = 0; c < m; ++c) {
      const int32_t len = cl_off[c + 1] - cl_off[c];
      if (len > 3 || (len > 0 && cl_grp[c] < 0)) {
        delete ctx;
        return fail(nullptr, MAXSAT_EINVAL, "internal: clause record of a long clause");
      }
      int32_t lv[3] = {0, 0, 0};
      int32_t neg = 0;
      for (int32_t k = 0; k < len; ++k) {
        const int32_t l = lit_var[cl_off[c] + k];
        lv[k] = l & 0x7FFFFFFF;
        if (l < 0) neg |= 1 << k;
      }
      cl4[c] = make_int4(lv[0], lv[1], lv[2], len > 0 ? (cl_grp[c] << 8) | (neg << 2) | len : 0);
    }
    UP(cl4, F.cl4);
  }
  T.plain3 = 0;
  if (T.one_chunk && m > 0) {
    bool all3 = true;
    for (int64_t c = 0; c < m && all3; ++c) all3 = cl_off[c + 1] - cl_off[c] == 3;
    bool sat = false;
    for (const GroupMeta& gm : ctx->tabs.meta) sat = sat || gm.sat;
    T.plain3 = all3 && !sat ? 1 : 0;
  }
  T.rec3 = nullptr;
  T.rec3_words = 0;
  if (T.one_chunk && (int64_t)T.n_groups * T.n_temps * 256 <= 32 * 1024) {
    // one 256-byte block per (group, temperature): the group's 2^K records,
    // then its flags at word 32 (bit 8: a saturated hidden unit)
    const int E = T.n_temps;
    std::vector<uint32_t> rec3((size_t)T.n_groups * E * 64, 0u);
    for (int g = 0; g < T.n_groups; ++g) {
      const GroupMeta& gm = ctx->tabs.meta[g];
      const int np = 1 << gm.len;
      if (np > 8) {  // one-chunk formulas have clauses of at most 3 literals
        delete ctx;
        return fail(nullptr, MAXSAT_EINVAL, "internal: record block of a long clause group");
      }
      for (int e = 0; e < E; ++e) {
        uint32_t* blk = rec3.data() + ((size_t)g * E + e) * 64;
        for (int w = 0; w < 4 * np; ++w) blk[w] = ctx->tabs.rec[(size_t)gm.rec_off + (size_t)e * 4 * np + w];
        blk[32] = gm.sat ? 0x100u : 0u;
      }
    }
    UP(rec3, T.rec3);
    T.rec3_words = (int32_t)rec3.size();
  }
  F.n_inst = n_inst;
  F.var_inst = nullptr;
  if (n_inst > 1) {
    std::vector<int2> vi(n);
    for (int k = 0; k < n_inst; ++k)
      for (int v = var_base[k]; v < var_base[k + 1]; ++v) vi[v] = make_int2(k, v - var_base[k]);
    UP(vi, F.var_inst);
  }
  UP(ctx->tabs.meta, T.meta);
  UP(ctx->tabs.rec, T.rec);
  UP(ctx->tabs.feq, T.feq);
  {
    // two-sided contribution table of the sparse visible update: a negated
    // literal adds the second, negated half, so its sum needs no sign
    std::vector<int16_t> gq2(ctx->tabs.gq);
    for (int16_t v : ctx->tabs.gq) gq2.push_back((int16_t)-v);
    UP(gq2, T.gq);
  }
  UP(ctx->tabs.pv, T.pv);
#define UP2(vec, dst)                                         \
  do {                                                        \
    int rc_ = upload(ctx, A, vec, &(dst));                    \
    if (rc_ != MAXSAT_OK) {                                   \
      std::string e_ = ctx->err;                              \
      delete ctx;                                             \
      return fail(nullptr, rc_, e_);                          \
    }                                                         \
  } while (0)
  {
    cudaError_t e = A.alloc(&ctx->d_t, 1);
    if (e == cudaSuccess) e = A.alloc(&ctx->d_err, 1);
    if (e == cudaSuccess) e = A.alloc(&ctx->d_bar, 2);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
      delete ctx;
      return cuda_fail(nullptr, e, "cudaMalloc");
    }
  }
  {
    int64_t wmax_ev = 0;
    const int rcp = upload_plan(ctx, ctx->formula_mem, clause_block_for(ctx->m), &ctx->ev_plan,
                                &wmax_ev);
    if (rcp != MAXSAT_OK) {
      std::string e_ = ctx->err;
      delete ctx;
      return fail(nullptr, rcp, e_);
    }
  }
  if (prm.path == MAXSAT_PATH_DENSE && n_inst == 1) {
    std::string why;
    const int drc = build_dense(ctx, n, m, off, lits, weights, var_off, var_inc, &why);
    if (drc != MAXSAT_OK) {
      delete ctx;
      return fail(nullptr, drc, why);
    }
    ctx->dense_built = true;
    ctx->dense = true;
  } else if (prm.path == MAXSAT_PATH_AUTO && n_inst == 1) {
    ctx->dense_pending = true;
    ctx->lazy_off.assign(off, off + m + 1);
    ctx->lazy_lits.assign(lits, lits + off[m]);
    ctx->lazy_var_off = var_off;
    ctx->lazy_var_inc = var_inc;
  }
  *out = ctx;
  return MAXSAT_OK;
}

int maxsat_create(maxsat_ctx** out, int32_t n, int64_t m, const int64_t* off,
                  const int32_t* lits, const int64_t* weights, const maxsat_params* params,
                  void* cuda_stream) {
  NvtxRange range("maxsat_create");
  g_create_error.clear();
  if (!out) return fail(nullptr, MAXSAT_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1) return fail(nullptr, MAXSAT_EINVAL, "n_vars must be >= 1");
  if (m < 0 || m > (int64_t)INT32_MAX / 2) return fail(nullptr, MAXSAT_EINVAL, "n_clauses out of range");
  return create_impl(out, n, m, off, lits, weights, params, cuda_stream, {0, n}, {0, (int32_t)m});
}

int maxsat_create_batch(maxsat_ctx** out, int32_t n_inst, const int32_t* n_vars,
                        const int64_t* n_clauses, const int64_t* clause_off, const int32_t* lits,
                        const int64_t* weights, const maxsat_params* params, void* cuda_stream) {
  NvtxRange range("maxsat_create_batch");
  g_create_error.clear();
  if (!out) return fail(nullptr, MAXSAT_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_inst < 1 || n_inst > 65535) return fail(nullptr, MAXSAT_EINVAL, "n_inst must be in 1..65535");
  if (!n_vars || !n_clauses) return fail(nullptr, MAXSAT_EINVAL, "n_vars / n_clauses is NULL");
  std::vector<int32_t> var_base(n_inst + 1, 0), cl_base(n_inst + 1, 0);
  for (int k = 0; k < n_inst; ++k) {
    if (n_vars[k] < 1) return fail(nullptr, MAXSAT_EINVAL, "every instance needs n_vars >= 1");
    if (n_clauses[k] < 0) return fail(nullptr, MAXSAT_EINVAL, "n_clauses must be >= 0");
    if ((int64_t)var_base[k] + n_vars[k] > INT32_MAX / 2 ||
        (int64_t)cl_base[k] + n_clauses[k] > INT32_MAX / 2)
      return fail(nullptr, MAXSAT_EINVAL, "batch too large");
    var_base[k + 1] = var_base[k] + n_vars[k];
    cl_base[k + 1] = cl_base[k] + (int32_t)n_clauses[k];
  }
  const int32_t n = var_base[n_inst];
  const int64_t m = cl_base[n_inst];
  if (!clause_off) return fail(nullptr, MAXSAT_EINVAL, "clause_off is NULL");
  if (clause_off[0] != 0) return fail(nullptr, MAXSAT_EINVAL, "clause_off[0] must be 0");
  for (int64_t c = 0; c < m; ++c)
    if (clause_off[c + 1] < clause_off[c] || clause_off[c + 1] - clause_off[c] > MAXSAT_MAX_LEN)
      return fail(nullptr, MAXSAT_EINVAL, "clause_off must be non-decreasing with lengths <= MAXSAT_MAX_LEN");
  const int64_t nnz = clause_off[m];
  if (nnz > (int64_t)INT32_MAX / 2) return fail(nullptr, MAXSAT_EINVAL, "too many literals");
  if (nnz > 0 && !lits) return fail(nullptr, MAXSAT_EINVAL, "lits is NULL");
  // instance-local DIMACS literals -> the union's numbering
  std::vector<int32_t> glits((size_t)nnz);
  for (int k = 0; k < n_inst; ++k)
    for (int64_t j = clause_off[cl_base[k]]; j < clause_off[cl_base[k + 1]]; ++j) {
      const int32_t l = lits[j];
      if (l == 0 || l > n_vars[k] || l < -n_vars[k])
        return fail(nullptr, MAXSAT_EINVAL, "instance " + std::to_string(k) + ": literal " +
                                                std::to_string(j) + " out of range");
      glits[j] = l > 0 ? l + var_base[k] : l - var_base[k];
    }
  return create_impl(out, n, m, clause_off, glits.data(), weights, params, cuda_stream, var_base,
                     cl_base);
}

int maxsat_get_clause_block(const maxsat_ctx* ctx) {
  if (!ctx) return MAXSAT_EINVAL;
  return ctx->gather_cb;
}

int maxsat_get_visible_batch(const maxsat_ctx* ctx) {
  if (!ctx) return MAXSAT_EINVAL;
  return ctx->vis_batch;
}

// the persistent round runs maxsat_step's rounds: requested, sparse chains
// that it covers, no per-kernel profiling, no GPU unit propagation pending
// (its side-stream kernel shares the SMs the cooperative launch must hold)
static bool persistent_round_active(const maxsat_ctx* ctx) {
  return ctx->prm.persistent_round && ctx->have_chains && !ctx->dense && !ctx->profiling &&
         !(ctx->up_pending && ctx->up_on_gpu) &&
         persistent_round_supported(ctx->T, ctx->C, ctx->F, ctx->wide_h);
}

int maxsat_get_persistent_round(const maxsat_ctx* ctx) {
  if (!ctx) return MAXSAT_EINVAL;
  return persistent_round_active(ctx) ? 1 : 0;
}

int maxsat_get_n_instances(const maxsat_ctx* ctx) {
  if (!ctx) return MAXSAT_EINVAL;
  return ctx->n_inst;
}

int maxsat_reset(maxsat_ctx* ctx, int32_t B, uint64_t seed) {
  return maxsat_reset_shard(ctx, B, seed, 0, B);
}

int maxsat_reset_shard(maxsat_ctx* ctx, int32_t B, uint64_t seed, int32_t chain_offset,
                       int32_t total_chains) {
  NvtxRange range("maxsat_reset_shard");
  if (!ctx) return MAXSAT_EINVAL;
  if (B < 1 || B > (1 << 26)) return fail(ctx, MAXSAT_EINVAL, "restarts must be in 1..2^26");
  if (chain_offset < 0 || chain_offset % 8 != 0 || total_chains < chain_offset + B ||
      (int64_t)total_chains + kChainTile > ((int64_t)1 << 26))
    return fail(ctx, MAXSAT_EINVAL,
                "chain_offset must be a non-negative multiple of 8 and chain_offset + restarts "
                "<= total_chains < 2^26 - 256");
  if (ctx->prm.path == MAXSAT_PATH_AUTO && (ctx->dense_built || ctx->dense_pending) &&
      ctx->auto_B != B) {
    int rc0 = choose_path(ctx, B);
    if (rc0 != MAXSAT_OK) return rc0;
  }
  if (ctx->prm.tune_blocks && !ctx->dense && ctx->tuned_B != B) {
    int rc0 = tune_blocks(ctx, B);
    if (rc0 != MAXSAT_OK) return rc0;
  }
  int rc = alloc_chains(ctx, B);
  if (rc != MAXSAT_OK) return rc;
  if (ctx->C.key0 != (uint32_t)seed || ctx->C.key1 != (uint32_t)(seed >> 32) ||
      ctx->C.g8_off != chain_offset / 8 || ctx->C.B_total != total_chains)
    destroy_graph(ctx);
  ctx->C.key0 = (uint32_t)seed;
  ctx->C.key1 = (uint32_t)(seed >> 32);
  ctx->C.keys = philox_keys(ctx->C.key0, ctx->C.key1);
  ctx->C.g8_off = chain_offset / 8;
  ctx->C.B_total = total_chains;
  ctx->C.inv_B_total = 1.0f / (float)total_chains;
  ctx->seed = seed;
  ctx->t = 0;
  ctx->d_t_synced = false;
  if (ctx->dense)
    CK(ctx, launch_init_dense(ctx->C, ctx->dX, ctx->dnu, ctx->dbest_x, ctx->n, ctx->n_pad,
                              ctx->e5m2, ctx->stream));
  else
    CK(ctx, launch_init_sparse(ctx->F, ctx->C, ctx->n, ctx->stream));
  ctx->have_chains = true;
  return MAXSAT_OK;
}

int maxsat_step(maxsat_ctx* ctx, int64_t steps) {
  NvtxRange range("maxsat_step");
  if (!ctx) return MAXSAT_EINVAL;
  if (!ctx->have_chains) return fail(ctx, MAXSAT_ESTATE, "maxsat_step before maxsat_reset");
  if (steps < 0) return fail(ctx, MAXSAT_EINVAL, "steps must be >= 0");
  if ((uint64_t)ctx->t + (uint64_t)steps > 0xFFFFFFFFull) return fail(ctx, MAXSAT_EINVAL, "round index would exceed 2^32");
  if (persistent_round_active(ctx)) {
    const int64_t chunk = std::max(1, ctx->prm.steps_per_graph);
    while (steps > 0) {
      const int r = (int)std::min(steps, chunk);
      CK(ctx, launch_round_persistent(ctx->F, ctx->T, ctx->C, ctx->plan, ctx->t, r,
                                      (float)ctx->prm.alpha, ctx->d_bar, ctx->d_err,
                                      ctx->stream));
      ctx->persist_ran = true;
      ctx->t += (uint32_t)r;
      ctx->d_t_synced = false;
      steps -= r;
    }
    return MAXSAT_OK;
  }
  const int S = ctx->profiling ? 0 : ctx->prm.steps_per_graph;
  while (steps > 0) {
    if (S > 0 && steps >= S) {
      if (!ctx->graph || ctx->graph_steps != S) {
        int rc = capture_graph(ctx, S);
        if (rc != MAXSAT_OK) return rc;
      }
      if (!ctx->d_t_synced) {
        CK(ctx, launch_set_u32(ctx->d_t, ctx->t, ctx->stream));
        ctx->d_t_synced = true;
      }
      CK(ctx, cudaGraphLaunch(ctx->graph, ctx->stream));
      ctx->t += (uint32_t)S;
      steps -= S;
    } else {
      int rc = launch_round(ctx, ctx->stream, nullptr, ctx->t);
      if (rc != MAXSAT_OK) return rc;
      ctx->t += 1;
      ctx->d_t_synced = false;
      steps -= 1;
    }
  }
  return MAXSAT_OK;
}

int maxsat_score(maxsat_ctx* ctx) {
  NvtxRange range("maxsat_score");
  if (!ctx) return MAXSAT_EINVAL;
  if (!ctx->have_chains) return fail(ctx, MAXSAT_ESTATE, "maxsat_score before maxsat_reset");
  const DevChains& C = ctx->C;
  if (ctx->dense) {
    cudaStream_t st = ctx->stream;
    TIMED(ctx, st, "gemm1_score",
          launch_gemm1_step(false, ctx->tmA, ctx->tmX, ctx->m, ctx->m_pad, ctx->n_pad, C.B, C.Bp,
                            ctx->e5m2, ctx->d_row_len, ctx->d_row_w, ctx->F.cl_grp,
                            ctx->d_grp_small, ctx->dcost_part, ctx->dfe_part, C.H, ctx->wide_h,
                            nullptr, 0, ctx->d_err, ctx->T, C, st));
    TIMED(ctx, st, "keep", launch_keep_dense(ctx->dcost_part, ctx->dfe_part, ctx->m_pad / 128, C, st));
    TIMED(ctx, st, "keep_copy",
          launch_keep_copy_dense(C, ctx->dX, ctx->dbest_x, ctx->n, ctx->n_pad, ctx->e5m2, st));
    return MAXSAT_OK;
  }
  TIMED(ctx, ctx->stream, "gather_score",
        launch_gather(kScore, ctx->F, ctx->T, C, C.xt, C.B, C.Bp, ctx->plan, nullptr, 0,
                      C.cost_part, C.fe_part, C.tickets, nullptr, ctx->wide_h, ctx->stream));
  TIMED(ctx, ctx->stream, "keep_copy", launch_keep_copy(ctx->F, C, ctx->n, ctx->stream));
  return MAXSAT_OK;
}

static void drain_marks(maxsat_ctx* ctx) {
  for (auto& mk : ctx->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, mk.start, mk.stop) == cudaSuccess) {
      ctx->prof_ms[mk.kernel] += ms;
      ctx->prof_count[mk.kernel] += 1;
    }
    cudaEventDestroy(mk.start);
    cudaEventDestroy(mk.stop);
  }
  ctx->marks.clear();
}

int maxsat_set_profiling(maxsat_ctx* ctx, int32_t on) {
  if (!ctx) return MAXSAT_EINVAL;
  if (!ctx->marks.empty()) {
    cudaStreamSynchronize(ctx->stream);
    drain_marks(ctx);
  }
  ctx->profiling = on != 0;
  ctx->prof_names.clear();
  ctx->prof_ms.clear();
  ctx->prof_count.clear();
  return MAXSAT_OK;
}

int maxsat_kernel_times(maxsat_ctx* ctx, int32_t max_kernels, char* names, int64_t* launches,
                        double* total_ms) {
  if (!ctx || max_kernels < 0) return MAXSAT_EINVAL;
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  drain_marks(ctx);
  const int k = std::min<int>(max_kernels, (int)ctx->prof_names.size());
  for (int i = 0; i < k; ++i) {
    if (names) {
      std::memset(names + 32 * i, 0, 32);
      std::strncpy(names + 32 * i, ctx->prof_names[i].c_str(), 31);
    }
    if (launches) launches[i] = ctx->prof_count[i];
    if (total_ms) total_ms[i] = ctx->prof_ms[i];
  }
  return k;
}

// sparse eval scratch for Bp chains (grown on demand)
static int ensure_eval_scratch(maxsat_ctx* ctx, int Bp) {
  if (Bp <= ctx->ev_Bp) return MAXSAT_OK;
  ctx->eval_mem.release();
  ctx->ev_Bp = 0;
  const size_t ntk = (size_t)ctx->n_inst * (Bp / kChainTile);
  CK(ctx, ctx->eval_mem.alloc(&ctx->ev_xt, (size_t)ctx->n * Bp));
  CK(ctx, ctx->eval_mem.alloc(&ctx->ev_part, (size_t)ctx->ev_plan.n_blk * Bp));
  CK(ctx, ctx->eval_mem.alloc(&ctx->ev_tickets, ntk));
  CK(ctx, cudaMemsetAsync(ctx->ev_tickets, 0, sizeof(int32_t) * ntk, ctx->stream));
  ctx->ev_Bp = Bp;
  return MAXSAT_OK;
}

int maxsat_eval(maxsat_ctx* ctx, const uint8_t* assign_dev, int32_t B, int64_t* cost_dev) {
  NvtxRange range("maxsat_eval");
  if (!ctx) return MAXSAT_EINVAL;
  if (B < 0 || (B > 0 && (!assign_dev || !cost_dev))) return fail(ctx, MAXSAT_EINVAL, "bad eval arguments");
  if (B == 0) return MAXSAT_OK;
  if (ctx->dense_built) {
    const int Bp = (B + 255) / 256 * 256;
    if (Bp > ctx->dev_Bp) {
      // grow the eval scratch (releasing the old one waits for the device)
      ctx->dense_eval_mem.release();
      ctx->dev_Bp = 0;
      for (int k = 0; k < 2; ++k) {
        CK(ctx, ctx->dense_eval_mem.alloc(&ctx->dXe[k], (size_t)Bp * ctx->n_pad));
        std::string e =
            make_tmap_2d(&ctx->tmXe[k], ctx->dXe[k], ctx->n_pad, Bp, ctx->n_pad, 128, 256, false);
        if (!e.empty()) return fail(ctx, MAXSAT_ECUDA, e);
      }
      ctx->dev_Bp = Bp;
    }
    const int Bt = ctx->dev_Bp;
    // alternate state buffers: this conversion may run beside the previous
    // evaluation's product, which reads the other one
    const int xb = ctx->ev_buf;
    ctx->ev_buf ^= 1;
    TIMED(ctx, ctx->stream, "assign_fp8",
          launch_assign_fp8(assign_dev, B, ctx->n, Bt, ctx->n_pad, ctx->e5m2, ctx->dXe[xb],
                            cost_dev, ctx->stream));
    TIMED(ctx, ctx->stream, "gemm1_eval",
          launch_gemm1_eval(ctx->tmA, ctx->tmXe[xb], ctx->m, ctx->m_pad, ctx->n_pad, B, Bt, ctx->e5m2,
                            ctx->d_row_len, ctx->d_row_w, ctx->d_grp_small, cost_dev, ctx->d_err,
                            ctx->stream));
    return MAXSAT_OK;
  }
  const int Bp = (B + kChainTile - 1) / kChainTile * kChainTile;
  const int rc = ensure_eval_scratch(ctx, Bp);
  if (rc != MAXSAT_OK) return rc;
  CK(ctx, launch_transpose_in(assign_dev, B, ctx->n, ctx->ev_xt, Bp, ctx->stream));
  CK(ctx, launch_gather(kEval, ctx->F, ctx->T, ctx->C, ctx->ev_xt, B, Bp, ctx->ev_plan, nullptr, 0,
                        ctx->ev_part, nullptr, ctx->ev_tickets, cost_dev, ctx->wide_h,
                        ctx->stream));
  return MAXSAT_OK;
}

// The best over the chains after the final score (maxsat_solve, maxsat_solve_timed).
static int copy_best(maxsat_ctx* ctx, int32_t B, uint8_t* best_assign, int64_t* best_cost);

int maxsat_solve(maxsat_ctx* ctx, int32_t B, int64_t steps, uint64_t seed,
                 uint8_t* best_assign, int64_t* best_cost) {
  NvtxRange range("maxsat_solve");
  if (!ctx) return MAXSAT_EINVAL;
  int rc = maxsat_reset(ctx, B, seed);
  if (rc == MAXSAT_OK) rc = maxsat_step(ctx, steps);
  if (rc == MAXSAT_OK) rc = maxsat_score(ctx);
  if (rc != MAXSAT_OK) return rc;
  return copy_best(ctx, B, best_assign, best_cost);
}

int maxsat_solve_timed(maxsat_ctx* ctx, int32_t B, double seconds, int64_t max_steps,
                       int64_t chunk, uint64_t seed, uint8_t* best_assign, int64_t* best_cost,
                       int64_t* steps_done) {
  NvtxRange range("maxsat_solve_timed");
  if (!ctx) return MAXSAT_EINVAL;
  if (!(seconds >= 0.0) || max_steps < 0)
    return fail(ctx, MAXSAT_EINVAL, "seconds and max_steps must be >= 0");
  const auto t0 = std::chrono::steady_clock::now();
  if (chunk <= 0) chunk = std::max(1, ctx->prm.steps_per_graph);
  int rc = maxsat_reset(ctx, B, seed);
  if (rc != MAXSAT_OK) return rc;
  int64_t done = 0;
  // the time left is checked on the host between chunks, each synchronised
  while (done < max_steps &&
         std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() < seconds) {
    const int64_t k = std::min(chunk, max_steps - done);
    if ((rc = maxsat_step(ctx, k)) != MAXSAT_OK) return rc;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    done += k;
  }
  if (steps_done) *steps_done = done;
  if ((rc = maxsat_score(ctx)) != MAXSAT_OK) return rc;
  return copy_best(ctx, B, best_assign, best_cost);
}

static int copy_best(maxsat_ctx* ctx, int32_t B, uint8_t* best_assign, int64_t* best_cost) {
  // per formula: its lowest best cost, ties to the lowest chain
  const int K = ctx->n_inst, Bp = ctx->C.Bp;
  std::vector<int64_t> best((size_t)K * B);
  CK(ctx, cudaMemcpy2DAsync(best.data(), sizeof(int64_t) * B, ctx->C.best, sizeof(int64_t) * Bp,
                            sizeof(int64_t) * B, K, cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < K; ++k) {
    const int64_t* bk = best.data() + (size_t)k * B;
    int bstar = 0;
    for (int b = 1; b < B; ++b)
      if (bk[b] < bk[bstar]) bstar = b;
    if (best_cost) best_cost[k] = bk[bstar];
    if (best_assign) {
      const int v0 = ctx->inst_var_base[k], nk = ctx->inst_var_base[k + 1] - v0;
      if (ctx->dense)
        CK(ctx, cudaMemcpyAsync(best_assign, ctx->dbest_x + (size_t)bstar * ctx->n_pad, ctx->n,
                                cudaMemcpyDeviceToHost, ctx->stream));
      else
        CK(ctx, cudaMemcpy2DAsync(best_assign + v0, 1, ctx->C.best_xt + (size_t)v0 * Bp + bstar, Bp,
                                  1, nk, cudaMemcpyDeviceToHost, ctx->stream));
    }
  }
  if (best_assign) CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->dense || ctx->persist_ran) return check_device_error(ctx);
  return MAXSAT_OK;
}

int maxsat_get_state(maxsat_ctx* ctx, uint8_t* x, float* nu, int64_t* best_cost,
                     uint8_t* best_x, int64_t* cost, float* free_energy, uint32_t* t) {
  NvtxRange range("maxsat_get_state");
  if (!ctx) return MAXSAT_EINVAL;
  if (!ctx->have_chains) return fail(ctx, MAXSAT_ESTATE, "no chains (call maxsat_reset)");
  const int B = ctx->C.B, Bp = ctx->C.Bp, n = ctx->n;
  const size_t nB = (size_t)n * Bp;
  if (ctx->dense) {
    const int np = ctx->n_pad;
    uint8_t one;
    fp8_encode_int(1, ctx->e5m2, &one);
    auto fetch_rows = [&](const void* dsrc, size_t elem, void* dst, bool fp8) -> int {
      std::vector<uint8_t> h((size_t)np * Bp * elem);
      CK(ctx, cudaMemcpyAsync(h.data(), dsrc, h.size(), cudaMemcpyDeviceToHost, ctx->stream));
      CK(ctx, cudaStreamSynchronize(ctx->stream));
      uint8_t* d = static_cast<uint8_t*>(dst);
      for (int b = 0; b < B; ++b)
        for (int i = 0; i < n; ++i) {
          const uint8_t* src = h.data() + ((size_t)b * np + i) * elem;
          if (fp8) d[(size_t)b * n + i] = *src == one ? 1 : 0;
          else std::memcpy(d + ((size_t)b * n + i) * elem, src, elem);
        }
      return MAXSAT_OK;
    };
    int rc2;
    if (x && (rc2 = fetch_rows(ctx->dX, 1, x, true)) != MAXSAT_OK) return rc2;
    if (nu && (rc2 = fetch_rows(ctx->dnu, 4, nu, false)) != MAXSAT_OK) return rc2;
    if (best_x && (rc2 = fetch_rows(ctx->dbest_x, 1, best_x, false)) != MAXSAT_OK) return rc2;
    if (best_cost) CK(ctx, cudaMemcpyAsync(best_cost, ctx->C.best, 8 * (size_t)B, cudaMemcpyDeviceToHost, ctx->stream));
    if (cost) CK(ctx, cudaMemcpyAsync(cost, ctx->C.cost, 8 * (size_t)B, cudaMemcpyDeviceToHost, ctx->stream));
    if (free_energy) CK(ctx, cudaMemcpyAsync(free_energy, ctx->C.fe, 4 * (size_t)B, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (t) *t = ctx->t;
    return check_device_error(ctx);
  }
  auto fetch_T = [&](const void* dsrc, size_t elem, void* dst) -> int {
    std::vector<uint8_t> h(nB * elem);
    CK(ctx, cudaMemcpyAsync(h.data(), dsrc, nB * elem, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    uint8_t* d = static_cast<uint8_t*>(dst);
    for (int b = 0; b < B; ++b)
      for (int i = 0; i < n; ++i)
        std::memcpy(d + ((size_t)b * n + i) * elem, h.data() + ((size_t)i * Bp + b) * elem, elem);
    return MAXSAT_OK;
  };
  int rc;
  if (x && (rc = fetch_T(ctx->C.xt, 1, x)) != MAXSAT_OK) return rc;
  if (nu && (rc = fetch_T(ctx->C.nu, 4, nu)) != MAXSAT_OK) return rc;
  if (best_x && (rc = fetch_T(ctx->C.best_xt, 1, best_x)) != MAXSAT_OK) return rc;
  // per-formula rows of B chains (Bp apart on the device)
  const int K = ctx->n_inst;
  if (best_cost)
    CK(ctx, cudaMemcpy2DAsync(best_cost, 8 * (size_t)B, ctx->C.best, 8 * (size_t)Bp, 8 * (size_t)B,
                              K, cudaMemcpyDeviceToHost, ctx->stream));
  if (cost)
    CK(ctx, cudaMemcpy2DAsync(cost, 8 * (size_t)B, ctx->C.cost, 8 * (size_t)Bp, 8 * (size_t)B, K,
                              cudaMemcpyDeviceToHost, ctx->stream));
  if (free_energy)
    CK(ctx, cudaMemcpy2DAsync(free_energy, 4 * (size_t)B, ctx->C.fe, 4 * (size_t)Bp, 4 * (size_t)B,
                              K, cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (t) *t = ctx->t;
  if (ctx->persist_ran) return check_device_error(ctx);
  return MAXSAT_OK;
}

int maxsat_set_state(maxsat_ctx* ctx, int32_t B, uint64_t seed, const uint8_t* x,
                     const float* nu, const int64_t* best_cost, const uint8_t* best_x,
                     uint32_t t) {
  NvtxRange range("maxsat_set_state");
  if (!ctx) return MAXSAT_EINVAL;
  if (!x || !nu || !best_cost || !best_x) return fail(ctx, MAXSAT_EINVAL, "set_state needs x, nu, best_cost, best_x");
  int rc = maxsat_reset(ctx, B, seed);  // allocates and fills the padding chains
  if (rc != MAXSAT_OK) return rc;
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  const int Bp = ctx->C.Bp, n = ctx->n;
  const size_t nB = (size_t)n * Bp;
  if (ctx->dense) {
    const int np = ctx->n_pad;
    uint8_t one, minus_one;
    fp8_encode_int(1, ctx->e5m2, &one);
    fp8_encode_int(-1, ctx->e5m2, &minus_one);
    auto put_rows = [&](void* ddst, size_t elem, const void* src, int kind) -> int {
      std::vector<uint8_t> h((size_t)np * Bp * elem);
      CK(ctx, cudaMemcpy(h.data(), ddst, h.size(), cudaMemcpyDeviceToHost));
      const uint8_t* sp = static_cast<const uint8_t*>(src);
      for (int b = 0; b < B; ++b)
        for (int i = 0; i < n; ++i) {
          uint8_t* d = h.data() + ((size_t)b * np + i) * elem;
          const uint8_t* v = sp + ((size_t)b * n + i) * elem;
          if (kind == 1) *d = *v ? one : minus_one;      // FP8 state
          else if (kind == 2) *d = *v ? 1 : 0;           // best assignment bytes
          else std::memcpy(d, v, elem);                  // nu
        }
      CK(ctx, cudaMemcpy(ddst, h.data(), h.size(), cudaMemcpyHostToDevice));
      return MAXSAT_OK;
    };
    if ((rc = put_rows(ctx->dX, 1, x, 1)) != MAXSAT_OK) return rc;
    if ((rc = put_rows(ctx->dnu, 4, nu, 0)) != MAXSAT_OK) return rc;
    if ((rc = put_rows(ctx->dbest_x, 1, best_x, 2)) != MAXSAT_OK) return rc;
    CK(ctx, cudaMemcpy(ctx->C.best, best_cost, 8 * (size_t)B, cudaMemcpyHostToDevice));
    ctx->t = t;
    ctx->d_t_synced = false;
    return MAXSAT_OK;
  }
  auto put_T = [&](void* ddst, size_t elem, const void* src) -> int {
    std::vector<uint8_t> h(nB * elem);
    CK(ctx, cudaMemcpy(h.data(), ddst, nB * elem, cudaMemcpyDeviceToHost));
    const uint8_t* s = static_cast<const uint8_t*>(src);
    for (int b = 0; b < B; ++b)
      for (int i = 0; i < n; ++i)
        std::memcpy(h.data() + ((size_t)i * Bp + b) * elem, s + ((size_t)b * n + i) * elem, elem);
    if (elem == 1)
      for (int b = 0; b < B; ++b)
        for (int i = 0; i < n; ++i) h[(size_t)i * Bp + b] = h[(size_t)i * Bp + b] != 0;
    CK(ctx, cudaMemcpy(ddst, h.data(), nB * elem, cudaMemcpyHostToDevice));
    return MAXSAT_OK;
  };
  if ((rc = put_T(ctx->C.xt, 1, x)) != MAXSAT_OK) return rc;
  if ((rc = put_T(ctx->C.nu, 4, nu)) != MAXSAT_OK) return rc;
  if ((rc = put_T(ctx->C.best_xt, 1, best_x)) != MAXSAT_OK) return rc;
  CK(ctx, cudaMemcpy2D(ctx->C.best, 8 * (size_t)Bp, best_cost, 8 * (size_t)B, 8 * (size_t)B,
                       ctx->n_inst, cudaMemcpyHostToDevice));
  ctx->t = t;
  ctx->d_t_synced = false;
  return MAXSAT_OK;
}

// Writes chain-major states x (B x n bytes) and nu (B x n floats) of chains
// 0..B-1 into the device layout of the current path; the padding chains and
// the best-so-far are untouched.
static int put_states(maxsat_ctx* ctx, const uint8_t* x, const float* nu) {
  const int B = ctx->C.B, Bp = ctx->C.Bp, n = ctx->n;
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->dense) {
    const int np = ctx->n_pad;
    uint8_t one, minus_one;
    fp8_encode_int(1, ctx->e5m2, &one);
    fp8_encode_int(-1, ctx->e5m2, &minus_one);
    std::vector<uint8_t> hx((size_t)np * Bp);
    std::vector<float> hn((size_t)np * Bp);
    CK(ctx, cudaMemcpy(hx.data(), ctx->dX, hx.size(), cudaMemcpyDeviceToHost));
    CK(ctx, cudaMemcpy(hn.data(), ctx->dnu, 4 * hn.size(), cudaMemcpyDeviceToHost));
    for (int b = 0; b < B; ++b)
      for (int i = 0; i < n; ++i) {
        hx[(size_t)b * np + i] = x[(size_t)b * n + i] ? one : minus_one;
        hn[(size_t)b * np + i] = nu[(size_t)b * n + i];
      }
    CK(ctx, cudaMemcpy(ctx->dX, hx.data(), hx.size(), cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(ctx->dnu, hn.data(), 4 * hn.size(), cudaMemcpyHostToDevice));
    return MAXSAT_OK;
  }
  const size_t nB = (size_t)n * Bp;
  std::vector<uint8_t> hx(nB);
  std::vector<float> hn(nB);
  CK(ctx, cudaMemcpy(hx.data(), ctx->C.xt, nB, cudaMemcpyDeviceToHost));
  CK(ctx, cudaMemcpy(hn.data(), ctx->C.nu, 4 * nB, cudaMemcpyDeviceToHost));
  for (int b = 0; b < B; ++b)
    for (int i = 0; i < n; ++i) {
      hx[(size_t)i * Bp + b] = x[(size_t)b * n + i] ? 1 : 0;
      hn[(size_t)i * Bp + b] = nu[(size_t)b * n + i];
    }
  CK(ctx, cudaMemcpy(ctx->C.xt, hx.data(), nB, cudaMemcpyHostToDevice));
  CK(ctx, cudaMemcpy(ctx->C.nu, hn.data(), 4 * nB, cudaMemcpyHostToDevice));
  return MAXSAT_OK;
}

static int ensure_merge_buffers(maxsat_ctx* ctx);
static int merge_on_device(maxsat_ctx* ctx, int B);

// The appendix code's B-of-2B merge: cand holds 2B x n states whose second
// half is filled by the caller; the first half receives the B current
// states. All 2B are scored exactly; sorted by satisfied weight ascending
// with a stable sort, the last B become chains 0..B-1 in that order, each
// proposed state with the nu of the chain it came from.
static int merge_candidates(maxsat_ctx* ctx, std::vector<uint8_t>& cand) {
  const int B = ctx->C.B, n = ctx->n;
  std::vector<float> nu((size_t)B * n);
  std::vector<uint8_t> cur((size_t)B * n);
  int rc = maxsat_get_state(ctx, cur.data(), nu.data(), nullptr, nullptr, nullptr, nullptr,
                            nullptr);
  if (rc != MAXSAT_OK) return rc;
  std::memcpy(cand.data(), cur.data(), cur.size());
  if (cand.size() > ctx->up_cap) {
    ctx->up_mem.release();
    ctx->up_cap = 0;
    CK(ctx, ctx->up_mem.alloc(&ctx->d_up_cand, cand.size()));
    CK(ctx, ctx->up_mem.alloc(&ctx->d_up_cost, (size_t)2 * B));
    ctx->up_cap = cand.size();
  }
  CK(ctx, cudaMemcpyAsync(ctx->d_up_cand, cand.data(), cand.size(), cudaMemcpyHostToDevice,
                          ctx->stream));
  rc = maxsat_eval(ctx, ctx->d_up_cand, 2 * B, ctx->d_up_cost);
  if (rc != MAXSAT_OK) return rc;
  std::vector<int64_t> cost((size_t)2 * B);
  CK(ctx, cudaMemcpyAsync(cost.data(), ctx->d_up_cost, 8 * cost.size(), cudaMemcpyDeviceToHost,
                          ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  std::vector<int32_t> rank((size_t)2 * B);
  std::iota(rank.begin(), rank.end(), 0);
  std::stable_sort(rank.begin(), rank.end(),
                   [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  std::vector<uint8_t> nx((size_t)B * n);
  std::vector<float> nnu((size_t)B * n);
  for (int j = 0; j < B; ++j) {
    const int32_t r = rank[(size_t)B + j];
    std::memcpy(nx.data() + (size_t)j * n, cand.data() + (size_t)r * n, (size_t)n);
    std::memcpy(nnu.data() + (size_t)j * n, nu.data() + (size_t)(r % B) * n, 4 * (size_t)n);
  }
  return put_states(ctx, nx.data(), nnu.data());
}

int maxsat_propose_flips(maxsat_ctx* ctx, const float* prob, float tau) {
  NvtxRange range("maxsat_propose_flips");
  if (!ctx || !prob) return MAXSAT_EINVAL;
  if (!ctx->have_chains) return fail(ctx, MAXSAT_ESTATE, "maxsat_propose_flips before maxsat_reset");
  if (ctx->n_inst != 1 && ctx->dense)
    return fail(ctx, MAXSAT_EINVAL, "flip proposals of a batch run on the sparse path");
  if (!(tau >= 0.f && tau < 0.5f)) return fail(ctx, MAXSAT_EINVAL, "tau must be in [0, 0.5)");
  if (ctx->up_pending) return fail(ctx, MAXSAT_ESTATE, "a unit-propagation round is pending");
  const int B = ctx->C.B, n = ctx->n;
  if (!ctx->dense) {
    // on the device: proposals from the current states, then the merge
    std::vector<uint8_t> code(n);
    for (int i = 0; i < n; ++i) code[i] = prob[i] >= 1.f - tau ? 1 : (prob[i] <= tau ? 0 : 2);
    int rc = ensure_merge_buffers(ctx);
    if (rc != MAXSAT_OK) return rc;
    CK(ctx, cudaMemcpyAsync(ctx->d_flip_code, code.data(), n, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, launch_flip_candidates(ctx->C.xt, ctx->C.Bp, ctx->d_flip_code, n, B, ctx->d_upg_cand,
                                   ctx->upg_Bp, ctx->stream));
    rc = merge_on_device(ctx, B);
    if (rc != MAXSAT_OK) return rc;
    // code is a host buffer read by the copy above
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MAXSAT_OK;
  }
  std::vector<uint8_t> cand((size_t)2 * B * n);
  int rc = maxsat_get_state(ctx, cand.data() + (size_t)B * n, nullptr, nullptr, nullptr, nullptr,
                            nullptr, nullptr);
  if (rc != MAXSAT_OK) return rc;
  // the proposal: every confident variable takes the network's value
  for (int i = 0; i < n; ++i) {
    const float p = prob[i];
    if (p >= 1.f - tau)
      for (int b = 0; b < B; ++b) cand[(size_t)(B + b) * n + i] = 1;
    else if (p <= tau)
      for (int b = 0; b < B; ++b) cand[(size_t)(B + b) * n + i] = 0;
  }
  return merge_candidates(ctx, cand);
}

int maxsat_pt_swap(maxsat_ctx* ctx, int32_t parity, int32_t* accepted) {
  NvtxRange range("maxsat_pt_swap");
  if (!ctx) return MAXSAT_EINVAL;
  if (!ctx->have_chains) return fail(ctx, MAXSAT_ESTATE, "maxsat_pt_swap before maxsat_reset");
  if (parity != 0 && parity != 1) return fail(ctx, MAXSAT_EINVAL, "parity must be 0 or 1");
  const int E = ctx->T.n_temps, B = ctx->C.B;
  if (ctx->dense || ctx->n_inst != 1)
    return fail(ctx, MAXSAT_EINVAL, "parallel tempering runs on the sparse path of a single formula");
  if (ctx->C.g8_off != 0 || ctx->C.B_total != B)
    return fail(ctx, MAXSAT_EINVAL, "parallel tempering needs the whole ensemble on one context");
  if (E < 2 || B % E != 0 || (B / E) % 8 != 0)
    return fail(ctx, MAXSAT_EINVAL, "parallel tempering needs restarts = E x S with S a multiple of 8");
  if (!ctx->tabs.feq_ok) return fail(ctx, MAXSAT_EINVAL, "free energies exceed the fixed-point range");
  if (!ctx->d_Tc) {
    std::vector<long long> Tc(65536);
    Tc[0] = INT64_MIN;
    for (int u = 1; u < 65536; ++u)
      Tc[u] = (long long)std::ceil(std::ldexp(std::log(u / 65536.0), 20));
    CK(ctx, ctx->pt_mem.alloc(&ctx->d_Tc, Tc.size()));
    CK(ctx, cudaMemcpy(ctx->d_Tc, Tc.data(), 8 * Tc.size(), cudaMemcpyHostToDevice));
    CK(ctx, ctx->pt_mem.alloc(&ctx->d_nacc, 1));
  }
  if (ctx->pt_Bp < ctx->C.Bp) {
    CK(ctx, ctx->pt_mem.alloc(&ctx->d_Fown, (size_t)ctx->C.Bp));
    CK(ctx, ctx->pt_mem.alloc(&ctx->d_Foth, (size_t)ctx->C.Bp));
    CK(ctx, ctx->pt_mem.alloc(&ctx->d_swap, (size_t)ctx->C.Bp + 8));
    ctx->pt_Bp = ctx->C.Bp;
  }
  CK(ctx, launch_pt_round(ctx->F, ctx->T, ctx->C, B / E, E, parity, ctx->t, ctx->d_Tc,
                          ctx->d_Fown, ctx->d_Foth, ctx->d_swap, ctx->d_nacc, ctx->stream));
  if (accepted) {
    int h = 0;
    CK(ctx, cudaMemcpyAsync(&h, ctx->d_nacc, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    *accepted = h;
  }
  return MAXSAT_OK;
}

// variables of the context's largest formula
static int max_formula_vars(const maxsat_ctx* ctx) {
  int mx = 0;
  for (int k = 0; k < ctx->n_inst; ++k)
    mx = std::max(mx, ctx->inst_var_base[k + 1] - ctx->inst_var_base[k]);
  return mx;
}

// the GPU form of unit propagation and of the merges applies: sparse path
// and every formula's chain state fits in shared memory
static bool gpu_merge_form(const maxsat_ctx* ctx) {
  return !ctx->dense && up_gpu_chains_per_block(max_formula_vars(ctx)) > 0;
}

// Device buffers of the GPU merge for the chains' B: snapshot of x and nu,
// the 2B candidates (n x Bp2), their costs and the permutation.
static int ensure_merge_buffers(maxsat_ctx* ctx) {
  const int B = ctx->C.B, Bp = ctx->C.Bp, n = ctx->n;
  const int Bp2 = (2 * B + kChainTile - 1) / kChainTile * kChainTile;
  if (ctx->upg_Bp == Bp2) return MAXSAT_OK;  // Bp2 determines Bp
  // earlier kernels that use the buffers are done before they are freed
  if (ctx->up_stream) CK(ctx, cudaStreamSynchronize(ctx->up_stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->upg_mem.release();
  ctx->upg_Bp = 0;
  CK(ctx, ctx->upg_mem.alloc(&ctx->d_upg_xs, (size_t)n * Bp));
  CK(ctx, ctx->upg_mem.alloc(&ctx->d_upg_nus, (size_t)n * Bp));
  CK(ctx, ctx->upg_mem.alloc(&ctx->d_upg_cand, (size_t)n * Bp2));
  // per formula: 2B costs and ranks, B permutation entries (B <= Bp2 / 2)
  const size_t per = (size_t)ctx->n_inst * Bp2;
  CK(ctx, ctx->upg_mem.alloc(&ctx->d_upg_cost, per));
  CK(ctx, ctx->upg_mem.alloc(&ctx->d_upg_perm, per));
  CK(ctx, ctx->upg_mem.alloc(&ctx->d_upg_rank, per));
  CK(ctx, ctx->upg_mem.alloc(&ctx->d_flip_code, (size_t)n));
  ctx->upg_Bp = Bp2;
  return MAXSAT_OK;
}

// The B-of-2B merge on the device, candidates B..2B-1 already in place:
// candidates 0..B-1 become the current states, all 2B are scored with the
// sparse eval gather, ranked, and chain j takes position B + j (nu of the
// chain it came from; the snapshot's nu buffer is the staging area).
static int merge_on_device(maxsat_ctx* ctx, int B) {
  const int n = ctx->n, Bp = ctx->C.Bp, Bp2 = ctx->upg_Bp;
  CK(ctx, cudaMemcpy2DAsync(ctx->d_upg_cand, Bp2, ctx->C.xt, Bp, B, n, cudaMemcpyDeviceToDevice,
                            ctx->stream));
  const int rc = ensure_eval_scratch(ctx, Bp2);
  if (rc != MAXSAT_OK) return rc;
  CK(ctx, launch_gather(kEval, ctx->F, ctx->T, ctx->C, ctx->d_upg_cand, 2 * B, Bp2, ctx->ev_plan,
                        nullptr, 0, ctx->ev_part, nullptr, ctx->ev_tickets, ctx->d_upg_cost,
                        ctx->wide_h, ctx->stream));
  CK(ctx, launch_up_merge(ctx->d_upg_cost, ctx->n_inst, B, ctx->d_upg_rank, ctx->d_upg_perm,
                          ctx->d_upg_cand, Bp2, ctx->C.xt, ctx->C.nu, ctx->d_upg_nus, Bp, n,
                          ctx->F.var_inst, ctx->stream));
  CK(ctx, cudaMemcpy2DAsync(ctx->C.nu, sizeof(float) * Bp, ctx->d_upg_nus, sizeof(float) * Bp,
                            sizeof(float) * B, n, cudaMemcpyDeviceToDevice, ctx->stream));
  return MAXSAT_OK;
}

// GPU round: snapshot of x and nu on the context's stream, propagation on
// the side stream (the Gibbs rounds may run meanwhile), merge on the
// context's stream after it.
static int up_begin_gpu(maxsat_ctx* ctx) {
  const int B = ctx->C.B, Bp = ctx->C.Bp, n = ctx->n;
  const int Bp2 = (2 * B + kChainTile - 1) / kChainTile * kChainTile;
  if (!ctx->d_occ_off) {
    std::vector<int32_t> oo(ctx->upf.occ_off.size()), oc(ctx->upf.occ.size());
    for (size_t i = 0; i < oo.size(); ++i) oo[i] = (int32_t)ctx->upf.occ_off[i];
    for (size_t k = 0; k < oc.size(); ++k) oc[k] = ctx->upf.occ[k] & 0x7FFFFFFF;
    CK(ctx, ctx->upg_formula.alloc(&ctx->d_occ_off, oo.size()));
    CK(ctx, ctx->upg_formula.alloc(&ctx->d_occ, oc.size()));
    CK(ctx, ctx->upg_formula.alloc(&ctx->d_inst_var_base, ctx->inst_var_base.size()));
    CK(ctx, ctx->upg_formula.alloc(&ctx->d_inst_cl_base, ctx->inst_cl_base.size()));
    CK(ctx, cudaMemcpy(ctx->d_inst_var_base, ctx->inst_var_base.data(),
                       4 * ctx->inst_var_base.size(), cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(ctx->d_inst_cl_base, ctx->inst_cl_base.data(),
                       4 * ctx->inst_cl_base.size(), cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(ctx->d_occ_off, oo.data(), 4 * oo.size(), cudaMemcpyHostToDevice));
    if (!oc.empty())
      CK(ctx, cudaMemcpy(ctx->d_occ, oc.data(), 4 * oc.size(), cudaMemcpyHostToDevice));
  }
  if (!ctx->up_stream) {
    CK(ctx, cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking));
    CK(ctx, cudaEventCreateWithFlags(&ctx->up_ev_snap, cudaEventDisableTiming));
    CK(ctx, cudaEventCreateWithFlags(&ctx->up_ev_done, cudaEventDisableTiming));
  }
  int rc = ensure_merge_buffers(ctx);
  if (rc != MAXSAT_OK) return rc;
  CK(ctx, cudaMemcpyAsync(ctx->d_upg_xs, ctx->C.xt, (size_t)n * Bp, cudaMemcpyDeviceToDevice,
                          ctx->stream));
  CK(ctx, cudaMemcpyAsync(ctx->d_upg_nus, ctx->C.nu, sizeof(float) * n * Bp,
                          cudaMemcpyDeviceToDevice, ctx->stream));
  CK(ctx, cudaEventRecord(ctx->up_ev_snap, ctx->stream));
  CK(ctx, cudaStreamWaitEvent(ctx->up_stream, ctx->up_ev_snap, 0));
  UpDev U;
  U.n = n;
  U.m = ctx->m;
  U.cl_off = ctx->F.cl_off;
  U.lit_var = ctx->F.lit_var;
  U.occ_off = ctx->d_occ_off;
  U.occ = ctx->d_occ;
  U.n_inst = ctx->n_inst;
  U.var_base = ctx->d_inst_var_base;
  U.cl_base = ctx->d_inst_cl_base;
  U.n_max = max_formula_vars(ctx);
  CK(ctx, launch_up_chains(U, ctx->d_upg_xs, ctx->d_upg_nus, Bp, B, ctx->d_upg_cand, Bp2, B,
                           ctx->up_stream));
  CK(ctx, cudaEventRecord(ctx->up_ev_done, ctx->up_stream));
  ctx->up_B = B;
  ctx->up_pending = true;
  ctx->up_on_gpu = true;
  return MAXSAT_OK;
}

static int up_end_gpu(maxsat_ctx* ctx) {
  ctx->up_pending = false;
  ctx->up_on_gpu = false;
  CK(ctx, cudaStreamWaitEvent(ctx->stream, ctx->up_ev_done, 0));
  const int B = ctx->up_B;
  if (!ctx->have_chains || ctx->C.B != B || ctx->dense || ctx->upg_Bp == 0)
    return fail(ctx, MAXSAT_ESTATE, "the chains were reset during unit propagation");
  return merge_on_device(ctx, B);
}

int maxsat_up_begin(maxsat_ctx* ctx) {
  NvtxRange range("maxsat_up_begin");
  if (!ctx) return MAXSAT_EINVAL;
  if (!ctx->have_chains) return fail(ctx, MAXSAT_ESTATE, "maxsat_up_begin before maxsat_reset");
  const bool gpu = ctx->prm.up_device && gpu_merge_form(ctx);
  if (ctx->n_inst != 1 && !gpu)
    return fail(ctx, MAXSAT_EINVAL,
                "unit propagation of a batch of formulas runs in its GPU form only (sparse path, "
                "params.up_device)");
  if (ctx->up_pending) return fail(ctx, MAXSAT_ESTATE, "a unit-propagation round is already pending");
  const int B = ctx->C.B, n = ctx->n;
  if (gpu) return up_begin_gpu(ctx);
  ctx->up_x0.resize((size_t)B * n);
  ctx->up_nu0.resize((size_t)B * n);
  ctx->up_out.resize((size_t)B * n);
  int rc = maxsat_get_state(ctx, ctx->up_x0.data(), ctx->up_nu0.data(), nullptr, nullptr, nullptr,
                            nullptr, nullptr);
  if (rc != MAXSAT_OK) return rc;
  ctx->up_B = B;
  ctx->up_pending = true;
  ctx->up_on_gpu = false;
  const int threads = (int)std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  ctx->up_worker = std::thread([ctx, B, threads]() {
    up_chains(ctx->upf, B, ctx->up_x0.data(), ctx->up_nu0.data(), ctx->up_out.data(), threads);
  });
  return MAXSAT_OK;
}

int maxsat_up_end(maxsat_ctx* ctx) {
  NvtxRange range("maxsat_up_end");
  if (!ctx) return MAXSAT_EINVAL;
  if (!ctx->up_pending) return fail(ctx, MAXSAT_ESTATE, "maxsat_up_end without maxsat_up_begin");
  if (ctx->up_on_gpu) return up_end_gpu(ctx);
  if (ctx->up_worker.joinable()) ctx->up_worker.join();
  ctx->up_pending = false;
  const int B = ctx->up_B, n = ctx->n;
  if (!ctx->have_chains || ctx->C.B != B)
    return fail(ctx, MAXSAT_ESTATE, "the chains were reset during unit propagation");
  std::vector<uint8_t> cand((size_t)2 * B * n);
  std::memcpy(cand.data() + (size_t)B * n, ctx->up_out.data(), (size_t)B * n);
  return merge_candidates(ctx, cand);
}

int maxsat_up(maxsat_ctx* ctx) {
  const int rc = maxsat_up_begin(ctx);
  if (rc != MAXSAT_OK) return rc;
  return maxsat_up_end(ctx);
}

// ------------------------------------------------------ learned proposal
struct maxsat_mp {
  MpLayout lay;
  DevAllocs mem;  // parameters, gradients, Adam moments
  float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
  __nv_bfloat16* Pb = nullptr;
  int step = 0;
  // activations and backward buffers for graphs up to (cap_n, cap_m)
  DevAllocs act;
  int cap_n = 0, cap_m = 0;
  float *f = nullptr, *g = nullptr, *inv_len = nullptr, *inv_deg = nullptr;
  float* hv[kMpMaxLayers + 1] = {};
  float* hc[kMpMaxLayers + 1] = {};
  float* mc[kMpMaxLayers] = {};
  float* av[kMpMaxLayers] = {};
  float *dz = nullptr, *dhv = nullptr, *dhv2 = nullptr, *dav = nullptr, *dhc = nullptr,
        *dhc2 = nullptr, *dmc = nullptr, *part = nullptr;
  double* loss_part = nullptr;
  std::string err;
};

namespace {
int mp_fail(maxsat_mp* mp, int code, const std::string& msg) {
  if (mp) mp->err = msg;
  else g_create_error = msg;
  return code;
}

// an MP launch, bracketed by CUDA events under the formula context's
// profiling (maxsat_set_profiling / maxsat_kernel_times), as the Gibbs kernels
#define MPT(mp, ctx, name, expr)                                                \
  do {                                                                          \
    if ((ctx)->profiling) {                                                     \
      const int rc_ = timed((ctx), (ctx)->stream, name, [&]() { return (expr); }); \
      if (rc_ != MAXSAT_OK) return mp_fail(mp, rc_, (ctx)->err);                \
    } else {                                                                    \
      MPCK(mp, expr);                                                           \
    }                                                                           \
  } while (0)
#define MPCK(mp, expr)                                                         \
  do {                                                                          \
    cudaError_t e_ = (expr);                                                    \
    if (e_ != cudaSuccess) return mp_fail(mp, MAXSAT_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// splitmix64 + Box-Muller: a deterministic normal stream for the initial weights
struct NormalStream {
  uint64_t s;
  double spare = 0.0;
  bool have = false;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double normal() {
    if (have) {
      have = false;
      return spare;
    }
    const double u1 = uniform(), u2 = uniform();
    const double r = std::sqrt(-2.0 * std::log(u1));
    spare = r * std::sin(6.283185307179586 * u2);
    have = true;
    return r * std::cos(6.283185307179586 * u2);
  }
};

int mp_reserve(maxsat_mp* mp, int n, int m) {
  if (n <= mp->cap_n && m <= mp->cap_m) return MAXSAT_OK;
  mp->act.release();
  mp->cap_n = mp->cap_m = 0;
  const int L = mp->lay.L;
  const size_t nH = (size_t)std::max(n, 1) * kMpHidden, mH = (size_t)std::max(m, 1) * kMpHidden;
  DevAllocs& A = mp->act;
  MPCK(mp, A.alloc(&mp->f, 3 * (size_t)std::max(n, 1)));
  MPCK(mp, A.alloc(&mp->g, 3 * (size_t)std::max(m, 1)));
  MPCK(mp, A.alloc(&mp->inv_len, (size_t)std::max(m, 1)));
  MPCK(mp, A.alloc(&mp->inv_deg, (size_t)std::max(n, 1)));
  for (int l = 0; l <= L; ++l) {
    MPCK(mp, A.alloc(&mp->hv[l], nH));
    MPCK(mp, A.alloc(&mp->hc[l], mH));
  }
  for (int l = 0; l < L; ++l) {
    MPCK(mp, A.alloc(&mp->mc[l], mH));
    MPCK(mp, A.alloc(&mp->av[l], nH));
  }
  MPCK(mp, A.alloc(&mp->dz, (size_t)std::max(n, 1)));
  MPCK(mp, A.alloc(&mp->dhv, nH));
  MPCK(mp, A.alloc(&mp->dhv2, nH));
  MPCK(mp, A.alloc(&mp->dav, nH));
  MPCK(mp, A.alloc(&mp->dhc, mH));
  MPCK(mp, A.alloc(&mp->dhc2, mH));
  MPCK(mp, A.alloc(&mp->dmc, mH));
  const size_t rows = (size_t)std::max(n, m);
  MPCK(mp, A.alloc(&mp->part, ((rows + 255) / 256) * (kMpHidden * 2 * kMpHidden + kMpHidden)));
  MPCK(mp, A.alloc(&mp->loss_part, (size_t)std::max(n, 1) / 8 + 1));
  mp->cap_n = n;
  mp->cap_m = m;
  return MAXSAT_OK;
}

// forward pass over the formula of ctx; with labels, dz and the loss partials
int mp_forward(maxsat_mp* mp, maxsat_ctx* ctx, const uint8_t* y, float* prob) {
  const DevFormula& F = ctx->F;
  const int n = F.n, m = F.m, L = mp->lay.L;
  cudaStream_t st = ctx->stream;
  int rc = mp_reserve(mp, n, m);
  if (rc != MAXSAT_OK) return rc;
  const MpLayout& Y = mp->lay;
  MPT(mp, ctx, "mp_features", mp_launch_features(F, mp->f, mp->g, mp->inv_len, mp->inv_deg, st));
  MPT(mp, ctx, "mp_proj", mp_launch_proj(mp->f, n, mp->Pb + Y.Wf, mp->hv[0], st));
  MPT(mp, ctx, "mp_proj", mp_launch_proj(mp->g, m, mp->Pb + Y.Wg, mp->hc[0], st));
  for (int l = 0; l < L; ++l) {
    MPT(mp, ctx, "mp_clause_agg", mp_launch_clause_agg(F, mp->hv[l], mp->inv_len, nullptr, mp->mc[l], false, st));
    MPT(mp, ctx, "mp_dense_fwd", mp_launch_dense_fwd(mp->mc[l], mp->hc[l], m, mp->Pb + Y.Wc[l], mp->P + Y.bc[l],
                                 mp->hc[l + 1], st));
    MPT(mp, ctx, "mp_var_agg", mp_launch_var_agg(F, mp->hc[l + 1], nullptr, mp->inv_deg, mp->av[l], false, st));
    MPT(mp, ctx, "mp_dense_fwd", mp_launch_dense_fwd(mp->av[l], mp->hv[l], n, mp->Pb + Y.Wv[l], mp->P + Y.bv[l],
                                 mp->hv[l + 1], st));
  }
  MPT(mp, ctx, "mp_out", mp_launch_out(mp->hv[L], n, mp->P + Y.wo, mp->P + Y.bo, y, prob, y ? mp->dz : nullptr,
                         y ? mp->loss_part : nullptr, st));
  return MAXSAT_OK;
}
}  // namespace

int maxsat_mp_create(maxsat_mp** out, int32_t n_layers, uint64_t seed) {
  g_create_error.clear();
  if (!out) return mp_fail(nullptr, MAXSAT_EINVAL, "out is NULL");
  *out = nullptr;
  MpLayout lay;
  if (mp_layout(n_layers, &lay) != 0) return mp_fail(nullptr, MAXSAT_EINVAL, "n_layers must be in 1..8");
  int rc = check_device(nullptr);
  if (rc != MAXSAT_OK) return rc;
  maxsat_mp* mp = new maxsat_mp();
  mp->lay = lay;
  const int T = lay.total;
  // He-normal weight matrices (std sqrt(2 / fan_in)), read-out sqrt(1 / 64), zero biases
  std::vector<float> h((size_t)T, 0.f);
  NormalStream R{seed};
  auto fill = [&](int off, int rows, int cols, double sd) {
    for (int e = 0; e < rows * cols; ++e) h[(size_t)off + e] = (float)(sd * R.normal());
  };
  fill(lay.Wf, kMpHidden, 3, std::sqrt(2.0 / 3));
  fill(lay.Wg, kMpHidden, 3, std::sqrt(2.0 / 3));
  for (int l = 0; l < n_layers; ++l) {
    fill(lay.Wc[l], kMpHidden, 2 * kMpHidden, std::sqrt(2.0 / (2 * kMpHidden)));
    fill(lay.Wv[l], kMpHidden, 2 * kMpHidden, std::sqrt(2.0 / (2 * kMpHidden)));
  }
  fill(lay.wo, 1, kMpHidden, std::sqrt(1.0 / kMpHidden));
  DevAllocs& A = mp->mem;
  cudaError_t e = A.alloc(&mp->P, T);
  if (e == cudaSuccess) e = A.alloc(&mp->G, T);
  if (e == cudaSuccess) e = A.alloc(&mp->M, T);
  if (e == cudaSuccess) e = A.alloc(&mp->V, T);
  if (e == cudaSuccess) e = A.alloc(&mp->Pb, T);
  if (e == cudaSuccess) e = cudaMemcpy(mp->P, h.data(), 4 * (size_t)T, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(mp->G, 0, 4 * (size_t)T);
  if (e == cudaSuccess) e = cudaMemset(mp->M, 0, 4 * (size_t)T);
  if (e == cudaSuccess) e = cudaMemset(mp->V, 0, 4 * (size_t)T);
  if (e == cudaSuccess) e = mp_launch_to_bf16(mp->P, mp->Pb, T, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    delete mp;
    return mp_fail(nullptr, MAXSAT_ECUDA, std::string("mp create: ") + cudaGetErrorString(e));
  }
  *out = mp;
  return MAXSAT_OK;
}

int maxsat_mp_n_params(const maxsat_mp* mp) { return mp ? mp->lay.total : MAXSAT_EINVAL; }

int maxsat_mp_set_params(maxsat_mp* mp, const float* theta) {
  if (!mp || !theta) return MAXSAT_EINVAL;
  MPCK(mp, cudaMemcpy(mp->P, theta, 4 * (size_t)mp->lay.total, cudaMemcpyHostToDevice));
  MPCK(mp, mp_launch_to_bf16(mp->P, mp->Pb, mp->lay.total, nullptr));
  MPCK(mp, cudaMemset(mp->M, 0, 4 * (size_t)mp->lay.total));
  MPCK(mp, cudaMemset(mp->V, 0, 4 * (size_t)mp->lay.total));
  mp->step = 0;
  MPCK(mp, cudaDeviceSynchronize());
  return MAXSAT_OK;
}

int maxsat_mp_get_params(maxsat_mp* mp, float* theta, float* grad) {
  if (!mp) return MAXSAT_EINVAL;
  MPCK(mp, cudaDeviceSynchronize());
  if (theta) MPCK(mp, cudaMemcpy(theta, mp->P, 4 * (size_t)mp->lay.total, cudaMemcpyDeviceToHost));
  if (grad) MPCK(mp, cudaMemcpy(grad, mp->G, 4 * (size_t)mp->lay.total, cudaMemcpyDeviceToHost));
  return MAXSAT_OK;
}

int maxsat_mp_forward(maxsat_mp* mp, maxsat_ctx* ctx, float* prob_dev) {
  NvtxRange range("maxsat_mp_forward");
  if (!mp || !ctx || !prob_dev) return MAXSAT_EINVAL;
  return mp_forward(mp, ctx, nullptr, prob_dev);
}

int maxsat_mp_gradient(maxsat_mp* mp, maxsat_ctx* ctx, const uint8_t* labels_dev, double* loss) {
  NvtxRange range("maxsat_mp_gradient");
  if (!mp || !ctx || !labels_dev) return MAXSAT_EINVAL;
  int rc = mp_forward(mp, ctx, labels_dev, nullptr);
  if (rc != MAXSAT_OK) return rc;
  const DevFormula& F = ctx->F;
  const int n = F.n, m = F.m, L = mp->lay.L;
  const MpLayout& Y = mp->lay;
  cudaStream_t st = ctx->stream;
  float* G = mp->G;
  MPT(mp, ctx, "mp_out_bwd", mp_launch_out_bwd(mp->hv[L], mp->dz, n, mp->P + Y.wo, mp->dhv, mp->part, G + Y.wo, st));
  bool carry = false;  // dhc holds the gradient of h_c^l from clause layer l + 1
  for (int l = L - 1; l >= 0; --l) {
    // variable layer l: h_v^{l+1} = relu(Wv_l [a_v ; h_v^l] + bv_l)
    MPT(mp, ctx, "mp_dense_bwd_x", mp_launch_dense_bwd_x(mp->dhv, mp->hv[l + 1], n,
                                 mp->Pb + Y.Wv[l], mp->dav, mp->dhv2, st));
    MPT(mp, ctx, "mp_dense_wgrad", mp_launch_dense_wgrad(mp->dhv, mp->hv[l + 1], mp->av[l],
                                 mp->hv[l], n, mp->part, G + Y.Wv[l], st));
    MPT(mp, ctx, "mp_dense_wsum", mp_launch_dense_wsum(mp->part, n, G + Y.Wv[l], st));
    // a_v = (1 / deg_v) sum s h_c^{l+1}: gradient of h_c^{l+1}
    MPT(mp, ctx, "mp_clause_agg", mp_launch_clause_agg(F, mp->dav, nullptr, mp->inv_deg, mp->dhc, carry, st));
    // clause layer l: h_c^{l+1} = relu(Wc_l [m_c ; h_c^l] + bc_l)
    MPT(mp, ctx, "mp_dense_bwd_x", mp_launch_dense_bwd_x(mp->dhc, mp->hc[l + 1], m,
                                 mp->Pb + Y.Wc[l], mp->dmc, mp->dhc2, st));
    MPT(mp, ctx, "mp_dense_wgrad", mp_launch_dense_wgrad(mp->dhc, mp->hc[l + 1], mp->mc[l],
                                 mp->hc[l], m, mp->part, G + Y.Wc[l], st));
    MPT(mp, ctx, "mp_dense_wsum", mp_launch_dense_wsum(mp->part, m, G + Y.Wc[l], st));
    // m_c = (1 / len_c) sum s h_v^l: gradient of h_v^l
    MPT(mp, ctx, "mp_var_agg", mp_launch_var_agg(F, mp->dmc, mp->inv_len, nullptr, mp->dhv2, true, st));
    std::swap(mp->dhv, mp->dhv2);
    std::swap(mp->dhc, mp->dhc2);
    carry = true;
  }
  MPT(mp, ctx, "mp_proj_bwd", mp_launch_proj_bwd(mp->dhv, mp->hv[0], mp->f, n, mp->part, G + Y.Wf, st));
  MPT(mp, ctx, "mp_proj_bwd", mp_launch_proj_bwd(mp->dhc, mp->hc[0], mp->g, m, mp->part, G + Y.Wg, st));
  if (loss) {
    const int nb = (n + 7) / 8;
    std::vector<double> lp((size_t)nb);
    MPCK(mp, cudaMemcpyAsync(lp.data(), mp->loss_part, 8 * (size_t)nb, cudaMemcpyDeviceToHost, st));
    MPCK(mp, cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : lp) s += v;
    *loss = s / std::max(n, 1);
  }
  return MAXSAT_OK;
}

int maxsat_mp_adam(maxsat_mp* mp, maxsat_ctx* ctx, float lr) {
  NvtxRange range("maxsat_mp_adam");
  if (!mp || !ctx || !(lr > 0.f)) return MAXSAT_EINVAL;
  mp->step += 1;
  MPT(mp, ctx, "mp_adam", mp_launch_adam(mp->P, mp->G, mp->M, mp->V, mp->lay.total, lr, 0.9f, 0.999f, 1e-8f,
                          mp->step, mp->Pb, ctx->stream));
  return MAXSAT_OK;
}

const char* maxsat_mp_last_error(const maxsat_mp* mp) {
  return mp ? mp->err.c_str() : g_create_error.c_str();
}

void maxsat_mp_destroy(maxsat_mp* mp) {
  if (!mp) return;
  cudaDeviceSynchronize();
  delete mp;
}

int maxsat_reset_probs(maxsat_ctx* ctx, int32_t B, uint64_t seed, const float* prob) {
  NvtxRange range("maxsat_reset_probs");
  if (!ctx || !prob) return MAXSAT_EINVAL;
  const int n = ctx->n;
  std::vector<uint32_t> P((size_t)n);
  for (int i = 0; i < n; ++i) {
    const double p = prob[i];
    if (!(p >= 0.0 && p <= 1.0)) return fail(ctx, MAXSAT_EINVAL, "probabilities must be in [0, 1]");
    P[i] = (uint32_t)std::nearbyint(p * 65536.0);
  }
  int rc = maxsat_reset(ctx, B, seed);
  if (rc != MAXSAT_OK) return rc;
  DevAllocs tmp;  // freed on return, after the synchronisation below
  uint32_t* dP = nullptr;
  CK(ctx, tmp.alloc(&dP, (size_t)n));
  CK(ctx, cudaMemcpyAsync(dP, P.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->dense) {
    uint8_t one, minus_one;
    fp8_encode_int(1, ctx->e5m2, &one);
    fp8_encode_int(-1, ctx->e5m2, &minus_one);
    CK(ctx, launch_init_probs_dense(n, ctx->n_pad, ctx->C, dP, ctx->dX, ctx->dbest_x, one,
                                    minus_one, ctx->stream));
  } else {
    CK(ctx, launch_init_probs_sparse(ctx->F, ctx->C, dP, ctx->stream));
  }
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return MAXSAT_OK;
}

void maxsat_destroy(maxsat_ctx* ctx) {
  if (!ctx) return;
  if (ctx->up_worker.joinable()) ctx->up_worker.join();
  if (ctx->up_stream) {
    cudaStreamSynchronize(ctx->up_stream);
    cudaStreamDestroy(ctx->up_stream);
  }
  if (ctx->up_ev_snap) cudaEventDestroy(ctx->up_ev_snap);
  if (ctx->up_ev_done) cudaEventDestroy(ctx->up_ev_done);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  drain_marks(ctx);
  destroy_graph(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

}  // extern "C"
