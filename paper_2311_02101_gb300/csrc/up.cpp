// Prioritized unit propagation on the host (Sec. 4.4; the heuristic of Si et
// al. 2019 that the paper applies periodically to the sampled assignments).
//
// For one chain with assignment x and per-variable moving-average variance nu
// (the FP32 nu the kernels maintain):
//   1. rank the variables by nu, highest first (ties: lower index first);
//   2. the first floor(n / 2) keep their values from x (the paper holds the
//      highest-variance half fixed), set without propagating;
//   3. every clause that is not satisfied and has exactly one unassigned
//      literal occurrence queues that literal (clauses in index order); the
//      queue is emptied first in, first out: a literal whose variable is
//      still unassigned is made true, and every clause of that variable (in
//      index order) that becomes unit queues its open literal;
//   4. the remaining variables, in rank order, each take its value from x if
//      still unassigned, and the queue is emptied again after each.
// Falsified clauses are left falsified (MaxSAT). Chains run in parallel on
// host threads; the work per chain is O(nnz + n log n).
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <numeric>
#include <thread>
#include <vector>

#include "internal.h"

namespace rbmsat {

void up_prepare(int32_t n, int64_t m, const int64_t* off, const int32_t* lits, UpFormula* F) {
  F->n = n;
  F->m = (int32_t)m;
  const int64_t nnz = off[m];
  F->cl_off.assign(off, off + m + 1);
  F->lit.assign(lits, lits + nnz);
  F->occ_off.assign((size_t)n + 1, 0);
  for (int64_t j = 0; j < nnz; ++j) F->occ_off[(size_t)(lits[j] > 0 ? lits[j] : -lits[j])]++;
  for (int32_t i = 0; i < n; ++i) F->occ_off[i + 1] += F->occ_off[i];
  F->occ.assign((size_t)nnz, 0);
  std::vector<int64_t> fill(F->occ_off.begin(), F->occ_off.end() - 1);
  // occurrences of each variable in clause order, sign in bit 31
  for (int64_t c = 0; c < m; ++c)
    for (int64_t j = off[c]; j < off[c + 1]; ++j) {
      const int32_t l = lits[j];
      const int32_t v = (l > 0 ? l : -l) - 1;
      F->occ[(size_t)fill[v]++] = (int32_t)c | (l < 0 ? (int32_t)0x80000000 : 0);
    }
}

namespace {

struct Scratch {
  std::vector<int8_t> val;
  std::vector<int32_t> nfalse;
  std::vector<uint8_t> sat;
  std::vector<int32_t> queue;
  std::vector<int32_t> order;
};

class Propagator {
 public:
  Propagator(const UpFormula& F, Scratch& S) : F_(F), S_(S) {}

  void run(const uint8_t* x, const float* nu, uint8_t* out) {
    const int n = F_.n, m = F_.m;
    S_.val.assign((size_t)n, -1);
    S_.nfalse.assign((size_t)std::max(m, 1), 0);
    S_.sat.assign((size_t)std::max(m, 1), 0);
    S_.queue.resize(F_.lit.size() + (size_t)m + 1);
    head_ = tail_ = 0;
    S_.order.resize((size_t)n);
    std::iota(S_.order.begin(), S_.order.end(), 0);
    std::sort(S_.order.begin(), S_.order.end(), [nu](int32_t a, int32_t b) {
      return nu[a] > nu[b] || (nu[a] == nu[b] && a < b);
    });
    const int half = n / 2;
    for (int r = 0; r < half; ++r) set(S_.order[r], x[S_.order[r]] != 0, false);
    for (int c = 0; c < m; ++c) queue_if_unit(c);
    drain();
    for (int r = half; r < n; ++r) {
      const int32_t v = S_.order[r];
      if (S_.val[v] >= 0) continue;
      set(v, x[v] != 0, true);
      drain();
    }
    for (int i = 0; i < n; ++i) out[i] = (uint8_t)S_.val[i];
  }

 private:
  // the first unassigned literal of clause c when it is open and unit
  void queue_if_unit(int32_t c) {
    if (S_.sat[c]) return;
    const int64_t j0 = F_.cl_off[c], j1 = F_.cl_off[c + 1];
    if (j1 - j0 - S_.nfalse[c] != 1) return;
    for (int64_t j = j0; j < j1; ++j) {
      const int32_t l = F_.lit[j];
      if (S_.val[(l > 0 ? l : -l) - 1] < 0) {
        S_.queue[tail_++] = l;
        return;
      }
    }
  }

  void set(int32_t v, bool value, bool check) {
    S_.val[v] = value ? 1 : 0;
    const int64_t k0 = F_.occ_off[v], k1 = F_.occ_off[v + 1];
    for (int64_t k = k0; k < k1; ++k) {
      const int32_t o = F_.occ[k];
      const int32_t c = o & 0x7FFFFFFF;
      const bool positive = o >= 0;
      if (positive == value) S_.sat[c] = 1;
      else S_.nfalse[c]++;
    }
    if (!check) return;
    for (int64_t k = k0; k < k1; ++k) queue_if_unit(F_.occ[k] & 0x7FFFFFFF);
  }

  void drain() {
    while (head_ < tail_) {
      const int32_t l = S_.queue[head_++];
      const int32_t v = (l > 0 ? l : -l) - 1;
      if (S_.val[v] < 0) set(v, l > 0, true);
    }
  }

  const UpFormula& F_;
  Scratch& S_;
  size_t head_ = 0, tail_ = 0;
};

}  // namespace

void up_chains(const UpFormula& F, int32_t B, const uint8_t* x, const float* nu, uint8_t* out,
               int threads) {
  threads = std::max(1, std::min(threads, (int)B));
  std::atomic<int32_t> next{0};
  auto work = [&]() {
    Scratch S;
    Propagator P(F, S);
    for (int32_t b; (b = next.fetch_add(1)) < B;)
      P.run(x + (size_t)b * F.n, nu + (size_t)b * F.n, out + (size_t)b * F.n);
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
}

}  // namespace rbmsat
