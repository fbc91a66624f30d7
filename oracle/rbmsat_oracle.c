/*
 * RbmSAT oracle: a plain, slow CPU restatement of "Solving MaxSAT with Matrix
 * Multiplication" (RbmSAT), in FP64 wherever a value is real.
 *
 * THIS IS TEST INFRASTRUCTURE, NOT PRODUCT CODE. Only the tests, the smoke
 * check and the benchmark's CPU-baseline / reference arm may load it. It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * What it computes, in the paper's order (Sec. 4.2, Fig. "code" in the
 * appendix), one Markov chain at a time and one clause at a time:
 *   1. score the current assignment literal by literal (Sec. 1 definition of
 *      MaxSAT; Sec. 4.3 "comparing thresholded signs ... OR ... summing"),
 *      giving the weighted unsatisfied cost;
 *   2. best-so-far tracking (Sec. 4.2 "retain the best assignment seen");
 *   3. per clause, the clause-RBM parameters after the negation transform
 *      (Eq. 4), the hidden logits b' + W'^T v (Eq. 2 / Eq. 6) and the formula
 *      free energy as the sum of clause free energies (Eq. 1, Sec. 4.1
 *      "CNF Boolean formula as an RBM");
 *   4. Bernoulli draws of the hidden units (Eq. 2);
 *   5. the visible logits as the scatter-sum of Eq. 7 (visible bias d = 0,
 *      Sec. 4.1 "visible biases are not required");
 *   6. the variance moving average nu (Sec. 4.4) and the Bernoulli draws of
 *      the new visible state (Eq. 3).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - randomness: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit
 *     seed, counter (a, chunk, t, phase); one 16-bit lane per draw; a draw u
 *     gives 1 with probability P/65536 via u < P, P = rint(sigma(a) * 65536);
 *   - the visible probability used for nu is that same rho = P/65536;
 *   - clause c uses the parameter set keyed by (length, weight bucket,
 *     temperature of the chain); chains are split into contiguous temperature
 *     blocks e_b = floor(b * E / B);
 *   - the assignment is scored before each update and once more after the
 *     last step (by the caller), so steps t = 0..T score x_0..x_T;
 *   - a batch of formulas: instance i's draws carry i in the high 24 bits of
 *     the phase word, with its own clause and variable indices.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_LEN 12 /* longest clause with an OR-gate RBM */
#define OR_MAX_H 16   /* most hidden units per clause RBM */

enum { PH_INIT = 1, PH_HID = 2, PH_VIS = 3 };

/* ---------------------------------------------------------------------- */
/* Philox4x32-10, from Salmon, Moraes, Dror and Shaw, "Parallel random      */
/* numbers: as easy as 1, 2, 3" (SC'11): 10 rounds of two 32x32->64         */
/* multiplies; the key is bumped by the Weyl constants between rounds.      */
/* ---------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4]) {
  uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One 16-bit draw. Chain b's draw for unit `a` (a clause for hidden units, a
 * variable for visible/initial units), hidden unit h, step t and phase comes
 * from the counter (a, (b>>3) | (h<<24), t, phase), lane b & 7. */
uint32_t oracle_draw16(uint64_t seed, uint32_t phase, uint32_t t, uint32_t a,
                       uint32_t h, uint32_t b) {
  uint32_t ctr[4] = {a, (b >> 3) | (h << 24), t, phase};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  oracle_philox4x32_10(ctr, key, out);
  uint32_t lane = b & 7u;
  return (out[lane >> 1] >> (16u * (lane & 1u))) & 0xFFFFu;
}

static double sigmoid(double a) { return 1.0 / (1.0 + exp(-a)); }

static double softplus(double a) {
  return a > 0.0 ? a + log1p(exp(-a)) : log1p(exp(a));
}

/* Probability on the 16-bit grid: rint rounds half to even. */
static uint32_t prob16(double a) { return (uint32_t)rint(sigmoid(a) * 65536.0); }

/* ---------------------------------------------------------------------- */
/* MaxSAT cost, literal by literal (Sec. 1; Sec. 4.3). Literal l > 0 is     */
/* true when x[l-1] == 1, literal l < 0 when x[-l-1] == 0. An empty clause  */
/* is never satisfied.                                                      */
/* ---------------------------------------------------------------------- */
static int clause_satisfied(const int32_t* lits, int64_t len, const uint8_t* x) {
  for (int64_t k = 0; k < len; ++k) {
    int32_t l = lits[k];
    int32_t v = (l > 0 ? l : -l) - 1;
    int value = x[v] != 0;
    if ((l > 0) == value) return 1;
  }
  return 0;
}

static int64_t assignment_cost(int64_t m, const int64_t* off, const int32_t* lits,
                               const int64_t* w, const uint8_t* x) {
  int64_t cost = 0;
  for (int64_t c = 0; c < m; ++c)
    if (!clause_satisfied(lits + off[c], off[c + 1] - off[c], x))
      cost += w ? w[c] : 1;
  return cost;
}

int oracle_eval(int32_t n, int64_t m, const int64_t* off, const int32_t* lits,
                const int64_t* w, const uint8_t* x, int32_t B, int64_t* cost) {
  (void)n;
  for (int32_t b = 0; b < B; ++b)
    cost[b] = assignment_cost(m, off, lits, w, x + (int64_t)b * n);
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Canonical OR-gate RBM parameter sets. Set s serves clauses of length     */
/* set_len[s] in weight bucket set_bucket[s] for temperature set_temp[s];   */
/* it has set_nh[s] hidden units, W[s][k][h] (k < len, h < nh, stride        */
/* OR_MAX_H, OR_MAX_LEN * OR_MAX_H per set) and b[s][h] (stride OR_MAX_H).   */
/* ---------------------------------------------------------------------- */
typedef struct {
  int32_t n_sets;
  const int32_t* set_len;
  const int32_t* set_bucket;
  const int32_t* set_temp;
  const int32_t* set_nh;
  const double* W;
  const double* b;
} rbm_table;

static int find_set(const rbm_table* t, int32_t len, int32_t bucket, int32_t temp) {
  for (int32_t s = 0; s < t->n_sets; ++s)
    if (t->set_len[s] == len && t->set_bucket[s] == bucket && t->set_temp[s] == temp)
      return s;
  return -1;
}

/* Weight bucket of a clause: the largest j < n_buckets with
 * w_min * 2^j <= w_c (integer arithmetic; the paper is unweighted). */
static int32_t weight_bucket(int64_t wc, int64_t wmin, int32_t n_buckets) {
  int32_t j = 0;
  while (j + 1 < n_buckets && wmin <= (INT64_MAX >> (j + 1)) &&
         (wmin << (j + 1)) <= wc)
    ++j;
  return j;
}

/* Clause-RBM parameters after the negation transform, Eq. 4:
 * W' = Lambda W and b' = b + 1/2 (1 - diag Lambda) W. */
static void negation_transform(const rbm_table* t, int s, const int32_t* lits,
                               int32_t len, double Wp[OR_MAX_LEN][OR_MAX_H],
                               double bp[OR_MAX_H]) {
  int32_t nh = t->set_nh[s];
  const double* W = t->W + (int64_t)s * OR_MAX_LEN * OR_MAX_H;
  const double* b = t->b + (int64_t)s * OR_MAX_H;
  for (int32_t h = 0; h < nh; ++h) bp[h] = b[h];
  for (int32_t k = 0; k < len; ++k) {
    double lambda = lits[k] > 0 ? 1.0 : -1.0;
    for (int32_t h = 0; h < nh; ++h) {
      Wp[k][h] = lambda * W[k * OR_MAX_H + h];
      bp[h] += 0.5 * (1.0 - lambda) * W[k * OR_MAX_H + h];
    }
  }
}

/* ---------------------------------------------------------------------- */
/* Chain initialisation (Fig. code: v ~ Bernoulli(0.5), nu = 0.25,          */
/* best-so-far empty).                                                      */
/* ---------------------------------------------------------------------- */
int oracle_init(int32_t n, int32_t B, uint64_t seed, const int32_t* chain_ids,
                uint8_t* x, double* nu, float* nu32, int64_t* best_cost, uint32_t inst) {
  for (int32_t b = 0; b < B; ++b) {
    uint32_t gb = (uint32_t)(chain_ids ? chain_ids[b] : b);
    for (int32_t i = 0; i < n; ++i) {
      uint32_t u = oracle_draw16(seed, PH_INIT | (inst << 8), 0u, (uint32_t)i, 0u, gb);
      x[(int64_t)b * n + i] = u < 32768u;
      nu[(int64_t)b * n + i] = 0.25;
      if (nu32) nu32[(int64_t)b * n + i] = 0.25f;
    }
    best_cost[b] = INT64_MAX;
  }
  return 0;
}

/* ---------------------------------------------------------------------- */
/* T rounds of block Gibbs sampling on B chains, starting at step t0.       */
/* inst: the instance's index when many formulas are solved as one batch;  */
/* it fills the high 24 bits of every draw's phase word (0 for a single     */
/* formula), so each instance's chains draw exactly as if run alone with    */
/* that index.                                                              */
/* State arrays are B x n, chain-major. Row b is chain chain_ids[b] of an   */
/* ensemble of B_total chains (identity when chain_ids is NULL): the index  */
/* selects its draws and its temperature. cost/free_energy receive the      */
/* score of the state scored in the last round. Returns 0, or -1 when a     */
/* clause has no parameter set.                                             */
/* ---------------------------------------------------------------------- */
int oracle_gibbs(int32_t n, int64_t m, const int64_t* off, const int32_t* lits,
                 const int64_t* w, int32_t n_sets, const int32_t* set_len,
                 const int32_t* set_bucket, const int32_t* set_temp,
                 const int32_t* set_nh, const double* W, const double* bias,
                 int32_t n_temps, int32_t n_buckets, double alpha, uint64_t seed,
                 int32_t B, const int32_t* chain_ids, int32_t B_total, uint32_t t0,
                 int32_t T, uint8_t* x, double* nu, float* nu32, int64_t* best_cost,
                 uint8_t* best_x, int64_t* cost, double* free_energy, int32_t n_threads,
                 uint32_t inst) {
  rbm_table tab = {n_sets, set_len, set_bucket, set_temp, set_nh, W, bias};
  int64_t wmin = INT64_MAX;
  for (int64_t c = 0; c < m; ++c) {
    int64_t wc = w ? w[c] : 1;
    if (wc < wmin) wmin = wc;
  }
  int bad = 0;
  if (!chain_ids) B_total = B;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
#endif
  for (int32_t b = 0; b < B; ++b) {
    uint32_t gb = (uint32_t)(chain_ids ? chain_ids[b] : b);
    int32_t e = (int32_t)(((int64_t)gb * n_temps) / B_total);
    uint8_t* xb = x + (int64_t)b * n;
    double* nub = nu + (int64_t)b * n;
    float* nu32b = nu32 ? nu32 + (int64_t)b * n : NULL;
    double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    uint8_t* hid = (uint8_t*)malloc((size_t)(m > 0 ? m : 1) * OR_MAX_H);
    for (int32_t step = 0; step < T && !bad; ++step) {
      uint32_t t = t0 + (uint32_t)step;
      /* 1. score the current state, literal by literal */
      int64_t cb = assignment_cost(m, off, lits, w, xb);
      cost[b] = cb;
      /* 2. best-so-far (strict: the first state reaching a cost is kept) */
      if (cb < best_cost[b]) {
        best_cost[b] = cb;
        memcpy(best_x + (int64_t)b * n, xb, (size_t)n);
      }
      /* 3-4. hidden logits (Eq. 2 with Eq. 4), free energy (Eq. 1), draws */
      double F = 0.0;
      for (int64_t c = 0; c < m; ++c) {
        int32_t len = (int32_t)(off[c + 1] - off[c]);
        if (len == 0) continue; /* an empty clause has no clause RBM */
        int32_t j = weight_bucket(w ? w[c] : 1, wmin, n_buckets);
        int s = find_set(&tab, len, j, e);
        if (s < 0) { bad = 1; break; }
        double Wp[OR_MAX_LEN][OR_MAX_H], bp[OR_MAX_H];
        negation_transform(&tab, s, lits + off[c], len, Wp, bp);
        for (int32_t h = 0; h < tab.set_nh[s]; ++h) {
          double a = bp[h];
          for (int32_t k = 0; k < len; ++k) {
            int32_t l = lits[off[c] + k];
            int32_t v = (l > 0 ? l : -l) - 1;
            a += Wp[k][h] * (double)xb[v];
          }
          F -= softplus(a);
          uint32_t u = oracle_draw16(seed, PH_HID | (inst << 8), t, (uint32_t)c, (uint32_t)h, gb);
          hid[c * OR_MAX_H + h] = u < prob16(a);
        }
      }
      if (bad) break;
      free_energy[b] = F;
      /* 5. visible logits: the scatter-sum of Eq. 7 (d = 0) */
      for (int32_t i = 0; i < n; ++i) z[i] = 0.0;
      for (int64_t c = 0; c < m; ++c) {
        int32_t len = (int32_t)(off[c + 1] - off[c]);
        if (len == 0) continue;
        int32_t j = weight_bucket(w ? w[c] : 1, wmin, n_buckets);
        int s = find_set(&tab, len, j, e);
        double Wp[OR_MAX_LEN][OR_MAX_H], bp[OR_MAX_H];
        negation_transform(&tab, s, lits + off[c], len, Wp, bp);
        for (int32_t k = 0; k < len; ++k) {
          int32_t l = lits[off[c] + k];
          int32_t v = (l > 0 ? l : -l) - 1;
          double contrib = 0.0;
          for (int32_t h = 0; h < tab.set_nh[s]; ++h)
            contrib += Wp[k][h] * (double)hid[c * OR_MAX_H + h];
          z[v] += contrib;
        }
      }
      /* 6. nu moving average and visible draws (Eq. 3) */
      for (int32_t i = 0; i < n; ++i) {
        uint32_t P = prob16(z[i]);
        double rho = (double)P / 65536.0;
        nub[i] = (1.0 - alpha) * nub[i] + alpha * rho * (1.0 - rho);
        if (nu32b) {
          /* the same update in FP32 with a fixed operation order (the
           * precision the solver ranks variables in): var = fl(P (65536 - P))
           * 2^-32, nu = fma(1 - alpha, nu, fl(alpha var)) */
          const float a32 = (float)alpha;
          const float keep = 1.0f - a32;
          const float var = (float)(P * (65536u - P)) * 0x1p-32f;
          const float av = a32 * var;
          nu32b[i] = fmaf(keep, nu32b[i], av);
        }
        uint32_t u = oracle_draw16(seed, PH_VIS | (inst << 8), t, (uint32_t)i, 0u, gb);
        xb[i] = u < P;
      }
    }
    free(z);
    free(hid);
  }
  return bad ? -1 : 0;
}

/* Free energy of arbitrary assignments under the temperature-e parameters
 * (Eq. 1 summed over clauses as in Sec. 4.1). */
/* The formula free energy (Eq. 1) of B assignments at temperature `temp`
 * (F_out, FP64) and, when Fq_out is given, its fixed-point form: the sum over
 * clauses of rint(2^20 F_c) (int64), the exact quantity parallel-tempering
 * swaps compare. */
int oracle_free_energy(int32_t n, int64_t m, const int64_t* off, const int32_t* lits,
                       const int64_t* w, int32_t n_sets, const int32_t* set_len,
                       const int32_t* set_bucket, const int32_t* set_temp,
                       const int32_t* set_nh, const double* W, const double* bias,
                       int32_t n_buckets, int32_t temp, const uint8_t* x, int32_t B,
                       double* F_out, int64_t* Fq_out) {
  rbm_table tab = {n_sets, set_len, set_bucket, set_temp, set_nh, W, bias};
  int64_t wmin = INT64_MAX;
  for (int64_t c = 0; c < m; ++c) {
    int64_t wc = w ? w[c] : 1;
    if (wc < wmin) wmin = wc;
  }
  for (int32_t b = 0; b < B; ++b) {
    const uint8_t* xb = x + (int64_t)b * n;
    double F = 0.0;
    int64_t Fq = 0;
    for (int64_t c = 0; c < m; ++c) {
      int32_t len = (int32_t)(off[c + 1] - off[c]);
      if (len == 0) continue;
      int s = find_set(&tab, len, weight_bucket(w ? w[c] : 1, wmin, n_buckets), temp);
      if (s < 0) return -1;
      double Wp[OR_MAX_LEN][OR_MAX_H], bp[OR_MAX_H];
      negation_transform(&tab, s, lits + off[c], len, Wp, bp);
      double Fc = 0.0;
      for (int32_t h = 0; h < tab.set_nh[s]; ++h) {
        double a = bp[h];
        for (int32_t k = 0; k < len; ++k) {
          int32_t l = lits[off[c] + k];
          a += Wp[k][h] * (double)xb[(l > 0 ? l : -l) - 1];
        }
        Fc -= softplus(a);
      }
      F += Fc;
      Fq += (int64_t)nearbyint(ldexp(Fc, 20));
    }
    F_out[b] = F;
    if (Fq_out) Fq_out[b] = Fq;
  }
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Prioritized unit propagation (Sec. 4.4, after Si et al. 2019) on one     */
/* assignment x, ranking variables by nu (the solver's FP32 nu):            */
/*   1. order the variables by nu, highest first (ties: lower index);       */
/*   2. the first floor(n/2) keep their values from x (no propagation yet); */
/*   3. every clause that is not satisfied and has exactly one unassigned   */
/*      literal occurrence puts that literal on a queue (clauses in index   */
/*      order); the queue is emptied first-in first-out: a literal whose    */
/*      variable is unassigned is made true, and each clause of that        */
/*      variable (in index order) that becomes unit queues its literal;     */
/*   4. the remaining variables, in order, each take its value from x if   */
/*      still unassigned, and the queue is emptied again.                   */
/* Falsified clauses are left as they are (MaxSAT). out gets the result.    */
/* ---------------------------------------------------------------------- */
typedef struct {
  int32_t n;
  int64_t m;
  const int64_t* off;
  const int32_t* lits;
  const int64_t* voff;   /* n + 1 offsets into vocc */
  const int64_t* vocc;   /* literal positions j of each variable, clause order */
  int8_t* val;           /* -1 unassigned, else 0 / 1 */
  int32_t* nfalse;       /* false literal occurrences per clause */
  uint8_t* sat;          /* clause has a true literal */
  int32_t* queue;        /* literals (DIMACS) */
  int64_t qhead, qtail;
} up_state;

static void up_push_if_unit(up_state* S, int64_t c) {
  const int64_t len = S->off[c + 1] - S->off[c];
  if (S->sat[c] || len - S->nfalse[c] != 1) return;
  for (int64_t j = S->off[c]; j < S->off[c + 1]; ++j) {
    const int32_t l = S->lits[j];
    const int32_t v = (l > 0 ? l : -l) - 1;
    if (S->val[v] < 0) {
      S->queue[S->qtail++] = l;
      return;
    }
  }
}

/* assigns variable v := b and updates its clauses; with `check`, clauses
 * that become unit queue their open literal */
static void up_assign(up_state* S, int32_t v, int8_t b, int check) {
  S->val[v] = b;
  for (int64_t k = S->voff[v]; k < S->voff[v + 1]; ++k) {
    const int64_t j = S->vocc[k];
    int64_t c = 0;
    /* clause of literal position j (binary search over off) */
    int64_t lo = 0, hi = S->m;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) / 2;
      if (S->off[mid] <= j) lo = mid; else hi = mid;
    }
    c = lo;
    const int32_t l = S->lits[j];
    if ((l > 0) == (b == 1)) S->sat[c] = 1;
    else S->nfalse[c]++;
  }
  if (!check) return;
  for (int64_t k = S->voff[v]; k < S->voff[v + 1]; ++k) {
    const int64_t j = S->vocc[k];
    int64_t lo = 0, hi = S->m;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) / 2;
      if (S->off[mid] <= j) lo = mid; else hi = mid;
    }
    up_push_if_unit(S, lo);
  }
}

static void up_drain(up_state* S) {
  while (S->qhead < S->qtail) {
    const int32_t l = S->queue[S->qhead++];
    const int32_t v = (l > 0 ? l : -l) - 1;
    if (S->val[v] < 0) up_assign(S, v, (int8_t)(l > 0), 1);
  }
}

typedef struct { float key; int32_t idx; } up_rank;

static int up_rank_cmp(const void* a, const void* b) {
  const up_rank* x = (const up_rank*)a;
  const up_rank* y = (const up_rank*)b;
  if (x->key > y->key) return -1;
  if (x->key < y->key) return 1;
  return (x->idx > y->idx) - (x->idx < y->idx);
}

int oracle_unit_prop(int32_t n, int64_t m, const int64_t* off, const int32_t* lits,
                     const uint8_t* x, const float* nu, uint8_t* out) {
  const int64_t nnz = off[m];
  int64_t* voff = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* vocc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t j = 0; j < nnz; ++j) voff[(lits[j] > 0 ? lits[j] : -lits[j])]++;
  for (int32_t i = 0; i < n; ++i) voff[i + 1] += voff[i];
  for (int32_t i = 0; i < n; ++i) fill[i] = voff[i];
  for (int64_t j = 0; j < nnz; ++j) {  /* positions in increasing order: clause order */
    const int32_t v = (lits[j] > 0 ? lits[j] : -lits[j]) - 1;
    vocc[fill[v]++] = j;
  }
  up_state S = {n, m, off, lits, voff, vocc, (int8_t*)malloc((size_t)n),
                (int32_t*)calloc((size_t)(m > 0 ? m : 1), sizeof(int32_t)),
                (uint8_t*)calloc((size_t)(m > 0 ? m : 1), 1),
                (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz + m + 1)), 0, 0};
  memset(S.val, -1, (size_t)n);
  up_rank* order = (up_rank*)malloc(sizeof(up_rank) * (size_t)n);
  for (int32_t i = 0; i < n; ++i) { order[i].key = nu[i]; order[i].idx = i; }
  qsort(order, (size_t)n, sizeof(up_rank), up_rank_cmp);
  const int32_t half = n / 2;
  for (int32_t r = 0; r < half; ++r) up_assign(&S, order[r].idx, (int8_t)(x[order[r].idx] != 0), 0);
  for (int64_t c = 0; c < m; ++c) up_push_if_unit(&S, c);
  up_drain(&S);
  for (int32_t r = half; r < n; ++r) {
    const int32_t v = order[r].idx;
    if (S.val[v] < 0) {
      up_assign(&S, v, (int8_t)(x[v] != 0), 1);
      up_drain(&S);
    }
  }
  for (int32_t i = 0; i < n; ++i) out[i] = (uint8_t)S.val[i];
  free(voff); free(vocc); free(fill); free(S.val); free(S.nfalse); free(S.sat); free(S.queue);
  free(order);
  return 0;
}

int oracle_max_len(void) { return OR_MAX_LEN; }
int oracle_max_hidden(void) { return OR_MAX_H; }
