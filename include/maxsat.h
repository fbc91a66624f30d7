/*
 * maxsat.h -- C ABI of the GB300 RbmSAT library (libmaxsat.so).
 *
 * RbmSAT ("Solving MaxSAT with Matrix Multiplication") turns a CNF formula into
 * a Restricted Boltzmann Machine whose free energy falls with every satisfied
 * clause (Sec. 4.1) and searches with block Gibbs sampling over many parallel
 * chains (Sec. 4.2), keeping the best assignment seen. Each Gibbs round is:
 *   - the "gather": every clause reads the truth of its literals for every
 *     chain (Sec. 4.3), giving the weighted unsatisfied cost and the clause
 *     free energy (Eq. 1);
 *   - hidden units drawn from p(h | v) (Eq. 2, Eq. 6) after the negation
 *     transform of the canonical OR-gate RBM (Eq. 4);
 *   - the "scatter-add" of the hidden units' contributions into the visible
 *     logits (Eq. 7) and new visible states drawn from p(v | h) (Eq. 3),
 *     plus the moving average nu of the conditional variance (Sec. 4.4);
 *   - best-so-far tracking (Sec. 4.2).
 *
 * Conventions (all entry points):
 *   - Return MAXSAT_OK (0) or a negative MAXSAT_E* code; the message is then
 *     available from maxsat_last_error(ctx) (or maxsat_last_error(NULL) when
 *     maxsat_create itself failed).
 *   - Assignments at the ABI are bytes, 1 = True, 0 = False, chain-major
 *     (B rows of n bytes). Any nonzero byte reads as True.
 *   - Pointers named *_dev are device pointers on the context's device; all
 *     others are host pointers. The caller owns every buffer it passes; the
 *     library copies what it keeps and never frees caller memory.
 *   - All device work is ordered on the CUDA stream given to maxsat_create.
 *     Calls that return results in host memory synchronise that stream.
 *   - A context is not thread-safe: one thread at a time per context.
 *   - There is no CPU fallback: without an sm_103 device every call that needs
 *     one fails with MAXSAT_ENODEV.
 */
#ifndef MAXSAT_H_
#define MAXSAT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MAXSAT_OK 0
#define MAXSAT_EINVAL (-1)    /* bad argument or an exactness precondition fails */
#define MAXSAT_ENOMEM (-2)    /* device or host allocation failed */
#define MAXSAT_ECUDA (-3)     /* a CUDA runtime call failed */
#define MAXSAT_ENODEV (-4)    /* no sm_103 device */
#define MAXSAT_ESTATE (-5)    /* call out of order (e.g. step before reset) */

#define MAXSAT_MAX_LEN 12     /* longest clause with an OR-gate RBM */
#define MAXSAT_MAX_HIDDEN 16  /* most hidden units per clause RBM */

#define MAXSAT_PATH_AUTO 0    /* measured choice: the first maxsat_reset for a
                                 given B times a few rounds of the sparse path,
                                 then of the dense path unless its two tensor-
                                 core products alone, at the GB300's nominal
                                 dense peaks, would take longer than the
                                 measured sparse round (the dense operands are
                                 built then, when exact and within 8 GB), and
                                 keeps the faster */
#define MAXSAT_PATH_DENSE 1   /* tensor-core products over dense operands */
#define MAXSAT_PATH_SPARSE 2  /* gather / pull-scatter over the literal lists */

/* One canonical (un-negated) OR-gate clause RBM: Sec. 4.1 "OR gate as an
 * RBM", general per-position weights W in R^{len x n_hidden} and hidden biases
 * b, no visible bias. It serves clauses of length `len` in weight bucket
 * `bucket` on chains of temperature `temp`. Every W entry must be a multiple
 * of 2^-quant_bits and every b entry a multiple of 2^-24 below 2^20 in
 * magnitude, so that every hidden logit is an exact double and every visible
 * logit an exact multiple of 2^-quant_bits (maxsat_fit_or_rbm returns such
 * values). The arrays are read during maxsat_create only. */
typedef struct {
  int32_t len;       /* 1 .. MAXSAT_MAX_LEN */
  int32_t bucket;    /* 0 .. n_buckets - 1 */
  int32_t temp;      /* 0 .. n_temps - 1 */
  int32_t n_hidden;  /* 1 .. MAXSAT_MAX_HIDDEN */
  const double* W;   /* len x n_hidden, row-major (row k = clause position k) */
  const double* b;   /* n_hidden */
} maxsat_rbm_set;

/* Solver parameters; maxsat_default_params fills the defaults. */
typedef struct {
  int32_t n_temps;       /* temperature ensemble size E (Sec. 4.2); default 2 */
  const double* fstar;   /* E targets F* (F_s = -F*); NULL = {0.068, 0.528}, the
                            paper's 1-TPU condition (appendix "Pretraining") */
  int32_t n_buckets;     /* weight buckets J (a reading: the paper is unweighted);
                            clause c uses bucket min(J-1, floor(log2(w_c / w_min)));
                            default 4 */
  double bucket_gamma;   /* bucket j fits target F* (1 + j gamma); default 0.5 */
  double alpha;          /* rate of the nu moving average (Sec. 4.4; the paper
                            gives none); default 0.01 */
  int32_t quant_bits;    /* Q: W on the 2^-Q grid; default 4 */
  int32_t path;          /* MAXSAT_PATH_*; default AUTO */
  int32_t fit_iters;     /* Adam iterations when fitting (lr 1e-3, appendix
                            "Pretraining"; the paper gives no count);
                            default 50000 */
  int32_t n_sets;        /* 0 with sets == NULL: fit every needed set at create */
  const maxsat_rbm_set* sets;
  int32_t steps_per_graph; /* Gibbs rounds per CUDA-graph launch (the paper runs
                              500 rounds per device dispatch); default 100:
                              the rounds' kernels overlap at their boundaries
                              (programmatic dependent launch), so longer
                              graphs run no faster and take longer to build;
                              0 = plain launches */
  int32_t tune_blocks;   /* 1: at the first maxsat_reset for each B, time a few
                            clause-block sizes of the sparse gather, then the
                            visible update's load batch (2, 4 or 8 incidences
                            in flight per thread), 6 rounds each in two
                            passes with CUDA events, and keep the fastest.
                            Costs, states and draws do not depend on either;
                            the free energy's float summation order depends
                            on the blocking. Default 0 (the wave-fitted size,
                            batch 4) */
  int32_t up_device;     /* 1: maxsat_up_begin / maxsat_up_end run unit
                            propagation and the merge on the GPU when the
                            chains are on the sparse path and one chain's
                            ranking state (8 n_pad + n bytes, n the
                            variables of the largest formula, n_pad = n
                            rounded up to a power of two) fits in 200 KB of
                            shared memory; otherwise, and with 0, on host
                            threads as the paper does (single formulas
                            only). Same results either way. Default 1 */
  int32_t visible_batch; /* incidences per thread whose hidden-pattern loads
                            the sparse visible update keeps in flight: 2, 4
                            or 8, or 0 for 4 unless tune_blocks measures
                            another. Same results for every value. Default 0 */
  int32_t persistent_round; /* 1: maxsat_step runs its sparse rounds as one
                            persistent cooperative launch per
                            max(1, steps_per_graph) rounds: every block
                            resident, the gather's and the visible update's
                            blocks walked by the same CTAs, grid barriers
                            between the phases (bounded waits: a wait that
                            gives up after about 2 s makes the next
                            maxsat_solve / maxsat_get_state fail with
                            MAXSAT_ECUDA). Only for clauses of at most 3
                            literals on single-temperature chain octets,
                            without profiling and while no GPU unit
                            propagation is pending; otherwise the two-launch
                            round runs (maxsat_get_persistent_round tells).
                            Same results bit for bit. Default 0 (two launches
                            per round with programmatic dependent launch,
                            replayed from CUDA graphs) */
} maxsat_params;

typedef struct maxsat_ctx maxsat_ctx;

/* Fills *p with the defaults listed above. */
void maxsat_default_params(maxsat_params* p);

/* Builds a solver for one weighted CNF formula.
 *   n_vars      number of variables n >= 1
 *   n_clauses   number of clauses m >= 0
 *   clause_off  m + 1 host int64 offsets into lits, clause_off[0] = 0,
 *               non-decreasing; clause c holds lits[clause_off[c] ..
 *               clause_off[c+1]) (at most MAXSAT_MAX_LEN literals)
 *   lits        DIMACS literals: +v is variable v (1-based) true, -v false
 *               (the signed index table T of Sec. 4.3); duplicates and x OR
 *               NOT x are allowed; an empty clause is never satisfied
 *   weights     m host int64 weights >= 1, or NULL for all 1
 *   params      NULL for the defaults
 *   cuda_stream cudaStream_t (as void*) all work is ordered on; NULL = legacy
 *               default stream
 * Fits any missing OR-gate RBM sets (Sec. 4.1), builds the probability and
 * free-energy tables and copies the formula to the device. *out receives the
 * context (NULL on failure). */
int maxsat_create(maxsat_ctx** out, int32_t n_vars, int64_t n_clauses,
                  const int64_t* clause_off, const int32_t* lits,
                  const int64_t* weights, const maxsat_params* params,
                  void* cuda_stream);

/* Builds one solver for a batch of n_inst independent weighted CNF formulas
 * of uneven size, run together in every launch. The paper runs independent
 * chains side by side and suggests clustering clauses by size (Sec. 4.2,
 * Sec. 5 "Datasets"); a batch extends this to many formulas.
 *   n_inst      number of formulas, 1 .. 65535
 *   n_vars      n_inst host int32: variables of each formula (>= 1)
 *   n_clauses   n_inst host int64: clauses of each formula (>= 0)
 *   clause_off  (sum of n_clauses) + 1 host int64 offsets into lits over the
 *               formulas' clauses concatenated in order, clause_off[0] = 0
 *   lits        DIMACS literals local to each formula (1 .. n_vars[k])
 *   weights     per clause as in maxsat_create (concatenated), or NULL
 * The context then behaves as one formula over the union of the variables
 * (formula k's variables follow those of formulas 0 .. k-1), except that
 * costs and the best-so-far are kept per formula: with B restarts, formula
 * k has its own B chains, and
 *   maxsat_eval       cost_dev is n_inst x B (row k: formula k's cost of
 *                     each assignment; assign_dev is B x total variables),
 *   maxsat_solve      best_assign gets every formula's best assignment
 *                     (total variables bytes) and best_cost n_inst values,
 *   maxsat_get_state / maxsat_set_state
 *                     best_cost, cost, free_energy are n_inst x B.
 * Draws of formula k use its own clause and variable indices with k in bits
 * 8..31 of the Philox phase word, so each formula follows exactly the
 * trajectory it would follow alone under that index. Weight buckets are
 * relative to each formula's lightest clause. Sparse path only
 * (MAXSAT_PATH_DENSE fails with MAXSAT_EINVAL; AUTO uses the sparse path).
 * Errors: MAXSAT_EINVAL for a bad count, offset or literal (the message
 * names the formula), MAXSAT_ENOMEM, MAXSAT_ECUDA, MAXSAT_ENODEV. */
int maxsat_create_batch(maxsat_ctx** out, int32_t n_inst, const int32_t* n_vars,
                        const int64_t* n_clauses, const int64_t* clause_off,
                        const int32_t* lits, const int64_t* weights,
                        const maxsat_params* params, void* cuda_stream);

/* Number of formulas of the context (1 unless made by maxsat_create_batch),
 * or a negative code. */
int maxsat_get_n_instances(const maxsat_ctx* ctx);

/* Clauses per block of the sparse gather for the current chains (wave-fitted
 * to the SM count, or measured with params.tune_blocks); 0 before the first
 * maxsat_reset; a negative code for a NULL context. */
int maxsat_get_clause_block(const maxsat_ctx* ctx);

/* Incidences per thread whose hidden-pattern loads the sparse visible update
 * keeps in flight together (params.visible_batch, else 4 or measured with
 * params.tune_blocks); a negative code for a NULL context. */
int maxsat_get_visible_batch(const maxsat_ctx* ctx);

/* 1 when maxsat_step runs the current chains' rounds as persistent launches
 * (params.persistent_round and the context qualifies), 0 when it runs the
 * two-launch round; a negative code for a NULL context. */
int maxsat_get_persistent_round(const maxsat_ctx* ctx);

/* Starts B fresh chains (Fig. code initialisation): every variable drawn
 * uniformly (Bernoulli(0.5)), nu = 0.25, best cost = INT64_MAX, step t = 0. */
int maxsat_reset(maxsat_ctx* ctx, int32_t restarts, uint64_t seed);

/* maxsat_reset for one shard of a larger ensemble (chains are independent,
 * Sec. 4.2): the local chains are chains chain_offset .. chain_offset + B - 1
 * of an ensemble of total_chains. Every draw and the temperature block of a
 * chain follow its global index, so shards on several GPUs together run
 * exactly the chains of one total_chains run. chain_offset must be a
 * multiple of 8; maxsat_reset(ctx, B, seed) is the shard (0, B). */
int maxsat_reset_shard(maxsat_ctx* ctx, int32_t restarts, uint64_t seed,
                       int32_t chain_offset, int32_t total_chains);

/* Runs `steps` Gibbs rounds on the current chains. Round t scores the current
 * state x_t (cost, free energy), keeps it if its cost is strictly below the
 * chain's best, draws h ~ p(h | x_t) and x_{t+1} ~ p(v | h) and updates nu.
 * Asynchronous on the context's stream. */
int maxsat_step(maxsat_ctx* ctx, int64_t steps);

/* Scores the current states and updates the best-so-far without drawing
 * (the evaluation after the last round, so rounds 0..T-1 plus this score
 * x_0 .. x_T). Asynchronous. */
int maxsat_score(maxsat_ctx* ctx);

/* Weighted unsatisfied cost of B arbitrary assignments (the MaxSAT objective,
 * Sec. 1). assign_dev: B x n device bytes, row-major, 0 = false and 1 =
 * true, no alignment required; cost_dev: B device int64 (n_inst x B for a
 * batch). Independent of the chains. Asynchronous; a call with a larger B
 * than any before grows the evaluation scratch first. */
int maxsat_eval(maxsat_ctx* ctx, const uint8_t* assign_dev, int32_t B,
                int64_t* cost_dev);

/* reset + `steps` rounds + score, then copies the best assignment over all
 * chains (lowest cost, ties to the lowest chain index) to best_assign (n host
 * bytes, may be NULL) and its cost to *best_cost (a batch: per formula, see
 * maxsat_create_batch). Synchronises. */
int maxsat_solve(maxsat_ctx* ctx, int32_t restarts, int64_t steps, uint64_t seed,
                 uint8_t* best_assign, int64_t* best_cost);

/* maxsat_solve under a wall-clock budget: the search samples until the time
 * limit and outputs the best assignment seen (Sec. 4.2; 300 s per instance in
 * the experiments, Sec. 5 "Incomplete score metric"; the appendix code
 * returns when its time budget is exhausted). reset, then chunks of
 * `chunk` rounds (<= 0: max(1, steps_per_graph)), each synchronised, while
 * less than `seconds` of host wall time have passed since the call and
 * fewer than max_steps rounds have run (the last chunk is cut to max_steps);
 * then the final score and the best as maxsat_solve. *steps_done (may be
 * NULL) receives the rounds run; with the same seed the result equals
 * maxsat_solve with that many steps. MAXSAT_EINVAL for a negative or NaN
 * budget. Synchronises. */
int maxsat_solve_timed(maxsat_ctx* ctx, int32_t restarts, double seconds, int64_t max_steps,
                       int64_t chunk, uint64_t seed, uint8_t* best_assign,
                       int64_t* best_cost, int64_t* steps_done);

/* Copies chain state to host buffers (each may be NULL): x and best_x are
 * B x n bytes, nu is B x n float, best_cost / cost are B int64 (cost = last
 * scored state), free_energy B float (last scored state, Eq. 1 summed over
 * clauses), *t the next round's index; for a batch best_cost, cost and
 * free_energy are n_inst x B. Synchronises. */
int maxsat_get_state(maxsat_ctx* ctx, uint8_t* x, float* nu, int64_t* best_cost,
                     uint8_t* best_x, int64_t* cost, float* free_energy,
                     uint32_t* t);

/* Restores chain state (checkpoint resume): B chains, the seed they were
 * started with, x / nu / best_cost / best_x as returned by maxsat_get_state and
 * the round index t. With the counter-based randomness, resuming continues
 * the same trajectory bit for bit. Synchronises. */
int maxsat_set_state(maxsat_ctx* ctx, int32_t restarts, uint64_t seed,
                     const uint8_t* x, const float* nu, const int64_t* best_cost,
                     const uint8_t* best_x, uint32_t t);

/* One parallel-tempering swap round between adjacent temperatures (the
 * ensemble of Sec. 4.2 with replica exchange; the paper lists tempering as
 * future work, Sec. 7). With E temperatures and restarts = E x S (S a
 * multiple of 8; whole ensemble on this context; sparse path), chain a =
 * e S + k of every block e = parity, parity + 2, ... (e + 1 < E) and chain
 * b = a + S exchange states x and nu iff
 *   D = F_e(x_a) + F_{e+1}(x_b) - F_e(x_b) - F_{e+1}(x_a) >= ceil(2^20 ln(u / 65536)),
 * the Metropolis rule min(1, exp(D)) for the targets exp(-F_e): F is the
 * exact fixed-point free energy sum_c rint(2^20 F_c) (Eq. 1 per clause) and
 * u the 16-bit draw of chain a at counter (0, a >> 3, current round, phase
 * 4), lane a & 7 (u = 0 always accepts). The best-so-far stays with the
 * chain index; the round index does not advance. *accepted (may be NULL)
 * receives the number of swaps (synchronises). MAXSAT_EINVAL when the
 * conditions above fail, MAXSAT_ESTATE without chains. */
int maxsat_pt_swap(maxsat_ctx* ctx, int32_t parity, int32_t* accepted);

/* Prioritized unit propagation with the B-of-2B merge (Sec. 4.4; the
 * appendix code's send / fetch / merge). maxsat_up_begin takes a snapshot of
 * the chains' states x and their nu and starts unit propagation: on the GPU
 * (params.up_device, one warp per chain on a side stream; the snapshot is a
 * device copy ordered on the context's stream), else on host threads after
 * copying the snapshot to the host. It returns at once; maxsat_step may run
 * meanwhile, as the paper keeps sampling while the host works. For each chain: variables ranked by
 * nu, highest first (ties to the lower index); the top floor(n/2) keep their
 * values; unit clauses are propagated first in, first out; the remaining
 * variables, in rank order, take their values from x when still unassigned,
 * each followed by propagation. maxsat_up_end waits for the results, scores
 * the B current states and the B propagated ones (exact costs), and keeps
 * the B with the lowest costs: sorted by satisfied weight ascending with a
 * stable sort over [current states, propagated states], the last B become
 * chains 0..B-1 in that order, each propagated state with the nu of the
 * chain it came from. The best-so-far of each chain is kept. maxsat_up is
 * begin + end. A batch of formulas (maxsat_create_batch) runs in the GPU form
 * only, every formula with its own B chains, ranking and merge
 * (MAXSAT_EINVAL otherwise); MAXSAT_ESTATE without chains, for a second
 * begin, for end without begin,
 * or when the chains were reset in between. The host form synchronises; the
 * GPU form's merge is ordered on the context's stream (scoring with the
 * sparse eval gather, a stable rank by counting, a column permutation). */
int maxsat_up_begin(maxsat_ctx* ctx);
int maxsat_up_end(maxsat_ctx* ctx);
int maxsat_up(maxsat_ctx* ctx);

/* ---------------------------------------------------------------------
 * Learned proposal: a message-passing network over the variable-clause
 * incidence that predicts p(x_v = 1) from the formula alone, trained on the
 * solver's own best assignments, and used as the distribution of the chains'
 * initial states (the paper names learned initial assignments as
 * complementary to RbmSAT, Sec. 2). With hidden size 64 and L layers:
 *   f_v = [pos_v / deg_v - 1/2, log(1 + deg_v) / 4, 1]
 *   g_c = [log(w_c) / 8, len_c / 4, 1]
 *   h_v^0 = relu(Wf f_v), h_c^0 = relu(Wg g_c)
 *   layer l: m_c = mean over c's literals of s h_v^{l-1};
 *            h_c^l = relu(Wc_l [m_c ; h_c^{l-1}] + bc_l);
 *            a_v = mean over v's occurrences of s h_c^l;
 *            h_v^l = relu(Wv_l [a_v ; h_v^{l-1}] + bv_l)
 *   z_v = wo . h_v^L + bo, p_v = sigmoid(z_v); loss = mean BCE(z_v, y_v)
 * (s = +1 / -1 for a plain / negated literal). The flat FP32 parameter
 * vector holds, in order: Wf (64 x 3), Wg (64 x 3), then per layer Wc (64 x
 * 128), bc (64), Wv (64 x 128), bv (64), then wo (64), bo (1), matrices
 * row-major. Weight matrices are used in BF16 (round to nearest even of the
 * FP32 master); activations and sums are FP32. Work runs on the stream of
 * the formula context passed in. */
typedef struct maxsat_mp maxsat_mp;

/* New network with L layers (1..8), He-normal weights from `seed`, zero
 * biases, Adam moments zero. MAXSAT_ENODEV without a device. */
int maxsat_mp_create(maxsat_mp** out, int32_t n_layers, uint64_t seed);
/* Number of parameters (the flat vector's length). */
int maxsat_mp_n_params(const maxsat_mp* mp);
/* Replaces the parameters (host FP32 vector) and clears the Adam state. */
int maxsat_mp_set_params(maxsat_mp* mp, const float* theta);
/* Copies the parameters and / or the last gradient to host buffers (NULL to
 * skip). Synchronises. */
int maxsat_mp_get_params(maxsat_mp* mp, float* theta, float* grad);
/* p_v for every variable of ctx's formula (a batch: every formula at once)
 * into prob_dev (n device floats). Asynchronous on ctx's stream. */
int maxsat_mp_forward(maxsat_mp* mp, maxsat_ctx* ctx, float* prob_dev);
/* Forward and backward against labels (n device bytes, 0 / 1): the
 * gradient of the mean binary cross entropy is kept for maxsat_mp_adam;
 * *loss (may be NULL) receives the loss (synchronises when given). */
int maxsat_mp_gradient(maxsat_mp* mp, maxsat_ctx* ctx, const uint8_t* labels_dev,
                       double* loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected) with the last
 * gradient, then the BF16 weights are refreshed. */
int maxsat_mp_adam(maxsat_mp* mp, maxsat_ctx* ctx, float lr);
const char* maxsat_mp_last_error(const maxsat_mp* mp);
void maxsat_mp_destroy(maxsat_mp* mp);

/* Flip proposals from the learned network: every chain proposes its state
 * with each confident variable set to the network's value (1 where prob[v]
 * >= 1 - tau, 0 where prob[v] <= tau; prob: n host floats, tau in [0,
 * 0.5)); the B current states and the B proposals are scored exactly and
 * merged as in maxsat_up_end (stable sort by satisfied weight over [current,
 * proposals], the last B become chains 0..B-1, a proposal keeps its chain's
 * nu; the best-so-far is kept). On the sparse path the proposals and the
 * merge run on the device, and a batch of formulas merges every formula
 * separately (prob: the batch's n variables); the dense path merges on the
 * host, single formulas only. Synchronises. */
int maxsat_propose_flips(maxsat_ctx* ctx, const float* prob, float tau);

/* maxsat_reset, except that variable v of every chain starts True with
 * probability prob[v] (n host floats in [0, 1]): x = [u < P_v], P_v =
 * rint(65536 prob[v]) in FP64, u the same 16-bit initial draw as
 * maxsat_reset (prob = 1/2 everywhere gives exactly maxsat_reset's states).
 * Synchronises. */
int maxsat_reset_probs(maxsat_ctx* ctx, int32_t restarts, uint64_t seed, const float* prob);

/* Per-kernel timing. While profiling is on, maxsat_step and maxsat_score use
 * plain launches (no CUDA graph) and bracket every kernel launch with CUDA
 * events on the context's stream (the learned proposal's launches on that
 * context too, named mp_*); maxsat_kernel_times then synchronises and
 * reports, per kernel name, the number of launches and their total device
 * time in milliseconds since profiling was switched on. names receives up to
 * max_kernels NUL-terminated names of at most 31 characters (32 bytes each).
 * Returns the number of kernels reported (>= 0) or a negative code. */
int maxsat_set_profiling(maxsat_ctx* ctx, int32_t on);
int maxsat_kernel_times(maxsat_ctx* ctx, int32_t max_kernels, char* names,
                        int64_t* launches, double* total_ms);

/* Which path the Gibbs rounds run on (MAXSAT_PATH_DENSE or _SPARSE); with
 * MAXSAT_PATH_AUTO the choice is made by the first maxsat_reset for each B. */
int maxsat_get_path(const maxsat_ctx* ctx);

/* Allocation-free cost evaluation (the paper has no counterpart: it is an
 * interface for callers that cannot allocate device memory). Some callers
 * cannot call cudaMalloc: frameworks whose own caching allocator owns the
 * device memory budget (an allocation behind its back can fail or fragment
 * its pool), and latency-critical loops that cannot take the implicit device
 * synchronisation that cudaMalloc or cudaFree may cause. This call allocates
 * nothing (no cudaMalloc, no cudaFree, no allocating library routine) and
 * needs no context: it computes the same weighted unsatisfied costs as
 * maxsat_eval for a formula held in the caller's device memory.
 *   n_vars, n_clauses, n_lits  sizes (n_lits = clause_off[n_clauses])
 *   clause_off_dev  n_clauses + 1 device int64 offsets (as maxsat_create)
 *   lits_dev        n_lits device int32 DIMACS literals (as maxsat_create);
 *                   offsets are clamped to [0, n_lits] and literals outside
 *                   [-n_vars, n_vars] \ {0} are skipped (a clause left with
 *                   no literal is unsatisfied), so nothing is read outside
 *                   the caller's buffers when the sizes given are theirs
 *   weights_dev     n_clauses device int64 weights, or NULL for all 1
 *   assign_dev      B x n_vars device bytes (nonzero = true); cost_dev: B int64
 * Its scratch memory (the assignments transposed to variable-major,
 * n_vars x B' bytes rounded up to 256, plus int64 cost partials,
 * ceil(n_clauses / max(64, ceil(n_clauses / 256))) x B' x 8 bytes, with B'
 * = B rounded up to 256) is one file-scope device array of
 * MAXSAT_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds
 * until exit; larger requests fail with MAXSAT_EINVAL before any launch. The
 * first call on each device looks the array's address up
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * Every call overwrites all of the scratch it reads, but all calls share the
 * one array: calls that overlap on the GPU (different streams or host
 * threads) race. Asynchronous on cuda_stream; every launch is checked before
 * the next is issued; on failure maxsat_last_error(NULL) gives the message. */
#define MAXSAT_NOALLOC_SCRATCH_BYTES (32u << 20)
int maxsat_eval_noalloc(int32_t n_vars, int64_t n_clauses, int64_t n_lits,
                        const int64_t* clause_off_dev, const int32_t* lits_dev,
                        const int64_t* weights_dev, const uint8_t* assign_dev,
                        int32_t B, int64_t* cost_dev, void* cuda_stream);

/* Frees the context and its device memory (NULL is a no-op). */
void maxsat_destroy(maxsat_ctx* ctx);

/* Message of the last failed call on ctx (or of the last failed
 * maxsat_create when ctx is NULL); "" when none. Valid until the next call. */
const char* maxsat_last_error(const maxsat_ctx* ctx);

/* Fits one canonical OR-gate RBM on the host (Sec. 4.1): minimises
 * F(0)^2 + sum_{v != 0} (F(v) - F_s)^2 over all 2^len inputs with Adam at
 * learning rate 1e-3, F_s = -fstar; then rounds W to the 2^-quant_bits grid,
 * refits b with W fixed and rounds b to the 2^-24 grid. W_out: len x n_hidden
 * row-major, b_out: n_hidden (host). No device needed. */
int maxsat_fit_or_rbm(int32_t len, int32_t n_hidden, double fstar,
                      int32_t quant_bits, int32_t iters, double* W_out,
                      double* b_out);

#ifdef __cplusplus
}
#endif

#endif /* MAXSAT_H_ */
