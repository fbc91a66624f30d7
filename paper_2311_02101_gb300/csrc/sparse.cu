// Sparse-gather path of one RbmSAT Gibbs round.
//
// The paper's experiments use the accelerator's vector unit with gathers for
// the clause inputs and a segment-sum for the scatter-add (appendix "Gather
// and scatter-add operations"); this is the GB300 counterpart. It works
// directly on the literal lists, never on a dense clause-variable matrix:
//   k_gather   one thread = one clause x 8 chains: reads the clause's literal
//              truths for 8 chains at once (8 bytes per literal from the
//              variable-major state), forms each chain's truth pattern, adds
//              the weight of unsatisfied clauses and the clause free energy
//              (Eq. 1), draws the hidden units (Eq. 2 / Eq. 6) and stores the
//              hidden pattern (one byte per clause and chain). The last block
//              to finish a tile of 256 chains reduces the per-block costs in a
//              fixed order and keeps improving states (Sec. 4.2).
//   k_visible  one thread = one variable x 8 chains: pull-based scatter-sum
//              over the variable's literals of the contribution table entry
//              selected by the clause's hidden pattern (Eq. 7; integer sums,
//              no atomics, deterministic), draws the new visible states
//              (Eq. 3), updates nu (Sec. 4.4) and copies improved states into
//              the best-so-far before they are overwritten.
// State layout: x and nu are variable-major (n x Bp) so 8 consecutive chains of
// one variable are one 8-byte (x) or 32-byte (nu) access. The small
// probability tables are staged in shared memory when they fit.
// A batch of formulas is their disjoint union: every instance has its own B
// chains in the same chain columns, clause blocks never straddle two
// instances (GatherPlan), per-instance costs and best-so-far live in
// n_inst x Bp arrays, and draws use the instance's own clause and variable
// indices with the instance index in bits 8..31 of the phase word, so each
// instance follows the trajectory it would follow alone under that index.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "internal.h"
#include "philox.cuh"

namespace rbmsat {

namespace {

__device__ __forceinline__ uint32_t step_index(const uint32_t* tdev, uint32_t t_rel) {
  return (tdev ? *tdev : 0u) + t_rel;
}

// Copies `bytes` (multiple of 16) from global to shared memory, whole block.
__device__ __forceinline__ void stage(void* dst, const void* src, int bytes) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = __ldg(s + i);
}

__host__ __device__ __forceinline__ int align16(int bytes) { return (bytes + 15) & ~15; }

// Programmatic dependent launch between the rounds' kernels: a gather or
// visible launch may start while its predecessor in the stream finishes. It
// lets its own dependent start early (release), stages its constant tables,
// and waits for the predecessor's completion and memory (griddepcontrol.wait)
// before it reads or writes any chain state. Without a programmatic
// predecessor both are no-ops.
__device__ __forceinline__ void pdl_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// (instance, index within it) of variable i
__device__ __forceinline__ int2 var_instance(const DevFormula& F, int i) {
  return F.var_inst ? __ldg(F.var_inst + i) : make_int2(0, i);
}

// Kernels over variables take vg0, the first group of 8 variables of this
// launch (grids have at most 65535 groups; larger n takes several launches).
__global__ void __launch_bounds__(256) k_init(DevFormula F, DevChains C, int n, int vg0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g8 = blockIdx.x * 32 + lane, b0 = g8 * 8;
  const int i = (vg0 + blockIdx.y) * 8 + warp;
  if (i < n) {
    const int2 vi = var_instance(F, i);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)vi.y, (uint32_t)(g8 + C.g8_off), 0u,
                                             kPhaseInit | ((uint32_t)vi.x << 8)),
                                  C.keys);
    uint64_t x = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) x |= (uint64_t)(lane16(r, q) < 32768u) << (8 * q);
    const size_t o = (size_t)i * C.Bp + b0;
    *reinterpret_cast<uint64_t*>(C.xt + o) = x;
    *reinterpret_cast<uint64_t*>(C.best_xt + o) = x;
    const float4 v = make_float4(0.25f, 0.25f, 0.25f, 0.25f);
    reinterpret_cast<float4*>(C.nu + o)[0] = v;
    reinterpret_cast<float4*>(C.nu + o)[1] = v;
  }
  if (vg0 + blockIdx.y == 0) {
    for (int in = warp; in < C.n_inst; in += 8) {
      const size_t ib = (size_t)in * C.Bp + b0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        C.best[ib + q] = INT64_MAX;
        C.improved[ib + q] = 0;
      }
      if (lane == 0) C.tickets[in * gridDim.x + blockIdx.x] = 0;
    }
  }
}

template <int MODE, bool SM, typename HT, bool ONE>
// 4 blocks per SM for one-chunk records (64 registers: a few loop-invariant
// values spill, and the fuller SM is 0.7 % faster per round at weighted
// 3-SAT n = 1000, m = 6000, 4096 chains); 3 for longer records, which spill
// far more at 64 registers
__global__ void __launch_bounds__(256, ONE ? 4 : 3) k_gather(DevFormula F, DevTables T, DevChains C,
                                                const uint8_t* __restrict__ xt, int B, int Bp,
                                                GatherPlan P, const uint32_t* tdev,
                                                uint32_t t_rel, int64_t* cost_part,
                                                float* fe_part, int32_t* tickets,
                                                int64_t* eval_out) {
  constexpr bool FE = MODE != kEval;
  constexpr bool SAMPLE = MODE == kStep;
  pdl_release();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int64_t s_cost[8][256];
  __shared__ float s_fe[8][256];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g8 = blockIdx.x * 32 + lane, b0 = g8 * 8;
  // this block's clauses: one instance, clauses c_begin .. c_end - 1
  const int4 bd = __ldg(P.blk + blockIdx.y);
  const int inst = bd.x, c_begin = bd.y, c_end = bd.z, cl_base = bd.w;
  const uint32_t phase_h = kPhaseHidden | ((uint32_t)inst << 8);
  const int E = T.n_temps;

  const GroupMeta* meta = T.meta;
  const uint32_t* rec = T.rec;
  if (SM && FE) {
    const int mb = align16(T.n_groups * (int)sizeof(GroupMeta));
    stage(smem, T.meta, mb);
    stage(smem + mb, T.rec, align16(T.rec_len * 4));
    __syncthreads();
    meta = reinterpret_cast<const GroupMeta*>(smem);
    rec = reinterpret_cast<const uint32_t*>(smem + mb);
  }

  // temperature of the thread's 8 chains: one value unless a temperature
  // block boundary falls inside them
  // global chain index: draws and temperatures follow it (chain shards)
  const int gb0 = C.g8_off * 8 + b0;
  const int e0 = FE ? temp_of(gb0, E, C.B_total, C.inv_B_total) : 0;
  const bool e_uniform = !FE || e0 == temp_of(gb0 + 7, E, C.B_total, C.inv_B_total);
  // UNI form of the clause loop (below) when every lane of the warp has one
  // temperature; only the one-chunk kernel carries both forms (the longer
  // records' kernel is at its register limit)
  const bool warp_uni = !ONE || __all_sync(0xFFFFFFFFu, e_uniform);
  // the 8 chains' temperatures, 6 bits each (E <= 64); filled for every lane
  // of a warp that takes the per-chain form
  uint64_t epack = 0;
  if (FE && (!ONE || !warp_uni)) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      epack |= (uint64_t)(e_uniform ? e0 : temp_of(gb0 + q, E, C.B_total, C.inv_B_total))
               << (6 * q);
  }
  // the weighted unsat cost accumulates in this warp's shared-memory row
  // (each entry is owned by one thread), the free energy in registers
  // (32-bit rows when every block's weight sum fits: C.cost32). Each thread
  // zeroes only the entries it owns in the view in use.
  int64_t* my_cost = &s_cost[warp][lane * 8];
  int32_t* my_cost32 = reinterpret_cast<int32_t*>(&s_cost[0][0]) + warp * 256 + lane * 8;
  if (MODE != kEval && C.cost32) {
#pragma unroll
    for (int q = 0; q < 8; ++q) my_cost32[q] = 0;
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) my_cost[q] = 0;
  }
  float fe[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) fe[q] = 0.f;
  pdl_wait();  // chain state from here on
  uint32_t t = 0;
  if (SAMPLE) t = step_index(tdev, t_rel);

  // the clause loop; UNI (all 8 chains of every lane of the warp share one
  // temperature, the common case) drops the per-chain temperature unpacking
  // from every clause. One-chunk records (ONE) are 4 words long.
  auto clause_loop = [&](auto uni_tag) {
    constexpr bool UNI = decltype(uni_tag)::value;
    // ONE: a clause's literals, length and group come from its 16-byte clause
    // record, loaded one iteration ahead (the state loads then wait on nothing)
    int4 nxt = make_int4(0, 0, 0, 0);
    if constexpr (ONE)
      if (c_begin + warp < c_end) nxt = __ldg(F.cl4 + c_begin + warp);
    for (int c = c_begin + warp; c < c_end; c += 8) {
      int len, grp_one = 0;
      // byte q of lo0|lo1 (chains 0..3 | 4..7): bits 0..7 of chain q's truth
      // pattern; of hi0|hi1: bits 8..15
      uint32_t lo0 = 0, lo1 = 0, hi0 = 0, hi1 = 0;
      if constexpr (ONE) {
        const int4 cur = nxt;
        if (c + 8 < c_end) nxt = __ldg(F.cl4 + c + 8);
        len = cur.w & 3;
        grp_one = cur.w >> 8;
        const int32_t lv[3] = {cur.x, cur.y, cur.z};
        uint2 x8[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
          x8[k] = k < len ? __ldg(reinterpret_cast<const uint2*>(xt + (size_t)lv[k] * Bp + b0))
                          : make_uint2(0u, 0u);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const uint32_t flip = ((cur.w >> (2 + k)) & 1) ? 0x01010101u : 0u;
          lo0 |= (x8[k].x ^ flip) << k;
          lo1 |= (x8[k].y ^ flip) << k;
        }
      } else {
        const int o = __ldg(F.cl_off + c);
        len = __ldg(F.cl_off + c + 1) - o;
        if (len <= 4) {
          // short clause: all literal and state loads in flight together
          int32_t lv[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) lv[k] = k < len ? __ldg(F.lit_var + o + k) : 0;
          uint2 x8[4];
#pragma unroll
          for (int k = 0; k < 4; ++k)
            x8[k] = k < len ? __ldg(reinterpret_cast<const uint2*>(
                                  xt + (size_t)(lv[k] & 0x7FFFFFFF) * Bp + b0))
                            : make_uint2(0u, 0u);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t flip = (k < len && lv[k] < 0) ? 0x01010101u : 0u;
            lo0 |= (x8[k].x ^ flip) << k;
            lo1 |= (x8[k].y ^ flip) << k;
          }
        } else {
          for (int k = 0; k < len; ++k) {
            const int32_t lv = __ldg(F.lit_var + o + k);
            const uint2 x8 =
                __ldg(reinterpret_cast<const uint2*>(xt + (size_t)(lv & 0x7FFFFFFF) * Bp + b0));
            const uint32_t flip = lv < 0 ? 0x01010101u : 0u;
            if (k < 8) {
              lo0 |= (x8.x ^ flip) << k;
              lo1 |= (x8.y ^ flip) << k;
            } else {
              hi0 |= (x8.x ^ flip) << (k - 8);
              hi1 |= (x8.y ^ flip) << (k - 8);
            }
          }
        }
      }
      int p[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if constexpr (ONE) {
          // byte q of the low word, zero-extended (selector 4: byte 0 of 0)
          p[q] = (int)__byte_perm(lo0, 0u, 0x4440u | q);
          p[q + 4] = (int)__byte_perm(lo1, 0u, 0x4440u | q);
        } else {
          // result byte 0 = byte q of the low word, byte 1 = byte q of the high word
          p[q] = (int)(__byte_perm(lo0, hi0, ((4u + q) << 4) | q) & 0xFFFFu);
          p[q + 4] = (int)(__byte_perm(lo1, hi1, ((4u + q) << 4) | q) & 0xFFFFu);
        }
      }
      // unsatisfied clauses are rare once chains settle: touch the cost rows
      // only when one of the 8 chains has p == 0
      uint32_t unsat = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) unsat |= (uint32_t)(p[q] == 0) << q;
      if (unsat) {
        const int64_t wc = __ldg(F.cl_w + c);
        if (MODE != kEval && C.cost32) {
          // each entry has one owner: the atomic is a one-instruction add
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if ((unsat >> q) & 1u) atomicAdd(my_cost32 + q, (int)wc);
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if ((unsat >> q) & 1u) my_cost[q] += wc;
        }
      }
      if (!FE || len == 0) continue;

      const int grp = ONE ? grp_one : __ldg(F.cl_grp + c);
      const GroupMeta gm = meta[grp];
      int row[8];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        row[q] = ((UNI ? e0 : (int)((epack >> (6 * q)) & 63u)) << len) + p[q];
      if constexpr (!SAMPLE) {
#pragma unroll
        for (int q = 0; q < 8; ++q) fe[q] += __uint_as_float(rec[gm.rec_off + row[q] * (ONE ? 4 : gm.stride)]);
      } else {
        // free energy (record word 0) and hidden draws from the records
        const uint4* tab = reinterpret_cast<const uint4*>(rec + gm.rec_off);
        int row4[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) row4[q] = ONE ? row[q] : row[q] * (gm.stride >> 2);
        uint32_t hp[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) hp[q] = 0;
        const uint32_t octet = (uint32_t)(g8 + C.g8_off);
        const int chunks = ONE ? 1 : gm.stride >> 2;
        const uint32_t lc = (uint32_t)(c - cl_base);  // clause index within its instance
        if (!gm.sat)
          hidden_draws<false, ONE>(tab, row4, chunks, gm.nh, lc, octet, t, phase_h, C.keys, hp, fe);
        else
          hidden_draws<true, ONE>(tab, row4, chunks, gm.nh, lc, octet, t, phase_h, C.keys, hp, fe);
        HT* H = static_cast<HT*>(C.H) + (size_t)c * Bp + b0;
        if (sizeof(HT) == 1) {
          uint64_t v = 0;
#pragma unroll
          for (int q = 0; q < 8; ++q) v |= (uint64_t)hp[q] << (8 * q);
          *reinterpret_cast<uint64_t*>(H) = v;
        } else {
          uint4 v;
          v.x = hp[0] | (hp[1] << 16);
          v.y = hp[2] | (hp[3] << 16);
          v.z = hp[4] | (hp[5] << 16);
          v.w = hp[6] | (hp[7] << 16);
          *reinterpret_cast<uint4*>(H) = v;
        }
      }
    }
  };
  if constexpr (ONE) {
    if (warp_uni)
      clause_loop(std::true_type{});
    else
      clause_loop(std::false_type{});
  } else {
    clause_loop(std::false_type{});
  }

  // per-block partial sums, then the block that arrives last among its
  // instance's blocks for this tile of 256 chains reduces their partials in
  // block order and keeps improvements
  if (FE) {
#pragma unroll
    for (int q = 0; q < 8; ++q) s_fe[warp][lane * 8 + q] = fe[q];
  }
  __syncthreads();
  const int tid = threadIdx.x;
  int64_t tc = 0;
  float tf = 0.f;
  const bool c32 = MODE != kEval && C.cost32;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    tc += c32 ? (int64_t)reinterpret_cast<const int32_t*>(&s_cost[0][0])[w * 256 + tid]
              : s_cost[w][tid];
    if (FE) tf += s_fe[w][tid];
  }
  const size_t out = (size_t)blockIdx.y * Bp + (size_t)blockIdx.x * 256 + tid;
  cost_part[out] = tc;
  if (FE) fe_part[out] = tf;
  __threadfence();
  __syncthreads();
  const int k0 = __ldg(P.inst_blk + inst), k1 = __ldg(P.inst_blk + inst + 1);
  int32_t* ticket = tickets + inst * gridDim.x + blockIdx.x;
  if (tid == 0) s_last = atomicAdd(ticket, 1) == k1 - k0 - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int b = blockIdx.x * 256 + tid;
  int64_t csum = 0;
  float fsum = 0.f;
  for (int k = k0; k < k1; ++k) {
    csum += __ldcg(cost_part + (size_t)k * Bp + b);
    if (FE) fsum += __ldcg(fe_part + (size_t)k * Bp + b);
  }
  if (MODE == kEval) {
    if (b < B) eval_out[(size_t)inst * B + b] = csum;
  } else {
    const size_t ib = (size_t)inst * Bp + b;
    C.cost[ib] = csum;
    C.fe[ib] = fsum;
    const bool imp = csum < C.best[ib];
    if (imp) C.best[ib] = csum;
    C.improved[ib] = imp ? 1 : 0;
  }
  if (tid == 0) *ticket = 0;
}

// ---------------------------------------------------------------------------
// Step gather for formulas whose clauses all have at most 3 literals (one
// 16-byte record per truth pattern) when every octet of chains has a single
// temperature: the same results as k_gather<kStep, true, uint8_t, true> with
// fewer instructions per clause and 8 chains.
//  - Philox4x32-10 rounds 0..2: unit h of chain octet o draws from counter
//    (clause, o | h << 24, t, phase). Round 0's product of word z (= t) is
//    the same for every unit and clause; round 1's product of word x depends
//    only on (o, h, t), so each thread computes it once; round 0's product of
//    word x, round 1's of word z and round 2's of word x depend only on the
//    clause, so the 3 units share them. A unit's own work starts with round
//    2's product of word z; the result is the Philox block, bit for bit.
//  - The truth patterns of 8 chains are two words of 4 bytes built by adds
//    (literal k contributes 2^k), the literal signs applied by one XOR with
//    the clause's flip mask.
//  - One SWAR test finds whether some chain leaves the clause unsatisfied.
//  - The records of each (group, temperature) form a 256-byte-aligned block,
//    so a chain's record address is one byte permute of 16 x its pattern
//    into the block's address.
//  - Each draw is a compare and a predicated OR into the hidden pattern word
//    (even chains move their draw into the high half first; groups with a
//    saturated unit, P = 65536 stored as 0xFFFF0001, also clear the low half
//    of odd chains' words).
//  - The weighted unsatisfied costs stay in registers: each chain adds the
//    clause weight times its 0/1 "no true literal" byte, without branches.
//  - Latency: the state bytes and weight of the next clause are loaded while
//    the current one is sampled, and each block first asks the L2 for its
//    slice of the chain tile's state rows and for its clause records and
//    weights (bulk prefetches), so the loop rarely waits on DRAM after the
//    previous round's writes. 2 blocks of 256 threads per SM (no spills;
//    measured faster than 3 or 4 blocks with spills, and than two clauses per
//    loop trip).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

__device__ __forceinline__ uint4 lds128(uint32_t addr) {
  uint4 v;
  asm("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
  return v;
}

// acc |= BIT when x < w (unsigned): one compare and one predicated OR
template <uint32_t BIT>
__device__ __forceinline__ void or_if_below(uint32_t& acc, uint32_t x, uint32_t w) {
  asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
      : "+r"(acc)
      : "r"(x), "r"(w), "n"(BIT));
}

// Asks the L2 to fetch `bytes` (a multiple of 16) from a 16-byte aligned
// global address (a bulk prefetch: no data returns to the thread).
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// A load of chain state: through the read-only path when the state cannot
// change during the launch, else from the L2 (CG: a persistent launch whose
// other phase writes it; read-only cache lines could be stale there).
template <bool CG, typename V>
__device__ __forceinline__ V ld_state(const V* p) {
  if constexpr (CG)
    return __ldcg(p);
  else
    return __ldg(p);
}

// The 8 state bytes of the thread's chains for each literal of clause record
// r (zero for absent literals; ALL3: every clause has 3 literals).
template <bool ALL3, bool CG>
__device__ __forceinline__ void load_clause_state(const uint8_t* xtb, int Bp, const int4& r,
                                                  uint2& xa, uint2& xb, uint2& xc) {
  const int len = ALL3 ? 3 : r.w & 3;
  xa = len > 0 ? ld_state<CG>(reinterpret_cast<const uint2*>(xtb + (size_t)r.x * Bp)) : make_uint2(0u, 0u);
  xb = len > 1 ? ld_state<CG>(reinterpret_cast<const uint2*>(xtb + (size_t)r.y * Bp)) : make_uint2(0u, 0u);
  xc = len > 2 ? ld_state<CG>(reinterpret_cast<const uint2*>(xtb + (size_t)r.z * Bp)) : make_uint2(0u, 0u);
}

// Unit H's draw for chain Q of the octet against threshold word w: bit
// 8 (Q & 3) + H of hw.
template <bool SAT, int Q, int H>
__device__ __forceinline__ void unit_draw(const uint4 (&R)[3], uint32_t w, uint32_t& hw) {
  const uint32_t word = word_of(R[H], Q >> 1);
  const uint32_t x = (Q & 1) ? (SAT ? (word & 0xFFFF0000u) : word) : (word << 16);
  or_if_below<(1u << (8 * (Q & 3) + H))>(hw, x, w);
}

// Chain Q of the octet: its record (free energy, thresholds of units 0..2)
// and its three draws.
template <bool SAT, int Q>
__device__ __forceinline__ void chain_draws(uint32_t addr_bytes, uint32_t rb, const uint4 (&R)[3],
                                            float& fe, uint32_t& hw) {
  const uint4 r = lds128(__byte_perm(addr_bytes, rb, 0x7650u | (Q & 3)));
  fe += __uint_as_float(r.x);
  unit_draw<SAT, Q, 0>(R, r.y, hw);
  unit_draw<SAT, Q, 1>(R, r.z, hw);
  unit_draw<SAT, Q, 2>(R, r.w, hw);
}

template <bool SAT>
__device__ __forceinline__ void octet_draws(uint32_t a_lo, uint32_t a_hi, uint32_t rb,
                                            const uint4 (&R)[3], float (&fe)[8], uint32_t& h_lo,
                                            uint32_t& h_hi) {
  chain_draws<SAT, 0>(a_lo, rb, R, fe[0], h_lo);
  chain_draws<SAT, 1>(a_lo, rb, R, fe[1], h_lo);
  chain_draws<SAT, 2>(a_lo, rb, R, fe[2], h_lo);
  chain_draws<SAT, 3>(a_lo, rb, R, fe[3], h_lo);
  chain_draws<SAT, 4>(a_hi, rb, R, fe[4], h_hi);
  chain_draws<SAT, 5>(a_hi, rb, R, fe[5], h_hi);
  chain_draws<SAT, 6>(a_hi, rb, R, fe[6], h_hi);
  chain_draws<SAT, 7>(a_hi, rb, R, fe[7], h_hi);
}

// PLAIN3: every clause has exactly 3 literals and no group has a saturated
// hidden unit (T.plain3). COST16: a warp's clauses of its block weigh less
// than 2^16 in total (C.cost16), so chains 2j and 2j + 1 keep their costs in
// the low and high half of one register.
// One block of the gather: chain tile bx of gx, clause block by of gy.
// PERSIST: a block of the persistent round (k_round_persistent), which has
// staged the record blocks already, orders its phases by grid barriers
// instead of programmatic dependent launch, and reads the chain state from
// the L2.
template <bool PLAIN3, bool COST16, bool PERSIST>
__device__ __forceinline__ void gather3_block(const DevFormula& F, const DevTables& T,
                                              const DevChains& C, const GatherPlan& P,
                                              const uint32_t* tdev, uint32_t t_rel,
                                              int64_t* cost_part, float* fe_part,
                                              int32_t* tickets, uint32_t vbx, uint32_t vby,
                                              uint32_t vgx, uint32_t vgy) {
  // the launch's own block and grid indices unless the block is virtual
#define G3_BX (PERSIST ? vbx : blockIdx.x)
#define G3_BY (PERSIST ? vby : blockIdx.y)
#define G3_GX (PERSIST ? vgx : gridDim.x)
#define G3_GY (PERSIST ? vgy : gridDim.y)
  if constexpr (!PERSIST) pdl_release();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int64_t s_cost[8][256];
  __shared__ float s_fe[8][256];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g8 = G3_BX * 32 + lane, b0 = g8 * 8;
  const int Bp = C.Bp;
  const int4 bd = __ldg(P.blk + G3_BY);
  const int inst = bd.x, c_begin = bd.y, c_end = bd.z, cl_base = bd.w;
  // the record blocks, staged at a 256-byte boundary of the dynamic shared memory
  const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t tab = (s0 + 255u) & ~255u;
  if constexpr (!PERSIST) {
    stage(smem + (tab - s0), T.rec3, T.rec3_words * 4);
    __syncthreads();
  }
  const int E = T.n_temps;
  const int e0 = temp_of(C.g8_off * 8 + b0, E, C.B_total, C.inv_B_total);
  const uint32_t tab_e = tab + (uint32_t)e0 * 256u;  // group 0 at the thread's temperature
  const uint32_t gstride = (uint32_t)E * 256u;       // from one group to the next
  // the weighted unsatisfied cost of the thread's 8 chains in registers:
  // the host runs this kernel only when every clause block's weight sum is
  // below 2^31 (C.cost32); with COST16, cost[j] packs chains 2j and 2j + 1
  int32_t cost[8];
  float fe[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    cost[q] = 0;
    fe[q] = 0.f;
  }
  if constexpr (!PERSIST) pdl_wait();  // chain state from here on
  // bulk L2 prefetches: the blocks of a chain tile split its n state rows
  // (256 bytes each) among themselves; each block fetches its own clause
  // records and weights
  for (int r = G3_BY + (int)G3_GY * threadIdx.x; r < F.n; r += (int)G3_GY * 256)
    l2_prefetch(C.xt + (size_t)r * Bp + G3_BX * 256, 256);
  if (threadIdx.x == 0 && c_end > c_begin) {
    l2_prefetch(F.cl4 + c_begin, (uint32_t)(c_end - c_begin) * 16u);
    const uintptr_t w0 = reinterpret_cast<uintptr_t>(F.cl_w + c_begin) & ~(uintptr_t)15;
    const uintptr_t w1 = reinterpret_cast<uintptr_t>(F.cl_w + c_end) & ~(uintptr_t)15;
    if (w1 > w0) l2_prefetch(reinterpret_cast<const void*>(w0), (uint32_t)(w1 - w0));
  }
  const uint32_t t = step_index(tdev, t_rel);
  const RoundKeys& K = C.keys;
  const uint32_t octet = (uint32_t)(g8 + C.g8_off);
  const uint32_t phase = kPhaseHidden | ((uint32_t)inst << 8);
  // round 0, word z = t: common to every unit and clause
  const uint64_t pt = (uint64_t)kPhiloxM1 * t;
  const uint32_t u1 = (uint32_t)(pt >> 32) ^ K.k0[0];
  const uint32_t u2 = (uint32_t)pt;
  // round 1, word x = round 0's (octet | h << 24) ^ u1: per thread and unit
  uint32_t th[3], sh[3];
#pragma unroll
  for (int h = 0; h < 3; ++h) {
    const uint64_t p = (uint64_t)kPhiloxM0 * ((octet | ((uint32_t)h << 24)) ^ u1);
    th[h] = (uint32_t)(p >> 32) ^ K.k1[1];
    sh[h] = (uint32_t)p;
  }
  const uint8_t* xtb = C.xt + b0;
  uint8_t* hb = static_cast<uint8_t*>(C.H) + b0;

  // software pipeline: the state bytes of the next clause and the record of
  // the one after it are loaded while the current clause is sampled
  const int c0 = c_begin + warp;
  int4 rec_n = make_int4(0, 0, 0, 0);
  if (c0 < c_end) rec_n = __ldg(F.cl4 + c0);
  uint2 xa, xb, xc;
  uint32_t info = (uint32_t)rec_n.w;
  int32_t wc = 0;
  if (c0 < c_end) wc = (int32_t)__ldg(F.cl_w + c0);
  load_clause_state<PLAIN3, PERSIST>(xtb, Bp, rec_n, xa, xb, xc);
  if (c0 + 8 < c_end) rec_n = __ldg(F.cl4 + c0 + 8);
  for (int c = c0; c < c_end; c += 8) {
    uint2 na = make_uint2(0u, 0u), nb = na, nc = na;
    const uint32_t ninfo = (uint32_t)rec_n.w;
    int32_t nwc = 0;
    if (c + 8 < c_end) {
      load_clause_state<PLAIN3, PERSIST>(xtb, Bp, rec_n, na, nb, nc);
      nwc = (int32_t)__ldg(F.cl_w + c + 8);
    }
    if (c + 16 < c_end) rec_n = __ldg(F.cl4 + c + 16);
    const int len = info & 3;
    // byte q: chain q's truth pattern (chains 0..3 | 4..7)
    const uint32_t flip = ((info >> 2) & 7u) * 0x01010101u;
    const uint32_t lo = (xa.x + 2u * xb.x + 4u * xc.x) ^ flip;
    const uint32_t hi = (xa.y + 2u * xb.y + 4u * xc.y) ^ flip;
    const uint32_t grp = info >> 8;
    const int32_t w_cur = wc;
    xa = na;
    xb = nb;
    xc = nc;
    info = ninfo;
    wc = nwc;
    // byte q is 1 when chain q has no true literal (pattern 0: 0x7F + p sets
    // bit 7 for every p in 1..7 and never carries), else 0; each chain adds
    // the clause weight times its byte, without branches
    const uint32_t u_lo = (~(lo + 0x7F7F7F7Fu) & 0x80808080u) >> 7;
    const uint32_t u_hi = (~(hi + 0x7F7F7F7Fu) & 0x80808080u) >> 7;
    if (COST16) {
      // bytes 2j, 2j + 1 -> 16-bit halves of one word
      cost[0] += (int32_t)(__byte_perm(u_lo, 0u, 0x4140u) * (uint32_t)w_cur);
      cost[1] += (int32_t)(__byte_perm(u_lo, 0u, 0x4342u) * (uint32_t)w_cur);
      cost[2] += (int32_t)(__byte_perm(u_hi, 0u, 0x4140u) * (uint32_t)w_cur);
      cost[3] += (int32_t)(__byte_perm(u_hi, 0u, 0x4342u) * (uint32_t)w_cur);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        cost[q] += (int32_t)__byte_perm(u_lo, 0u, 0x4440u | q) * w_cur;
        cost[q + 4] += (int32_t)__byte_perm(u_hi, 0u, 0x4440u | q) * w_cur;
      }
    }
    if (!PLAIN3 && len == 0) continue;  // an empty clause has no clause RBM

    const uint32_t rb = tab_e + grp * gstride;
    const bool sat = !PLAIN3 && (lds32(rb + 128u) & 0x100u) != 0;
    // Philox rounds 0..2: the clause's share, then each unit's
    const uint32_t cl = (uint32_t)(c - cl_base);
    const uint64_t p0 = (uint64_t)kPhiloxM0 * cl;
    const uint32_t c1 = (uint32_t)(p0 >> 32) ^ phase ^ K.k1[0];
    const uint32_t c2 = (uint32_t)p0;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c1;
    const uint32_t c3 = (uint32_t)(p1 >> 32) ^ u2 ^ K.k0[1];
    const uint32_t c4 = (uint32_t)p1;
    const uint64_t p2 = (uint64_t)kPhiloxM0 * c3;
    const uint32_t c5 = (uint32_t)(p2 >> 32) ^ K.k1[2];
    const uint32_t c6 = (uint32_t)p2;
    uint4 R[3];
#pragma unroll
    for (int h = 0; h < 3; ++h) {
      const uint64_t pz = (uint64_t)kPhiloxM1 * (th[h] ^ c2);
      R[h] = philox_rounds<3>(
          make_uint4((uint32_t)(pz >> 32) ^ c4 ^ K.k0[2], (uint32_t)pz, c5 ^ sh[h], c6), K);
    }
    uint32_t h_lo = 0, h_hi = 0;
    if (!sat)
      octet_draws<false>(lo << 4, hi << 4, rb, R, fe, h_lo, h_hi);
    else
      octet_draws<true>(lo << 4, hi << 4, rb, R, fe, h_lo, h_hi);
    *reinterpret_cast<uint2*>(hb + (size_t)c * Bp) = make_uint2(h_lo, h_hi);
  }

  // per-block partial sums; the block that arrives last among its instance's
  // blocks for this tile of 256 chains reduces them in block order and keeps
  // improvements (as k_gather)
  if (COST16) {
#pragma unroll
    for (int j = 3; j >= 0; --j) {
      cost[2 * j + 1] = (int32_t)((uint32_t)cost[j] >> 16);
      cost[2 * j] = cost[j] & 0xFFFF;
    }
  }
  int32_t* my_cost32 = reinterpret_cast<int32_t*>(&s_cost[0][0]) + warp * 256 + lane * 8;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    my_cost32[q] = cost[q];
    s_fe[warp][lane * 8 + q] = fe[q];
  }
  __syncthreads();
  const int tid = threadIdx.x;
  int64_t tc = 0;
  float tf = 0.f;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    tc += reinterpret_cast<const int32_t*>(&s_cost[0][0])[w * 256 + tid];
    tf += s_fe[w][tid];
  }
  const size_t out = (size_t)G3_BY * Bp + (size_t)G3_BX * 256 + tid;
  cost_part[out] = tc;
  fe_part[out] = tf;
  __threadfence();
  __syncthreads();
  const int k0 = __ldg(P.inst_blk + inst), k1 = __ldg(P.inst_blk + inst + 1);
  int32_t* ticket = tickets + inst * G3_GX + G3_BX;
  if (tid == 0) s_last = atomicAdd(ticket, 1) == k1 - k0 - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int b = G3_BX * 256 + tid;
  int64_t csum = 0;
  float fsum = 0.f;
  for (int k = k0; k < k1; ++k) {
    csum += __ldcg(cost_part + (size_t)k * Bp + b);
    fsum += __ldcg(fe_part + (size_t)k * Bp + b);
  }
  const size_t ib = (size_t)inst * Bp + b;
  C.cost[ib] = csum;
  C.fe[ib] = fsum;
  const bool imp = csum < (PERSIST ? __ldcg(C.best + ib) : C.best[ib]);
  if (imp) C.best[ib] = csum;
  C.improved[ib] = imp ? 1 : 0;
  if (tid == 0) *ticket = 0;
#undef G3_BX
#undef G3_BY
#undef G3_GX
#undef G3_GY
}

template <bool PLAIN3, bool COST16>
__global__ void __launch_bounds__(256, 2) k_gather3(DevFormula F, DevTables T, DevChains C,
                                                    GatherPlan P, const uint32_t* tdev,
                                                    uint32_t t_rel, int64_t* cost_part,
                                                    float* fe_part, int32_t* tickets) {
  gather3_block<PLAIN3, COST16, false>(F, T, C, P, tdev, t_rel, cost_part, fe_part, tickets,
                                       blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}

// CG: the improved flags come from the L2 (a persistent launch: another
// block wrote them in this launch)
template <bool CG = false>
__device__ __forceinline__ void keep_improved(const DevChains& C, int inst, size_t o, int b0,
                                              uint64_t xold) {
  const unsigned long long* fl =
      reinterpret_cast<const unsigned long long*>(C.improved + (size_t)inst * C.Bp + b0);
  const uint64_t imp = CG ? __ldcg(fl) : *fl;
  if (imp) {
    const uint64_t mask = imp * 0xFFull;  // 0x01 flags -> 0xFF byte masks
    uint64_t* bx = reinterpret_cast<uint64_t*>(C.best_xt + o);
    *bx = (*bx & ~mask) | (xold & mask);
  }
}

// The end of a visible update for one variable and 8 chains given their
// integer logits z (units 2^-Q): best-so-far copy of improved chains, the
// visible draws x ~ Bernoulli(P[z]) (Eq. 3) and nu (Sec. 4.4).
template <bool CG = false>
__device__ __forceinline__ void visible_tail(const DevTables& T, const DevChains& C,
                                             const uint32_t* pv, float alpha, uint32_t t,
                                             int2 vi, int g8, size_t o, int b0, uint64_t xold,
                                             float4 n0, float4 n1, const int (&z)[8]) {
  keep_improved<CG>(C, vi.x, o, b0, xold);
  const uint4 r =
      philox4x32_10(make_uint4((uint32_t)vi.y, (uint32_t)(g8 + C.g8_off), t,
                               kPhaseVisible | ((uint32_t)vi.x << 8)),
                    C.keys);
  float nu[8] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
  // nu in FP32 with a fixed operation sequence (one rounding per step):
  // var = fl(P (65536 - P)) 2^-32, nu = fma(1 - alpha, nu, fl(alpha var))
  const float keep = __fsub_rn(1.0f, alpha);
  uint64_t xnew = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int qq = max(-T.qmax, min(T.qmax, z[q]));
    const uint32_t P = pv[qq + T.qmax];
    // rho (1 - rho) with rho = P / 65536: P (65536 - P) <= 2^30, scaled by 2^-32
    const float var = __fmul_rn(__uint2float_rn(P * (65536u - P)), 2.3283064365386963e-10f);
    nu[q] = __fmaf_rn(keep, nu[q], __fmul_rn(alpha, var));
    xnew |= (uint64_t)(lane16(r, q) < P) << (8 * q);
  }
  float4* nu4 = reinterpret_cast<float4*>(C.nu + o);
  nu4[0] = make_float4(nu[0], nu[1], nu[2], nu[3]);
  nu4[1] = make_float4(nu[4], nu[5], nu[6], nu[7]);
  *reinterpret_cast<uint64_t*>(C.xt + o) = xnew;
}

// BATCH: incidences whose pattern loads are in flight together (a divisor
// of 32; the launch picks it, measured by the block tuner). Batch 8 runs 3
// blocks per SM (its loads need more than 64 registers), the others 4.
// One block of the visible update: chain tile `tile`, variable group
// `vgroup` (8 variables, one per warp). With SM the tables are staged at
// byte vis_off of the dynamic shared memory. PERSIST: a block of the
// persistent round (k_round_persistent), which has staged the tables already,
// orders its phases by grid barriers and reads the hidden patterns from the
// L2.
template <bool SM, typename HT, int BATCH, bool PERSIST>
__device__ __forceinline__ void visible_block(const DevFormula& F, const DevTables& T,
                                              const DevChains& C, float alpha,
                                              const uint32_t* tdev, uint32_t t_rel, int tile,
                                              int vgroup, int vis_off) {
  static_assert(32 % BATCH == 0, "incidence windows hold whole batches");
  if constexpr (!PERSIST) pdl_release();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int4 s_inc[8][32];  // per warp: a window of its variable's incidences
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g8 = tile * 32 + lane, b0 = g8 * 8;
  const int16_t* gq = T.gq;
  const uint32_t* pv = T.pv;
  if (SM) {
    const int gb = align16(T.gq_len * 4);  // both halves
    if constexpr (!PERSIST) {
      stage(smem + vis_off, T.gq, gb);
      stage(smem + vis_off + gb, T.pv, align16(T.pv_len * 4));
      __syncthreads();
    }
    gq = reinterpret_cast<const int16_t*>(smem + vis_off);
    pv = reinterpret_cast<const uint32_t*>(smem + vis_off + gb);
  }
  // variables in descending degree: a block's 8 warps carry similar work
  const int slot = vgroup * 8 + warp;
  if (slot >= F.n) return;
  const int i = F.var_order ? __ldg(F.var_order + slot) : slot;
  const int2 vi = var_instance(F, i);
  if constexpr (!PERSIST) pdl_wait();  // chain state from here on
  const uint32_t t = step_index(tdev, t_rel);
  const int gb0 = C.g8_off * 8 + b0;  // global chain index
  const int e0 = temp_of(gb0, T.n_temps, C.B_total, C.inv_B_total);
  const bool e_uni = e0 == temp_of(gb0 + 7, T.n_temps, C.B_total, C.inv_B_total);
  int z[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) z[q] = 0;
  const HT* H = static_cast<const HT*>(C.H);
  using HV = typename std::conditional<sizeof(HT) == 1, unsigned long long, uint4>::type;
  // this thread's state loads go out first; they are used after the sums
  const size_t o = (size_t)i * C.Bp + b0;
  const uint64_t xold = *reinterpret_cast<const uint64_t*>(C.xt + o);
  float4* nu4 = reinterpret_cast<float4*>(C.nu + o);
  const float4 n0 = nu4[0], n1 = nu4[1];
  const int j_begin = __ldg(F.var_off + i), j_end = __ldg(F.var_off + i + 1);
  // z += sgn * 2^Q G[e][pattern][slot] over the variable's incidences
  // (clause inc.x, table base | sign inc.y, stride K inc.z, per-temperature
  // stride 2^L K inc.w); a negated literal's base lies in the table's negated
  // half, so the sum is plain adds. UNI: the 8 chains share temperature e0.
  auto sums = [&](auto uni) {
    constexpr bool UNI = decltype(uni)::value;
    int e[8];
    if constexpr (!UNI) {
#pragma unroll
      for (int q = 0; q < 8; ++q) e[q] = temp_of(gb0 + q, T.n_temps, C.B_total, C.inv_B_total);
    }
    // the variable's incidences pass through this warp's shared-memory slot
    // 32 at a time (one coalesced load); BATCH (a divisor of 32) per
    // pass, their pattern loads in flight together, the last pass predicated
    // (warp-uniform)
    for (int jj = j_begin; jj < j_end; jj += BATCH) {
      const int w = (jj - j_begin) & 31;
      if (w == 0) {
        __syncwarp();
        if (jj + lane < j_end) s_inc[warp][lane] = __ldg(F.var_inc + jj + lane);
        __syncwarp();
      }
      HV v[BATCH];
#pragma unroll
      for (int u = 0; u < BATCH; ++u)
        if (jj + u < j_end)
          v[u] = ld_state<PERSIST>(reinterpret_cast<const HV*>(H + (size_t)s_inc[warp][w + u].x * C.Bp + b0));
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        if (jj + u >= j_end) break;
        const int4 inc = s_inc[warp][w + u];
        const int base = inc.y & 0x7FFFFFFF;
        uint32_t hp[8];
        if constexpr (sizeof(HT) == 1) {
#pragma unroll
          for (int q = 0; q < 8; ++q) hp[q] = (uint32_t)(v[u] >> (8 * q)) & 0xFFu;
        } else {
          const uint32_t wv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
          for (int q = 0; q < 8; ++q) hp[q] = (wv[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
        }
        if constexpr (UNI) {
          if constexpr (SM) {
            // byte offsets into the staged table: one multiply-add per address
            const unsigned char* tb =
                reinterpret_cast<const unsigned char*>(gq + base + e0 * inc.w);
            const int k2 = 2 * inc.z;
#pragma unroll
            for (int q = 0; q < 8; ++q)
              z[q] += (int)*reinterpret_cast<const int16_t*>(tb + (int)hp[q] * k2);
          } else {
            const int bo = base + e0 * inc.w;
#pragma unroll
            for (int q = 0; q < 8; ++q) z[q] += (int)gq[bo + (int)hp[q] * inc.z];
          }
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            z[q] += (int)gq[base + e[q] * inc.w + (int)hp[q] * inc.z];
        }
      }
    }
  };
  // one form per warp: its lanes share the incidence window
  if (__all_sync(0xFFFFFFFFu, e_uni))
    sums(std::true_type{});
  else
    sums(std::false_type{});
  visible_tail<PERSIST>(T, C, pv, alpha, t, vi, g8, o, b0, xold, n0, n1, z);
}

template <bool SM, typename HT, int BATCH>
__global__ void __launch_bounds__(256, BATCH >= 8 ? 3 : 4) k_visible(DevFormula F, DevTables T, DevChains C,
                                                 float alpha, const uint32_t* tdev,
                                                 uint32_t t_rel, int v0, int tile_major) {
  // tile_major: blocks walk every variable group of one chain tile before the
  // next tile (x = variable group, y = chain tile from v0), so a tile's hidden
  // patterns, m x 256 entries, stay in the L2 while its variables pull them
  // (taken when all of them would not fit). Otherwise x = chain tile, y =
  // variable group from v0.
  const int tile = tile_major ? v0 + (int)blockIdx.y : (int)blockIdx.x;
  const int vgroup = tile_major ? (int)blockIdx.x : v0 + (int)blockIdx.y;
  visible_block<SM, HT, BATCH, false>(F, T, C, alpha, tdev, t_rel, tile, vgroup, 0);
}

// ---------------------------------------------------------------------------
// Persistent round: `rounds` Gibbs rounds in one cooperative launch. Every
// block walks the virtual blocks of the gather (chain tile fastest, as the
// gather's grid), meets the other blocks at a grid barrier, walks the
// virtual blocks of the visible update (the visible launch's order), and
// meets them again before the next round. The blocks are the same as the
// two-launch round's, so states, costs, draws and free energies are the
// same bit for bit. Clauses of at most 3 literals on single-temperature
// octets, byte hidden patterns, tables in shared memory (the k_gather3 and
// k_visible<true, uint8_t, 4> case); the host checks this.
// ---------------------------------------------------------------------------
constexpr long long kBarrierWaitCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr int kErrGridBarrier = 16;                    // device error code of a barrier timeout

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier of a cooperative launch (every block resident): bar[0] counts
// arrivals over the launch (zeroed before it), bar[1] is set when some block
// gave up waiting. A wait gives up after about 2 s, records kErrGridBarrier
// in *err and sets bar[1]; every block then leaves at its next barrier, so
// the launch ends and the host reads the code. Returns false when the block
// must leave.
__device__ __forceinline__ bool grid_barrier(uint32_t* bar, uint32_t& target, int* err) {
  __shared__ int s_go;
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    int go = 1;
    const long long t0 = clock64();
    while (ld_acquire_gpu(bar) < target) {
      if (ld_acquire_gpu(bar + 1) != 0u) {
        go = 0;
        break;
      }
      if (clock64() - t0 > kBarrierWaitCycles) {
        atomicCAS(err, 0, kErrGridBarrier);
        atomicExch(bar + 1, 1u);
        go = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_go = go;
  }
  __syncthreads();
  return s_go != 0;
}

template <bool PLAIN3, bool COST16>
__global__ void __launch_bounds__(256, 2)
    k_round_persistent(DevFormula F, DevTables T, DevChains C, GatherPlan P, uint32_t t0,
                       int rounds, float alpha, int tile_major, int vis_off, uint32_t* bar,
                       int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  // both kernels' tables, once: the gather's record blocks at the first
  // 256-byte boundary, the visible update's tables at vis_off
  const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t tab = (s0 + 255u) & ~255u;
  stage(smem + (tab - s0), T.rec3, T.rec3_words * 4);
  const int gb = align16(T.gq_len * 4);
  stage(smem + vis_off, T.gq, gb);
  stage(smem + vis_off + gb, T.pv, align16(T.pv_len * 4));
  __syncthreads();
  const uint32_t tiles = (uint32_t)(C.Bp / kChainTile);
  const uint32_t n_blk = (uint32_t)P.n_blk;
  const uint32_t groups = (uint32_t)((F.n + 7) / 8);
  const uint32_t n_gather = tiles * n_blk, n_visible = tiles * groups;
  uint32_t target = 0;
  for (int r = 0; r < rounds; ++r) {
    const uint32_t t = t0 + (uint32_t)r;
    for (uint32_t vb = blockIdx.x; vb < n_gather; vb += gridDim.x)
      gather3_block<PLAIN3, COST16, true>(F, T, C, P, nullptr, t, C.cost_part, C.fe_part,
                                          C.tickets, vb % tiles, vb / tiles, tiles, n_blk);
    if (!grid_barrier(bar, target, err)) return;
    for (uint32_t vb = blockIdx.x; vb < n_visible; vb += gridDim.x) {
      const int tile = (int)(tile_major ? vb / groups : vb % tiles);
      const int vgroup = (int)(tile_major ? vb % groups : vb / tiles);
      visible_block<true, uint8_t, 4, true>(F, T, C, alpha, nullptr, t, tile, vgroup, vis_off);
    }
    if (!grid_barrier(bar, target, err)) return;
  }
}

__global__ void __launch_bounds__(256) k_keep_copy(DevFormula F, DevChains C, int n, int vg0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b0 = (blockIdx.x * 32 + lane) * 8;
  const int i = (vg0 + blockIdx.y) * 8 + warp;
  if (i >= n) return;
  const size_t o = (size_t)i * C.Bp + b0;
  keep_improved(C, var_instance(F, i).x, o, b0, *reinterpret_cast<const uint64_t*>(C.xt + o));
}

__global__ void k_advance(uint32_t* tdev, uint32_t by) { *tdev += by; }
__global__ void k_set_u32(uint32_t* dst, uint32_t value) { *dst = value; }

// assign (B x n, chain-major, any nonzero = 1) -> xt (n x Bp, 0/1); chains
// B..Bp-1 read as all-false.
__global__ void k_transpose_in(const uint8_t* __restrict__ assign, int B, int n,
                               uint8_t* __restrict__ xt, int Bp) {
  __shared__ uint8_t tile[32][33];
  const int i0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
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

int gather_smem_bytes(const DevTables& T) {
  return align16(T.n_groups * (int)sizeof(GroupMeta)) + align16(T.rec_len * 4);
}

int visible_smem_bytes(const DevTables& T) {
  return align16(T.gq_len * 4) + align16(T.pv_len * 4);
}

constexpr int kSmemLimit = 160 * 1024;
constexpr int kMaxGridY = 65535;

// a launch that may overlap its predecessor's tail (see pdl_wait)
template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kern)(Params...), dim3 grid, int smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// dynamic shared memory of k_gather3: the record blocks plus the slack that
// moves them to a 256-byte boundary
int gather3_smem_bytes(const DevTables& T) { return T.rec3_words * 4 + 256; }

using Gather3Fn = void (*)(DevFormula, DevTables, DevChains, GatherPlan, const uint32_t*,
                           uint32_t, int64_t*, float*, int32_t*);

Gather3Fn gather3_kernel(const DevTables& T, const DevChains& C) {
  if (T.plain3) return C.cost16 ? k_gather3<true, true> : k_gather3<true, false>;
  return C.cost16 ? k_gather3<false, true> : k_gather3<false, false>;
}

// every octet of chains has one temperature: each temperature block starts
// at a multiple of 8 (block e starts at ceil(e B_total / E); local chain 0 is
// a multiple of 8 of the ensemble)
bool octets_single_temperature(const DevTables& T, const DevChains& C) {
  const long long Bt = C.B_total, E = T.n_temps;
  for (long long e = 1; e < E; ++e)
    if (((e * Bt + E - 1) / E) % 8 != 0) return false;
  return true;
}

template <int MODE, bool SM, typename HT>
cudaError_t gather_variant(dim3 grid, int smem, cudaStream_t st, const DevFormula& F,
                           const DevTables& T, const DevChains& C, const uint8_t* xt, int B,
                           int Bp, const GatherPlan& P, const uint32_t* tdev, uint32_t t_rel,
                           int64_t* cost_part, float* fe_part, int32_t* tickets,
                           int64_t* eval_out) {
  if constexpr (MODE == kStep && SM && sizeof(HT) == 1) {
    if (T.one_chunk && T.rec3 && F.cl4 && C.cost32 && octets_single_temperature(T, C)) {
      const int sm3 = gather3_smem_bytes(T);
      auto kern = gather3_kernel(T, C);
      const cudaError_t e = allow_dynamic_smem(kern, sm3);
      if (e != cudaSuccess) return e;
      return launch_pdl(kern, grid, sm3, st, F, T, C, P, tdev, t_rel, cost_part, fe_part,
                        tickets);
    }
  }
  // one-chunk records (L <= 3 everywhere): the sampling has no chunk loop
  auto kern = k_gather<MODE, SM, HT, false>;
  if constexpr (MODE == kStep && sizeof(HT) == 1)
    if (T.one_chunk) kern = k_gather<MODE, SM, HT, true>;
  {
    const cudaError_t e = allow_dynamic_smem(kern, smem);
    if (e != cudaSuccess) return e;
  }
  if constexpr (MODE == kStep)
    return launch_pdl(kern, grid, smem, st, F, T, C, xt, B, Bp, P, tdev, t_rel, cost_part,
                      fe_part, tickets, eval_out);
  kern<<<grid, 256, smem, st>>>(F, T, C, xt, B, Bp, P, tdev, t_rel, cost_part, fe_part, tickets,
                                eval_out);
  return cudaGetLastError();
}

template <bool SM, typename HT, bool ONE>
int gather_occupancy(int smem) {
  auto kern = k_gather<kStep, SM, HT, ONE>;
  if (allow_dynamic_smem(kern, smem) != cudaSuccess) return 1;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 256, smem) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

template <int MODE>
cudaError_t gather_mode(dim3 grid, cudaStream_t st, bool wide, const DevFormula& F,
                        const DevTables& T, const DevChains& C, const uint8_t* xt, int B, int Bp,
                        const GatherPlan& P, const uint32_t* tdev, uint32_t t_rel,
                        int64_t* cost_part, float* fe_part, int32_t* tickets, int64_t* eval_out) {
  const int sm = gather_smem_bytes(T);
  const bool use_sm = MODE != kEval && sm <= kSmemLimit;
  if (use_sm && !wide)
    return gather_variant<MODE, true, uint8_t>(grid, sm, st, F, T, C, xt, B, Bp, P, tdev, t_rel,
                                               cost_part, fe_part, tickets, eval_out);
  if (use_sm)
    return gather_variant<MODE, true, uint16_t>(grid, sm, st, F, T, C, xt, B, Bp, P, tdev, t_rel,
                                                cost_part, fe_part, tickets, eval_out);
  if (!wide)
    return gather_variant<MODE, false, uint8_t>(grid, 0, st, F, T, C, xt, B, Bp, P, tdev, t_rel,
                                                cost_part, fe_part, tickets, eval_out);
  return gather_variant<MODE, false, uint16_t>(grid, 0, st, F, T, C, xt, B, Bp, P, tdev, t_rel,
                                               cost_part, fe_part, tickets, eval_out);
}

template <bool SM, typename HT>
cudaError_t visible_variant(dim3 grid, int smem, cudaStream_t st, const DevFormula& F,
                            const DevTables& T, const DevChains& C, float alpha,
                            const uint32_t* tdev, uint32_t t_rel, int batch) {
  auto kern = batch >= 8 ? k_visible<SM, HT, 8> : batch <= 2 ? k_visible<SM, HT, 2>
                                                             : k_visible<SM, HT, 4>;
  {
    const cudaError_t e = allow_dynamic_smem(kern, smem);
    if (e != cudaSuccess) return e;
  }
  const int groups = (F.n + 7) / 8, tiles = (int)grid.x;
  // tile-major when the hidden patterns exceed half the L2
  static int l2 = -1;
  if (l2 < 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
      l2 = 0;
  }
  const int tm = (double)F.m * C.Bp * sizeof(HT) > 0.5 * (double)l2 ? 1 : 0;
  if (tm) {
    // x = variable groups, y = chain tiles (launches of at most kMaxGridY tiles)
    grid.x = (unsigned)groups;
    for (int t0 = 0; t0 < tiles; t0 += kMaxGridY) {
      grid.y = std::min(kMaxGridY, tiles - t0);
      const cudaError_t e = launch_pdl(kern, grid, smem, st, F, T, C, alpha, tdev, t_rel, t0, tm);
      if (e != cudaSuccess) return e;
    }
  } else {
    // x = chain tiles, y = variable groups (launches of at most kMaxGridY groups)
    for (int vg0 = 0; vg0 < groups; vg0 += kMaxGridY) {
      grid.y = std::min(kMaxGridY, groups - vg0);
      const cudaError_t e = launch_pdl(kern, grid, smem, st, F, T, C, alpha, tdev, t_rel, vg0, tm);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

}  // namespace

int clause_block_for(int m) {
  const int per = (m + 255) / 256;
  return per > kClauseBlock ? per : kClauseBlock;
}

int clause_blocks_for(int m) {
  const int cb = clause_block_for(m);
  const int nb = (m + cb - 1) / cb;
  return nb > 0 ? nb : 1;
}

// below this many clauses per block, the per-block table staging dominates
constexpr int kMinClauseBlock = 16;

int gather_clause_block(int m, int tiles, int slots) {
  int best = clause_block_for(m);
  if (m <= 0 || tiles <= 0 || slots <= 0) return best;
  auto fill = [&](int cb) {
    const long long items = (long long)tiles * ((m + cb - 1) / cb);
    const long long waves = (items + slots - 1) / slots;
    return (double)items / (double)(waves * slots);
  };
  double best_fill = fill(best);
  // fewest waves first: a later candidate must fill clearly better
  for (int waves = 1; waves <= 64; ++waves) {
    const long long y = (long long)waves * slots / tiles;
    if (y < 1) continue;
    const int cb = std::max((int)((m + y - 1) / y), kMinClauseBlock);
    const double f = fill(cb);
    if (f > best_fill + 0.01) {
      best_fill = f;
      best = cb;
    }
    if (cb == kMinClauseBlock) break;
  }
  return best;
}

// resident blocks per SM of the step gather that will run (the one-chunk
// variant when every record is one chunk)
int gather_blocks_per_sm(const DevTables& T, bool wide) {
  const int sm = gather_smem_bytes(T);
  const bool use_sm = sm <= kSmemLimit;
  const bool one = T.one_chunk && !wide;
  if (use_sm && one && T.rec3) {
    // k_gather3 runs whenever the chains' octets have single temperatures
    // (the variant with the most registers stands for all four)
    const int sm3 = gather3_smem_bytes(T);
    if (allow_dynamic_smem(k_gather3<false, false>, sm3) != cudaSuccess) return 1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gather3<false, false>, 256, sm3) !=
        cudaSuccess)
      return 1;
    return nb > 0 ? nb : 1;
  }
  if (use_sm && one) return gather_occupancy<true, uint8_t, true>(sm);
  if (!use_sm && one) return gather_occupancy<false, uint8_t, true>(0);
  if (use_sm && !wide) return gather_occupancy<true, uint8_t, false>(sm);
  if (use_sm) return gather_occupancy<true, uint16_t, false>(sm);
  if (!wide) return gather_occupancy<false, uint8_t, false>(0);
  return gather_occupancy<false, uint16_t, false>(0);
}

cudaError_t launch_init_sparse(const DevFormula& F, const DevChains& C, int n, cudaStream_t st) {
  const int groups = std::max((n + 7) / 8, 1);
  for (int vg0 = 0; vg0 < groups; vg0 += kMaxGridY) {
    dim3 grid(C.Bp / kChainTile, std::min(kMaxGridY, groups - vg0));
    k_init<<<grid, 256, 0, st>>>(F, C, n, vg0);
  }
  return cudaGetLastError();
}

cudaError_t launch_gather(GatherMode mode, const DevFormula& F, const DevTables& T,
                          const DevChains& C, const uint8_t* xt, int B, int Bp,
                          const GatherPlan& P, const uint32_t* tdev, uint32_t t_rel,
                          int64_t* cost_part, float* fe_part, int32_t* tickets,
                          int64_t* eval_out, bool wide, cudaStream_t st) {
  if (P.n_blk < 1 || P.n_blk > kMaxGridY) return cudaErrorInvalidValue;
  dim3 grid(Bp / kChainTile, P.n_blk);
  switch (mode) {
    case kStep:
      return gather_mode<kStep>(grid, st, wide, F, T, C, xt, B, Bp, P, tdev, t_rel, cost_part,
                                fe_part, tickets, eval_out);
    case kScore:
      return gather_mode<kScore>(grid, st, wide, F, T, C, xt, B, Bp, P, tdev, t_rel, cost_part,
                                 fe_part, tickets, eval_out);
    default:
      return gather_mode<kEval>(grid, st, wide, F, T, C, xt, B, Bp, P, tdev, t_rel, cost_part,
                                fe_part, tickets, eval_out);
  }
}

cudaError_t launch_visible(const DevFormula& F, const DevTables& T, const DevChains& C,
                           float alpha, const uint32_t* tdev, uint32_t t_rel, bool wide,
                           cudaStream_t st, int batch) {
  dim3 grid(C.Bp / kChainTile, (F.n + 7) / 8);
  const int sm = visible_smem_bytes(T);
  const bool use_sm = sm <= kSmemLimit;
  if (use_sm && !wide)
    return visible_variant<true, uint8_t>(grid, sm, st, F, T, C, alpha, tdev, t_rel, batch);
  if (use_sm) return visible_variant<true, uint16_t>(grid, sm, st, F, T, C, alpha, tdev, t_rel, batch);
  if (!wide) return visible_variant<false, uint8_t>(grid, 0, st, F, T, C, alpha, tdev, t_rel, batch);
  return visible_variant<false, uint16_t>(grid, 0, st, F, T, C, alpha, tdev, t_rel, batch);
}

bool persistent_round_supported(const DevTables& T, const DevChains& C, const DevFormula& F,
                                bool wide) {
  return !wide && T.one_chunk && T.rec3 && F.cl4 && C.cost32 && octets_single_temperature(T, C) &&
         gather_smem_bytes(T) <= kSmemLimit && visible_smem_bytes(T) <= kSmemLimit;
}

cudaError_t launch_round_persistent(const DevFormula& F, const DevTables& T, const DevChains& C,
                                    const GatherPlan& P, uint32_t t0, int rounds, float alpha,
                                    uint32_t* bar, int* err, cudaStream_t st) {
  if (rounds < 1 || rounds > kMaxPersistentRounds) return cudaErrorInvalidValue;
  auto kern = T.plain3 ? (C.cost16 ? k_round_persistent<true, true> : k_round_persistent<true, false>)
                       : (C.cost16 ? k_round_persistent<false, true> : k_round_persistent<false, false>);
  const int vis_off = align16(gather3_smem_bytes(T));
  const int smem = vis_off + visible_smem_bytes(T);
  cudaError_t e = allow_dynamic_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0, l2 = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // every block resident (cooperative launch); never more blocks than either
  // phase has virtual blocks
  const long long tiles = C.Bp / kChainTile;
  const long long work = std::max(tiles * P.n_blk, tiles * ((F.n + 7) / 8));
  const int grid = (int)std::min<long long>((long long)per_sm * sms, std::max(work, 1LL));
  // tile-major visible order when the hidden patterns exceed half the L2 (as
  // the two-launch round)
  const int tm = (double)F.m * C.Bp > 0.5 * (double)l2 ? 1 : 0;
  if ((e = cudaMemsetAsync(bar, 0, 2 * sizeof(uint32_t), st)) != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, F, T, C, P, t0, rounds, alpha, tm, vis_off, bar, err);
}

cudaError_t launch_keep_copy(const DevFormula& F, const DevChains& C, int n, cudaStream_t st) {
  const int groups = (n + 7) / 8;
  for (int vg0 = 0; vg0 < groups; vg0 += kMaxGridY) {
    dim3 grid(C.Bp / kChainTile, std::min(kMaxGridY, groups - vg0));
    k_keep_copy<<<grid, 256, 0, st>>>(F, C, n, vg0);
  }
  return cudaGetLastError();
}

cudaError_t launch_advance(uint32_t* tdev, uint32_t by, cudaStream_t st) {
  k_advance<<<1, 1, 0, st>>>(tdev, by);
  return cudaGetLastError();
}

cudaError_t launch_set_u32(uint32_t* dst, uint32_t value, cudaStream_t st) {
  k_set_u32<<<1, 1, 0, st>>>(dst, value);
  return cudaGetLastError();
}

cudaError_t launch_transpose_in(const uint8_t* assign, int B, int n, uint8_t* xt, int Bp,
                                cudaStream_t st) {
  dim3 grid((n + 31) / 32, Bp / 32);
  k_transpose_in<<<grid, dim3(32, 8), 0, st>>>(assign, B, n, xt, Bp);
  return cudaGetLastError();
}

}  // namespace rbmsat
