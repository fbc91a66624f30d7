// Probability and free-energy tables of the clause RBMs.
//
// With the negation transform (Eq. 4), hidden unit h of a clause sees the
// logit b'_h + sum_k W'_kh v_k = b_h + sum_k W_kh tau_k, where tau_k is the
// truth of the clause's k-th literal. So one clause's hidden conditional
// (Eq. 2 / Eq. 6) and free energy (Eq. 1) depend only on the pattern
// p = sum_k tau_k 2^k of true literals, and its contributions to the visible
// logits (Eq. 7) only on the pattern hp = sum_h h_h 2^h of sampled hidden
// units. Per group g (clause length K, weight bucket) with L hidden units and
// per temperature e the tables hold
//   rec[g][e][p][.]   one record of 4 ceil((L + 1) / 4) u32 words per
//                     pattern: word 0 the clause free energy
//                     -sum_h softplus(b_h + sum_k W_kh tau_k(p)) (float bits),
//                     word 1 + h hidden unit h's threshold
//                     P = rint(65536 sigma(b_h + sum_k W_kh tau_k(p))) as
//                     (min(P, 65535) << 16) | [P == 65536], then zeros
//   feq[g][e][p]      rint(2^20 F) of that free energy (int32; parallel tempering)
//   gq[g][e][hp][k]   2^Q sum_h W_kh [bit h of hp]                     (int16)
// A 16-bit draw u gives 1 iff u < P. With a threshold word t, u in the high
// half of a 32-bit word x (any low half) gives x < t iff u < min(P, 65535),
// so the draw is [x < t] | (t & 1): no field needs extracting.
// and the visible table pv[q] = rint(65536 sigma(q 2^-Q)) for |q| <= qmax.
// A Bernoulli draw with a 16-bit uniform u is [u < P]. Beyond |z| >= 12 the
// 16-bit probabilities are exactly 0 and 65536, so qmax = 12 * 2^Q clamps
// without changing any draw.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace rbmsat {

namespace {
double sigmoid(double a) { return 1.0 / (1.0 + std::exp(-a)); }
double softplus(double a) { return a > 0 ? a + std::log1p(std::exp(-a)) : std::log1p(std::exp(a)); }
uint32_t prob16(double a) { return (uint32_t)std::nearbyint(sigmoid(a) * 65536.0); }
}  // namespace

std::string build_tables(const std::vector<RbmSet>& sets, int E, int Q,
                         const std::vector<int32_t>& grp_len,
                         const std::vector<int32_t>& grp_bucket, HostTables* T) {
  const int G = (int)grp_len.size();
  T->n_groups = G;
  T->n_temps = E;
  T->quant_bits = Q;
  T->qmax = 12 << Q;
  T->grp_len = grp_len;
  T->grp_bucket = grp_bucket;
  T->grp_nh.assign(G, 0);
  T->meta.assign(G, GroupMeta{});
  T->rec.clear();
  T->feq.clear();
  T->feq_ok = true;
  T->gq.clear();
  T->gq_absmax = 0;
  T->max_nh = 0;
  const double scale = std::ldexp(1.0, Q);
  for (int g = 0; g < G; ++g) {
    const int K = grp_len[g];
    GroupMeta& gm = T->meta[g];
    gm.len = K;
    gm.rec_off = (int32_t)T->rec.size();
    gm.feq_off = (int32_t)T->feq.size();
    gm.gq_off = (int32_t)T->gq.size();
    for (int e = 0; e < E; ++e) {
      const RbmSet* s = nullptr;
      for (const auto& c : sets)
        if (c.len == K && c.bucket == grp_bucket[g] && c.temp == e) s = &c;
      if (!s)
        return "no OR-gate RBM set for clause length " + std::to_string(K) + ", bucket " +
               std::to_string(grp_bucket[g]) + ", temperature " + std::to_string(e);
      const int L = s->nh;
      if (e == 0) {
        T->grp_nh[g] = L;
        gm.nh = L;
        gm.stride = 4 * ((L + 1 + 3) / 4);
        T->max_nh = std::max(T->max_nh, L);
      }
      if (T->grp_nh[g] != L)
        return "sets of one length and bucket must share n_hidden across temperatures";
      std::vector<int32_t> Wq((size_t)K * L);
      for (int i = 0; i < K * L; ++i) {
        const double v = s->W[i] * scale;
        if (!std::isfinite(v) || v != std::nearbyint(v) || std::fabs(v) > 16384.0)
          return "W entries must be multiples of 2^-quant_bits below 16384 * 2^-quant_bits";
        Wq[i] = (int32_t)v;
      }
      for (int h = 0; h < L; ++h) {
        const double v = std::ldexp(s->b[h], 24);
        if (!std::isfinite(v) || v != std::nearbyint(v) || std::fabs(s->b[h]) > 1048576.0)
          return "b entries must be multiples of 2^-24 below 2^20 in magnitude";
      }
      for (int p = 0; p < (1 << K); ++p) {
        double F = 0.0;
        std::vector<uint32_t> words(gm.stride, 0);
        for (int h = 0; h < L; ++h) {
          int64_t acc = 0;
          for (int k = 0; k < K; ++k)
            if ((p >> k) & 1) acc += Wq[k * L + h];
          const double a = s->b[h] + (double)acc / scale;
          const uint32_t P = prob16(a);
          words[1 + h] = ((P < 65535u ? P : 65535u) << 16) | (P == 65536u ? 1u : 0u);
          if (P == 65536u) gm.sat = 1;
          F -= softplus(a);
        }
        const double Fq = std::nearbyint(std::ldexp(F, 20));
        if (!(std::fabs(Fq) < 2147483647.0)) T->feq_ok = false;
        T->feq.push_back(T->feq_ok ? (int32_t)Fq : 0);
        const float Ff = (float)F;
        std::memcpy(&words[0], &Ff, 4);
        for (uint32_t w : words) T->rec.push_back(w);
      }
      for (int hp = 0; hp < (1 << L); ++hp) {
        for (int k = 0; k < K; ++k) {
          int32_t acc = 0;
          for (int h = 0; h < L; ++h)
            if ((hp >> h) & 1) acc += Wq[k * L + h];
          if (acc > 32767 || acc < -32767) return "2^Q G exceeds the int16 range";
          T->gq.push_back((int16_t)acc);
          if (std::abs(acc) > T->gq_absmax) T->gq_absmax = std::abs(acc);
        }
      }
      // byte counts of the tables (gq: two-sided on the device) fit an int
      if (T->rec.size() > (size_t)INT32_MAX / 4 || T->gq.size() > (size_t)INT32_MAX / 4)
        return "tables too large";
    }
  }
  T->pv.resize(2 * (size_t)T->qmax + 1);
  for (int q = -T->qmax; q <= T->qmax; ++q) T->pv[q + T->qmax] = prob16((double)q / scale);
  return "";
}

}  // namespace rbmsat
