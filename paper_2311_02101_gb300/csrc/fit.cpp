// Host-side fitting of canonical OR-gate clause RBMs (Sec. 4.1 "Learning OR
// gate RBM parameters"; appendix "Pretraining").
//
// The clause free energy with no visible bias is
//   F(v) = -sum_h softplus(b_h + sum_k W_kh v_k)            (Eq. 1)
// and the fit regresses it onto the OR target over all 2^K inputs:
//   min ||F(0)||^2 + sum_{v != 0} ||F(v) - F_s||^2,  F_s = -F*,
// with Adam at learning rate 1e-3. W is then rounded to the 2^-Q grid, b is
// refitted with W held fixed and rounded to the 2^-24 grid, so that every
// hidden logit is an exact double and every visible logit an exact multiple
// of 2^-Q.
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace rbmsat {

int hidden_units_for(int len) { return len <= 3 ? 3 : len + 1; }

namespace {

double softplus(double a) { return a > 0 ? a + std::log1p(std::exp(-a)) : std::log1p(std::exp(a)); }
double sigmoid(double a) { return 1.0 / (1.0 + std::exp(-a)); }

// Deterministic N(0, 0.1) start (splitmix64 + Box-Muller): breaks the symmetry
// between hidden units; the fit is not required to match any other fitter.
struct SplitMix {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
};

struct Adam {
  std::vector<double> m1, m2;
  int it = 0;
  explicit Adam(size_t n) : m1(n, 0.0), m2(n, 0.0) {}
  void step(std::vector<double>& p, const std::vector<double>& g, double lr, size_t from,
            size_t to) {
    ++it;
    const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
    const double c1 = 1.0 - std::pow(b1, it), c2 = 1.0 - std::pow(b2, it);
    for (size_t i = from; i < to; ++i) {
      m1[i] = b1 * m1[i] + (1 - b1) * g[i];
      m2[i] = b2 * m2[i] + (1 - b2) * g[i] * g[i];
      p[i] -= lr * (m1[i] / c1) / (std::sqrt(m2[i] / c2) + eps);
    }
  }
};

// Gradient of the regression loss. p = [W (K x L row-major), b (L)].
void loss_grad(int K, int L, double fstar, const std::vector<double>& p,
               std::vector<double>& g) {
  std::fill(g.begin(), g.end(), 0.0);
  const int P = 1 << K;
  std::vector<double> a(L);
  for (int v = 0; v < P; ++v) {
    double F = 0.0;
    for (int h = 0; h < L; ++h) {
      double s = p[K * L + h];
      for (int k = 0; k < K; ++k)
        if ((v >> k) & 1) s += p[k * L + h];
      a[h] = s;
      F -= softplus(s);
    }
    const double r = F - (v == 0 ? 0.0 : -fstar);
    for (int h = 0; h < L; ++h) {
      const double ga = 2.0 * r * (-sigmoid(a[h]));
      g[K * L + h] += ga;
      for (int k = 0; k < K; ++k)
        if ((v >> k) & 1) g[k * L + h] += ga;
    }
  }
}

}  // namespace

int fit_or_rbm(int K, int L, double fstar, int Q, int iters, double* W_out,
               double* b_out) {
  if (K < 1 || K > MAXSAT_MAX_LEN || L < 1 || L > MAXSAT_MAX_HIDDEN || Q < 0 || Q > 12 ||
      iters < 0 || !std::isfinite(fstar))
    return MAXSAT_EINVAL;
  const double lr = 1e-3;
  std::vector<double> p(K * L + L, 0.0), g(p.size());
  SplitMix rng{0x5EED0000ull + 131ull * K + 7ull * L};
  for (int i = 0; i < K * L; ++i) {
    double u1 = rng.uniform(), u2 = rng.uniform();
    p[i] = 0.1 * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
  Adam opt(p.size());
  for (int it = 0; it < iters; ++it) {
    loss_grad(K, L, fstar, p, g);
    opt.step(p, g, lr, 0, p.size());
  }
  // W onto the 2^-Q grid (round half to even), then refit b with W fixed
  const double scale = std::ldexp(1.0, Q);
  for (int i = 0; i < K * L; ++i) p[i] = std::nearbyint(p[i] * scale) / scale;
  Adam opt_b(p.size());
  const int refit = 2000;
  for (int it = 0; it < refit; ++it) {
    loss_grad(K, L, fstar, p, g);
    opt_b.step(p, g, lr, K * L, p.size());
  }
  for (int i = 0; i < K * L; ++i) W_out[i] = p[i];
  for (int h = 0; h < L; ++h) b_out[h] = std::nearbyint(std::ldexp(p[K * L + h], 24)) / 16777216.0;
  return MAXSAT_OK;
}

}  // namespace rbmsat

extern "C" int maxsat_fit_or_rbm(int32_t len, int32_t n_hidden, double fstar,
                                 int32_t quant_bits, int32_t iters, double* W_out,
                                 double* b_out) {
  if (!W_out || !b_out) return MAXSAT_EINVAL;
  return rbmsat::fit_or_rbm(len, n_hidden, fstar, quant_bits, iters, W_out, b_out);
}
