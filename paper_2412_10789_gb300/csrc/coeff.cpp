// Host FP64 coefficient engine: Chebyshev coefficients c_k of the SSPPR and
// HKPR functions, their tails, Taylor coefficients for the PwMethod baseline,
// and the truncation rules.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gp_internal.h"

namespace gp {

namespace {

// Lemma 2: with root = sqrt(2 alpha - alpha^2), gamma = alpha / root and
// beta = (1 - root) / (1 - alpha); c_0 = gamma, c_k = 2 gamma beta^k.
// Because 1 - root^2 = (1 - alpha)^2, beta = (1 - alpha) / (1 + root), which
// avoids the cancellation of 1 - root when alpha is close to 1.
void ppr_terms(double alpha, int kmax, double* c, double* gamma_out, double* beta_out) {
  const double root = std::sqrt(alpha * (2.0 - alpha));
  const double gamma = alpha / root;
  const double beta = (1.0 - alpha) / (1.0 + root);
  c[0] = gamma;
  double p = 1.0;
  for (int k = 1; k <= kmax; ++k) {
    p *= beta;
    c[k] = 2.0 * gamma * p;
  }
  if (gamma_out) *gamma_out = gamma;
  if (beta_out) *beta_out = beta;
}

// Highest order the HKPR recurrence starts from for coefficients up to kmax.
int hkpr_top(double t, int kmax) { return std::max(kmax, (int)std::ceil(t + 12.0 * std::sqrt(t) + 40.0)) + 24; }

// Lemma 3: c_0 = e^-t I_0(t), c_k = 2 e^-t I_k(t), for k = 0..top into
// all[0..top] (v needs top + 2 entries of scratch).  The scaled values
// e^-t I_k(t) come from Miller's backward recurrence
// I_{k-1}(t) = (2k / t) I_k(t) + I_{k+1}(t), started far above the wanted
// orders with an arbitrary small value and normalised by the generating-function
// identity I_0(t) + 2 sum_{k>=1} I_k(t) = e^t (equivalently sum_k c_k = 1).
void hkpr_terms(double t, int top, double* v, double* all) {
  v[top + 1] = 0.0;
  v[top] = 1e-280;
  for (int k = top; k >= 1; --k) {
    v[k - 1] = (2.0 * k / t) * v[k] + v[k + 1];
    if (v[k - 1] > 1e250) {  // rescale to stay in range; ratios are what matter
      for (int j = k - 1; j <= top; ++j) v[j] *= 1e-250;
    }
  }
  double norm = v[0];
  for (int k = 1; k <= top; ++k) norm += 2.0 * v[k];
  all[0] = v[0] / norm;
  for (int k = 1; k <= top; ++k) all[k] = 2.0 * v[k] / norm;
}

void ppr_coefficients(double alpha, int kmax, std::vector<double>& c, std::vector<double>& tail) {
  c.assign(kmax + 1, 0.0);
  tail.assign(kmax + 1, 0.0);
  double gamma = 0.0, beta = 0.0;
  ppr_terms(alpha, kmax, c.data(), &gamma, &beta);
  // tail(k) = sum_{l>k} 2 gamma beta^l = 2 gamma beta^{k+1} / (1 - beta)
  for (int k = 0; k <= kmax; ++k) tail[k] = 2.0 * gamma * std::pow(beta, k + 1) / (1.0 - beta);
}

void hkpr_coefficients(double t, int kmax, std::vector<double>& c, std::vector<double>& tail) {
  const int top = hkpr_top(t, kmax);
  std::vector<double> v(top + 2, 0.0), all(top + 1);
  hkpr_terms(t, top, v.data(), all.data());
  c.assign(all.begin(), all.begin() + kmax + 1);
  tail.assign(kmax + 1, 0.0);
  // tail(k) = sum_{l>k} c_l, summed from the top (small terms first)
  double s = 0.0;
  std::vector<double> suffix(top + 2, 0.0);
  for (int k = top; k >= 0; --k) {
    suffix[k] = s;  // sum over l > k
    s += all[k];
  }
  for (int k = 0; k <= kmax; ++k) tail[k] = suffix[k];
}

}  // namespace

int cheb_coefficients_work(int function, double param, int kmax) {
  return function == GP_FN_PPR ? 0 : 2 * hkpr_top(param, kmax) + 3;
}

bool cheb_coefficients_into(int function, double param, int kmax, double* c, double* work, int work_len) {
  if (function == GP_FN_PPR) {
    ppr_terms(param, kmax, c, nullptr, nullptr);
    return true;
  }
  const int top = hkpr_top(param, kmax);
  if (work_len < 2 * top + 3) return false;
  double* v = work;             // top + 2
  double* all = work + top + 2; // top + 1
  hkpr_terms(param, top, v, all);
  for (int k = 0; k <= kmax; ++k) c[k] = all[k];
  return true;
}

void cheb_coefficients(int function, double param, int kmax, std::vector<double>& c,
                       std::vector<double>& tail) {
  if (function == GP_FN_PPR)
    ppr_coefficients(param, kmax, c, tail);
  else
    hkpr_coefficients(param, kmax, c, tail);
}

void taylor_coefficients(int function, double param, double tol, int nmax, std::vector<double>& z) {
  z.clear();
  if (function == GP_FN_PPR) {
    // zeta_k = alpha (1-alpha)^k; sum_{k>=N} zeta_k = (1-alpha)^N
    double p = 1.0;
    for (int k = 0; k < nmax; ++k) {
      z.push_back(param * p);
      p *= (1.0 - param);
      if (p <= tol) break;
    }
  } else {
    // zeta_k = e^-t t^k / k!; the tail is summed forward until negligible
    std::vector<double> all;
    double term = std::exp(-param);
    for (int k = 0; k < nmax + 64; ++k) {
      all.push_back(term);
      term = term * param / (double)(k + 1);
      if (k > param && term < 1e-300) break;
    }
    std::vector<double> suffix(all.size() + 1, 0.0);
    for (int k = (int)all.size() - 1; k >= 0; --k) suffix[k] = suffix[k + 1] + all[k];
    for (int k = 0; k < nmax && k < (int)all.size(); ++k) {
      z.push_back(all[k]);
      if (suffix[k + 1] <= tol) break;
    }
  }
}

int paper_k(int function, double param, double tol) {
  double k = function == GP_FN_PPR ? std::log(1.0 / tol) / std::sqrt(param)
                                   : std::sqrt(param) * std::log(1.0 / tol);
  return std::max(1, (int)std::ceil(k));
}

int k_lower(const std::vector<double>& tail, double tol, double cmin) {
  for (size_t k = 1; k < tail.size(); ++k)
    if (tail[k] * cmin <= tol) return (int)k;
  return (int)tail.size() - 1;
}

}  // namespace gp
