// theta_m(tol) for the truncated Taylor series (Al-Mohy & Higham, Section 3),
// computed on the host in double precision when the library is first used.
//
// Definition: with T_m the degree-m Taylor polynomial of exp,
//   h_{m+1}(x) = log(exp(-x) T_m(x)) = sum_{k>m} g_k x^k,
// theta_m is the largest theta with sum_{k>m} |g_k| theta^(k-1) <= tol.
//
// Method (independent of any other table in this project):
//   exp(-x) T_m(x) = 1 + sum_{k>m} a_k x^k with the closed form
//     a_k = (-1)^(k+m) / (k * m! * (k-1-m)!)
//   (the alternating binomial sum sum_{j<=m} (-1)^j C(k,j) = (-1)^m C(k-1,m)),
//   generated by the ratio a_{k+1} / a_k = -k / ((k-m)(k+1));
//   log of a series with constant term 1 by g_k = a_k - (1/k) sum_j j g_j a_{k-j};
//   everything is carried scaled by S^k (S = max(1, m/4)) to keep the terms
//   of degree up to m + 320 inside the double range;
//   theta by 200 bisection steps on the increasing function above.
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "qsw_internal.h"

namespace qsw {
namespace {

constexpr int kExtraTerms = 320;

double theta_for(int m, double tol) {
  const int kmax = m + kExtraTerms;
  const double S = m / 4.0 > 1.0 ? m / 4.0 : 1.0;
  std::vector<double> a(kmax + 1, 0.0), g(kmax + 1, 0.0);
  // a_{m+1} S^{m+1} = -S^{m+1} / (m+1)!
  double v = -1.0;
  for (int i = 1; i <= m + 1; ++i) v *= S / i;
  a[m + 1] = v;
  for (int k = m + 1; k < kmax; ++k) a[k + 1] = -a[k] * S * k / ((double)(k - m) * (k + 1));
  for (int k = m + 1; k <= kmax; ++k) {
    double acc = 0.0;
    for (int j = m + 1; j <= k - m - 1; ++j) acc += j * g[j] * a[k - j];
    g[k] = a[k] - acc / k;
  }
  // excess(theta) = sum |g_k| theta^(k-1) - tol, with g stored scaled by S^k:
  // |g_k| theta^(k-1) = |ghat_k| (theta/S)^k / theta.
  auto excess = [&](double th) {
    const double r = th / S;
    double pw = 1.0;
    for (int i = 0; i < m; ++i) pw *= r;   // r^m
    double sum = 0.0;
    for (int k = m + 1; k <= kmax; ++k) {
      pw *= r;
      sum += fabs(g[k]) * pw;
    }
    return sum / th - tol;
  };
  double lo = 0.0, hi = 1e-300;
  while (excess(hi) <= 0.0) {
    lo = hi;
    hi *= 2.0;
  }
  for (int it = 0; it < 2000 && hi - lo > 1e-17 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (excess(mid) <= 0.0) lo = mid;
    else hi = mid;
  }
  return lo;
}

std::once_flag g_once;
double g_theta[2][kMMax];

void fill_tables() {
  for (int m = 1; m <= kMMax; ++m) {
    g_theta[0][m - 1] = theta_for(m, ldexp(1.0, -53));
    g_theta[1][m - 1] = theta_for(m, ldexp(1.0, -24));
  }
}

}  // namespace

double tolerance(int precision) { return precision == QSW_C64_BULK ? ldexp(1.0, -24) : ldexp(1.0, -53); }

const double* theta_table(int precision) {
  std::call_once(g_once, fill_tables);
  return g_theta[precision == QSW_C64_BULK ? 1 : 0];
}

}  // namespace qsw
