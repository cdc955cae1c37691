// CPU ORACLE — test infrastructure only (see philox.hpp for the rule).
//
// Constant tables of the models, built here in FP64 from their definitions.
// The product library builds its own copies with its own code; tests compare
// them entry by entry.
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>

namespace orc {

// Sensor of the rock-sample robots (Sec. IV-A, multi-agent Rock Sample): its
// accuracy falls exponentially with distance, 0.5 + 0.5 * 2^(-d/20). A sense
// reading is correct iff the 32-bit draw u satisfies u < T[d^2] with
// T[d^2] = floor(p(d) * 2^32), kept as a 64-bit integer so that p = 1 at d = 0
// means "always correct".
inline std::vector<uint64_t> sensor_thresholds(int max_d2) {
  std::vector<uint64_t> t(max_d2 + 1);
  for (int d2 = 0; d2 <= max_d2; ++d2) {
    double d = std::sqrt((double)d2);
    double p = 0.5 + 0.5 * std::exp2(-d / 20.0);
    t[d2] = (uint64_t)std::floor(p * 4294967296.0);
  }
  return t;
}

// Discount powers gamma^k, k = 0..n-1, of the FP32 gamma evaluated in FP64.
template <class Real>
std::vector<Real> gamma_powers(float gamma, int n) {
  std::vector<Real> g(n);
  for (int k = 0; k < n; ++k) g[k] = (Real)std::pow((double)gamma, (double)k);
  return g;
}

// Standard normal CDF from the complementary error function.
inline double normal_cdf(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }

// Inverse-normal table for the pedestrian noise of the driving task: entry i is
// the (i + 0.5)/4096 quantile of N(0, 1), found by bisection on the CDF until
// the bracket stops shrinking.
inline std::vector<double> gauss_table_f64() {
  std::vector<double> t(4096);
  for (int i = 0; i < 4096; ++i) {
    double p = (i + 0.5) / 4096.0;
    double lo = -10.0, hi = 10.0;
    for (int it = 0; it < 400; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid == lo || mid == hi) break;
      if (normal_cdf(mid) < p)
        lo = mid;
      else
        hi = mid;
    }
    t[i] = 0.5 * (lo + hi);
  }
  return t;
}

}  // namespace orc
