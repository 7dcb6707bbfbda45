// Gauss-Legendre nodes and the shifted Legendre basis used by the host-side
// L2 projections (the polynomial tables of Section 2.3 and Section 5.1).
#pragma once

#include <cmath>
#include <vector>

namespace aicdf {

// n-point Gauss-Legendre rule on [-1, 1]: Newton on P_n from the
// Chebyshev-like start, P_n and P_n' by the three-term recurrence.
inline void gl_nodes(int n, std::vector<double> &x, std::vector<double> &w) {
  const double pi = 3.14159265358979323846;
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// shifted Legendre L_0..L_3 on [0, 1] as monomial coefficients [j][power];
// orthogonal with int_0^1 L_j^2 = 1 / (2j + 1)
constexpr double kShiftedLegendre[4][4] = {{1, 0, 0, 0}, {-1, 2, 0, 0}, {1, -6, 6, 0}, {-1, 12, -30, 20}};

// Accumulates the projections int_0^1 L_j(s) f ds (j = 0..3) of one interval
// and expands sum_{j <= deg} (2j+1) proj_j L_j(s) into monomial coefficients.
struct LegendreProjector {
  double proj[4] = {0, 0, 0, 0};
  void add(double s, double f, double weight) {
    for (int j = 0; j < 4; ++j) {
      const double *c = kShiftedLegendre[j];
      proj[j] += weight * (((c[3] * s + c[2]) * s + c[1]) * s + c[0]) * f;
    }
  }
  void monomials(int deg, double *out4) const {
    for (int p = 0; p < 4; ++p) out4[p] = 0.0;
    for (int j = 0; j <= deg; ++j) {
      const double dj = (2.0 * j + 1.0) * proj[j];
      for (int p = 0; p < 4; ++p) out4[p] += dj * kShiftedLegendre[j][p];
    }
  }
};

}  // namespace aicdf
