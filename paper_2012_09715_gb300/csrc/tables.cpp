// Host FP64 construction of the approximation tables.
//
//  * Piecewise constant on n equal intervals (Section 2.2, Corollary 2.3):
//    Z^E (conditional mean), Z^C (centre), Z^I (endpoint nearest 1/2).
//  * Piecewise linear on dyadic intervals (Section 2.3, Theorem 2.4, r = 1/2):
//    L2-optimal line per interval from the moments
//      M0 = int_a^b Phi^{-1}(u) du     = phi(z_a) - phi(z_b)
//      M1 = int_a^b u Phi^{-1}(u) du   = a phi(z_a) - b phi(z_b)
//                                        + (Phi(sqrt2 z_b) - Phi(sqrt2 z_a)) / (2 sqrt pi)
//    solved in the centred basis 1, (u - m): beta = 12 (M1 - m M0) / h^3,
//    alpha = M0 / h - beta m  (m = (a+b)/2, h = b - a), which is the solution
//    of the normal equations of the proof of Theorem 2.4.
#include <cmath>
#include <cstdlib>
#include <new>

#include "aicdf_internal.h"
#include "quad.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kInvSqrt2Pi = 0.39894228040143267794;

double npdf(double z) { return kInvSqrt2Pi * std::exp(-0.5 * z * z); }
// lower-tail CDF without cancellation
double ncdf(double z) { return 0.5 * std::erfc(-z / std::sqrt(2.0)); }

}  // namespace

namespace aicdf {

// Phi^{-1}(p): start from the rational approximation of Abramowitz & Stegun
// 26.2.23 (error < 4.5e-4) and take Halley steps on Phi(z) - p; the residual
// uses erf near the centre and erfc in the tail to avoid cancellation.
double host_phiinv(double p) {
  if (!(p >= 0.0 && p <= 1.0)) return NAN;
  if (p == 0.0) return -INFINITY;
  if (p == 1.0) return INFINITY;
  if (p == 0.5) return 0.0;
  const bool upper = p > 0.5;
  const double q = upper ? 1.0 - p : p;  // exact for p >= 1/2
  const double t = std::sqrt(-2.0 * std::log(q));
  double z = -(t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                       (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t));
  for (int it = 0; it < 6; ++it) {
    double r = (q < 0.3) ? ncdf(z) - q : 0.5 * std::erf(z / std::sqrt(2.0)) - (q - 0.5);
    double d = npdf(z);
    if (d <= 0.0) break;
    double s = r / d;                     // Newton step
    double zn = z - s / (1.0 + 0.5 * z * s);  // Halley correction (Phi'' = -z phi)
    if (zn == z) break;
    z = zn;
  }
  return upper ? -z : z;
}

}  // namespace aicdf

static aicdf_status build_pwc(aicdf_table_s *t, int n, int cons) {
  t->c0.resize(n);
  std::vector<double> z(n + 1);
  for (int k = 0; k <= n; ++k) z[k] = aicdf::host_phiinv((double)k / n);
  for (int k = 0; k < n; ++k) {
    const double lo = (double)k / n, hi = (double)(k + 1) / n;
    double q;
    if (cons == AICDF_Z_E || cons == AICDF_Z_V) {
      // n * (phi(z_k) - phi(z_{k+1})), written as
      // -n phi(z_k) expm1(-(z_{k+1} - z_k)(z_{k+1} + z_k)/2) to keep digits near 1/2.
      if (k == 0) q = -n * npdf(z[1]);
      else if (k == n - 1) q = n * npdf(z[n - 1]);
      else q = -n * npdf(z[k]) * std::expm1(-0.5 * (z[k + 1] - z[k]) * (z[k + 1] + z[k]));
    } else if (cons == AICDF_Z_C) {
      q = aicdf::host_phiinv(0.5 * (lo + hi));
    } else {
      q = (lo >= 0.5) ? z[k] : (hi < 0.5 ? z[k + 1] : 0.0);
    }
    t->c0[k] = q;
  }
  if (cons == AICDF_Z_V) {  // unit mean square (n = 2: the Rademacher values +-1)
    double m2 = 0.0;
    for (int k = 0; k < n; ++k) m2 += t->c0[k] * t->c0[k];
    const double sc = 1.0 / std::sqrt(m2 / n);
    for (int k = 0; k < n; ++k) t->c0[k] *= sc;
  }
  t->c1.clear();
  return AICDF_OK;
}

static aicdf_status build_pwl(aicdf_table_s *t, int K) {
  t->c0.assign(K + 1, 0.0);
  t->c1.assign(K + 1, 0.0);
  for (int k = 1; k <= K; ++k) {
    const double b = std::ldexp(1.0, -k);
    const double a = (k == K) ? 0.0 : 0.5 * b;
    const double zb = aicdf::host_phiinv(b);
    const double pb = npdf(zb), Pb2 = ncdf(std::sqrt(2.0) * zb);
    double pa = 0.0, Pa2 = 0.0;
    if (a > 0.0) {
      const double za = aicdf::host_phiinv(a);
      pa = npdf(za);
      Pa2 = ncdf(std::sqrt(2.0) * za);
    }
    const double M0 = pa - pb;
    const double M1 = a * pa - b * pb + (Pb2 - Pa2) / (2.0 * std::sqrt(kPi));
    const double h = b - a, m = 0.5 * (a + b);
    const double beta = 12.0 * (M1 - m * M0) / (h * h * h);
    const double alpha = M0 / h - beta * m;
    t->c0[k] = alpha;
    t->c1[k] = beta;
  }
  return AICDF_OK;
}

// Piecewise polynomial of degree d on the dyadic intervals (Section 2.3: the
// best L2 polynomial on each interval) in the local variable s in [0, 1).
// Projection onto shifted Legendre polynomials L_j(s) (orthogonal on [0,1],
// int L_j^2 = 1/(2j+1)), so no linear system is solved:
//   D = sum_j (2j+1) <f, L_j>_s L_j(s),  <f, L_j>_s = (1/h) int_{I_k} L_j(s(u)) f(u) du,
// then expanded to monomials in s.  Moments: Gauss-Legendre in u on the regular
// intervals; on the singular interval (0, b) the substitution u = b e^{-w}
// (s = e^{-w}, w in [0, 80], 40 panels).
static aicdf_status build_pwp(aicdf_table_s *t, int K, int deg) {
  t->c0.assign(4 * (K + 1), 0.0);  // row-major [row][power]
  std::vector<double> gx, gw;
  aicdf::gl_nodes(40, gx, gw);
  for (int k = 1; k <= K; ++k) {
    const double b = std::ldexp(1.0, -k);
    aicdf::LegendreProjector pr;  // (1/h) int L_j(s) f du = int_0^1 L_j(s) f(u(s)) ds
    if (k < K) {
      const double a = 0.5 * b, h = b - a;
      for (size_t i = 0; i < gx.size(); ++i) {
        const double s = 0.5 * (gx[i] + 1.0);
        pr.add(s, aicdf::host_phiinv(a + h * s), 0.5 * gw[i]);
      }
    } else {
      // s = e^{-w}, ds = e^{-w} dw
      const int panels = 40;
      const double wmax = 80.0;
      for (int p = 0; p < panels; ++p) {
        const double w0 = wmax * p / panels, w1 = wmax * (p + 1) / panels;
        for (size_t i = 0; i < gx.size(); ++i) {
          const double wv = 0.5 * (w1 - w0) * gx[i] + 0.5 * (w1 + w0);
          const double s = std::exp(-wv);
          pr.add(s, aicdf::host_phiinv(b * s), 0.5 * (w1 - w0) * gw[i] * s);
        }
      }
    }
    pr.monomials(deg, &t->c0[4 * k]);
  }
  t->c1.clear();
  return AICDF_OK;
}

// The kernels' form of a polynomial table: row k's polynomial p(s) = sum_i
// c_i s^i, with c_i its FP32 coefficients, rewritten in v = min(u, 1 - u):
// s = alpha v + beta (alpha = 2^(k+1), beta = -1 on I_k = [2^-(k+1), 2^-k);
// alpha = 2^K, beta = 0 on the singular row K), so
// d_j = alpha^j sum_{i >= j} C(i, j) beta^(i - j) c_i, in FP64, rounded once
// to FP32.  The polynomial is the same up to that rounding; its terms d_j v^j
// stay within a small factor of the row's values because alpha v lies in
// [1, 2) on a regular interval.
static void pwp_rows_in_v(aicdf_table_s *t) {
  static const double binom[4][4] = {{1, 0, 0, 0}, {1, 1, 0, 0}, {1, 2, 1, 0}, {1, 3, 3, 1}};
  const int K = t->n;
  t->fv.assign(t->f0.size(), 0.0f);
  for (int r = 0; r <= K; ++r) {
    const double alpha = std::ldexp(1.0, r == K ? K : r + 1), beta = r == K ? 0.0 : -1.0;
    double ap = 1.0;  // alpha^j
    for (int j = 0; j < 4; ++j) {
      double d = 0.0, bp = 1.0;  // beta^(i - j)
      for (int i = j; i < 4; ++i) {
        d += binom[i][j] * bp * (double)t->f0[4 * r + i];
        bp *= beta;
      }
      t->fv[4 * r + j] = (float)(ap * d);
      ap *= alpha;
    }
  }
}

extern "C" aicdf_status aicdf_table_build(int method, int n, int construction, aicdf_table *out) {
  if (!out) return AICDF_ERR_ARG;
  *out = nullptr;
  if (method == AICDF_PWC) {
    if (n < 2 || n > 4096 || (n & (n - 1))) return AICDF_ERR_ARG;
    if (construction < AICDF_Z_E || construction > AICDF_Z_V) return AICDF_ERR_ARG;
  } else if (method == AICDF_PWL) {
    if (n < 1 || n > 31) return AICDF_ERR_ARG;
  } else if (method == AICDF_PWP) {
    if (n < 1 || n > 31 || construction < 1 || construction > 3) return AICDF_ERR_ARG;
  } else {
    return AICDF_ERR_ARG;
  }
  aicdf_table_s *t = new (std::nothrow) aicdf_table_s();
  if (!t) return AICDF_ERR_NOMEM;
  t->magic = AICDF_TABLE_MAGIC;
  t->method = method;
  t->n = n;
  t->construction = construction;
  aicdf_status s = (method == AICDF_PWC)   ? build_pwc(t, n, construction)
                   : (method == AICDF_PWL) ? build_pwl(t, n)
                                           : build_pwp(t, n, construction);
  if (s != AICDF_OK) {
    delete t;
    return s;
  }
  t->f0.assign(t->c0.begin(), t->c0.end());
  t->f1.assign(t->c1.begin(), t->c1.end());
  if (method == AICDF_PWP) pwp_rows_in_v(t);
  *out = t;
  return AICDF_OK;
}

extern "C" void aicdf_table_destroy(aicdf_table t) {
  if (t && t->magic == AICDF_TABLE_MAGIC) {
    t->magic = 0;
    delete t;
  }
}

extern "C" aicdf_status aicdf_table_get(aicdf_table t, double *c0, double *c1, int cap, int *n_out) {
  if (!aicdf::table_ok(t) || !c0 || cap < 0) return AICDF_ERR_ARG;
  const int cnt = (int)t->c0.size();
  if (cap < cnt) return AICDF_ERR_ARG;
  for (int i = 0; i < cnt; ++i) c0[i] = t->c0[i];
  if (t->method == AICDF_PWL) {
    if (!c1) return AICDF_ERR_ARG;
    for (int i = 0; i < cnt; ++i) c1[i] = t->c1[i];
  }
  if (n_out) *n_out = cnt;
  return AICDF_OK;
}

extern "C" aicdf_status aicdf_table_info(aicdf_table t, int *method, int *n) {
  if (!aicdf::table_ok(t)) return AICDF_ERR_ARG;
  if (method) *method = t->method;
  if (n) *n = t->n;
  return AICDF_OK;
}
