// Exact non-central chi-squared quantile on the GPU, FP64 (Section 5).
//
// C_nu(x; lambda) = sum_j Pois(j; lambda/2) P(nu/2 + j, x/2)   (Poisson mixture of
// central chi-squared CDFs), and the upper tail Q = 1 - C the same with the
// regularised upper gamma Q(s, y).  With y = x/2, s_j = nu/2 + j and
// g_j = y^{s_j} e^-y / Gamma(s_j + 1):
//   P(s_j - 1, y) = P(s_j, y) + g_{j-1},   g_{j-1} = g_j s_j / y     (downward, adds)
//   Q(s_j + 1, y) = Q(s_j, y) + g_j,       g_{j+1} = g_j y / (s_j + 1) (upward, adds)
// so the lower CDF is summed downward from the top of the Poisson range and
// the upper tail upward from its bottom: every recurrence step adds positive
// terms.  Only one incomplete gamma is evaluated directly (series below
// s + 1, continued fraction above, each giving the small one of P and Q).  The
// density is sum_j p_j g_{j-1} / 2.  The quantile solves C = u for u <= 1/2 and
// Q = 1 - u above (1 - u is exact for FP32 u >= 1/2), by Newton steps kept
// inside a bracket, started from Sankaran's approximation (Section 5.1).
// Every loop has a fixed cap; hitting one sets the returned status bit.  The
// functions are host+device: the table builder of Section 5.1 runs them on
// the host in FP64.
#pragma once

#include <cmath>
#include <cstdint>

#define AICDF_HD __host__ __device__ __forceinline__

namespace aicdf {

constexpr int kNcx2NoConverge = 1;

// log Gamma(s), s > 0: shift to s >= 12 (one log of the product), then the
// Stirling series through the s^-11 term (truncation error < 1e-16).
AICDF_HD double lgamma_pos(double s) {
  double prod = 1.0;
  while (s < 12.0) {  // at most 12 iterations for s > 0
    prod *= s;
    s += 1.0;
  }
  const double r = 1.0 / s, r2 = r * r;
  const double series =
      r * (1.0 / 12.0 -
           r2 * (1.0 / 360.0 -
                 r2 * (1.0 / 1260.0 - r2 * (1.0 / 1680.0 - r2 * (1.0 / 1188.0 - r2 * (691.0 / 360360.0))))));
  return (s - 0.5) * log(s) - s + 0.91893853320467274178 + series - log(prod);
}

// P(s, y), Q(s, y) and g(s) = y^s e^-y / Gamma(s+1): the series for y < s + 1
// (gives P), the continued fraction for Q otherwise (modified Lentz).
AICDF_HD void gamma_pq(double s, double y, double *P, double *Q, double *g, int *status) {
  const double lg = s * log(y) - y - lgamma_pos(s + 1.0);
  *g = exp(lg);
  if (y < s + 1.0) {
    double term = 1.0, sum = 1.0, d = s;
    int it = 0;
    for (; it < 2000; ++it) {
      d += 1.0;
      term *= y / d;
      sum += term;
      if (term < sum * 1e-17) break;
    }
    if (it == 2000) *status |= kNcx2NoConverge;
    *P = fmin(*g * sum, 1.0);
    *Q = 1.0 - *P;
    return;
  }
  const double tiny = 1e-300;
  double b = y + 1.0 - s, c = 1.0 / tiny, dd = 1.0 / b, h = dd;
  int i = 1;
  for (; i < 2000; ++i) {
    const double an = -i * (i - s);
    b += 2.0;
    dd = an * dd + b;
    if (fabs(dd) < tiny) dd = tiny;
    c = b + an / c;
    if (fabs(c) < tiny) c = tiny;
    dd = 1.0 / dd;
    const double del = dd * c;
    h *= del;
    if (fabs(del - 1.0) < 1e-16) break;
  }
  if (i == 2000) *status |= kNcx2NoConverge;
  *Q = fmin((*g) * s * h, 1.0);  // e^-y y^s / Gamma(s) = g s
  *P = 1.0 - *Q;
}

// Poisson range [jlo, jhi] of the mixture weights Pois(j; lambda/2) holding
// all but ~1e-20 of the mass, walked from the mode, with the weights at both
// ends.  It depends on lambda only, so a quantile computes it once.
struct Ncx2Range {
  int jlo, jhi;
  double plo, phi;
};

AICDF_HD Ncx2Range ncx2_range(double lam, int *status) {
  Ncx2Range r{0, 0, 1.0, 1.0};
  const double m = 0.5 * lam;
  if (m > 0.0) {
    const int j0 = (int)floor(m);
    const double p0 = exp(-m + j0 * log(m) - lgamma_pos(j0 + 1.0));
    const double rm = 1.0 / m;
    double p = p0;
    int j = j0, it = 0;
    for (; j > 0 && p > 1e-20 && it < 100000; ++it) {
      p *= (double)j * rm;
      --j;
    }
    if (it == 100000) *status |= kNcx2NoConverge;
    r.jlo = j;
    r.plo = p;
    p = p0;
    j = j0;
    for (it = 0; p > 1e-20 && it < 100000; ++it) {
      p *= m / (double)(j + 1);
      ++j;
    }
    if (it == 100000) *status |= kNcx2NoConverge;
    r.jhi = j;
    r.phi = p;
  }
  return r;
}

// Lower CDF (upper = false) or upper tail (upper = true) of chi'^2_nu(lambda)
// at x, and the density, over the Poisson range rg of lambda.
AICDF_HD void ncx2_tail_pdf(double x, double nu, double lam, const Ncx2Range &rg, bool upper, double *T,
                            double *f, int *status) {
  if (x <= 0.0) {
    *T = upper ? 1.0 : 0.0;
    *f = 0.0;
    return;
  }
  const double y = 0.5 * x, a = 0.5 * nu, m = 0.5 * lam;
  const double ry = 1.0 / y, h2y = 0.5 * ry;  // loop-invariant reciprocals
  const int jlo = rg.jlo, jhi = rg.jhi;
  const double plo = rg.plo, phi = rg.phi;
  double acc = 0.0, dens = 0.0;
  if (!upper) {
    const double rm = 1.0 / m;  // only used when jhi > jlo, i.e. m > 0
    double P, Q, g;
    gamma_pq(a + jhi, y, &P, &Q, &g, status);
    double p = phi;
    acc = p * P;
    dens = p * g * (a + jhi) * h2y;
    for (int j = jhi; j > jlo; --j) {
      g = g * (a + j) * ry;  // g_{j-1}
      P += g;                // P(s_{j-1})
      p *= (double)j * rm;   // p_{j-1}
      acc += p * P;
      dens += p * g * (a + j - 1) * h2y;
    }
  } else {
    double P, Q, g;
    gamma_pq(a + jlo, y, &P, &Q, &g, status);
    double p = plo;
    acc = p * Q;
    dens = p * g * (a + jlo) * h2y;
    for (int j = jlo; j < jhi; ++j) {
      Q += g;                    // Q(s_{j+1})
      g = g * y / (a + j + 1);   // g_{j+1}
      p *= m / (double)(j + 1);  // p_{j+1}
      acc += p * Q;
      dens += p * g * (a + j + 1) * h2y;
    }
  }
  *T = fmin(acc, 1.0);
  *f = dens;
}

// Sankaran's approximation of the quantile (Section 5.1; with sqrt(2 c2) in
// the normal term) at the normal quantile z = Phi^{-1}(u), used as the start.
AICDF_HD double ncx2_sankaran(double z, double nu, double lam) {
  const double k = nu, h0 = k + lam, h2 = k + 2.0 * lam;
  const double c1 = 1.0 - (2.0 / 3.0) * h0 * (k + 3.0 * lam) / (h2 * h2);
  const double c2 = h2 / (h0 * h0);
  const double c3 = (c1 - 1.0) * (1.0 - 3.0 * c1);
  const double base = 1.0 + c1 * c2 * (c1 - 1.0 + 0.5 * (2.0 - c1) * c2 * c3) +
                      c1 * sqrt(2.0 * c2) * (1.0 + 0.5 * c2 * c3) * z;
  if (!(base > 0.0) || !(fabs(c1) > 1e-3)) return h0;  // outside its range: start at the mean
  const double r = h0 * pow(base, 1.0 / c1);
  return (r > 0.0 && isfinite(r)) ? r : h0;
}

// The x with C(x) = target (upper = false) or 1 - C(x) = target (upper = true),
// 0 < target <= 1/2, from Sankaran's start at the normal quantile z of the
// same probability (FP64).  Lower tail: Newton on ln C(e^t) - ln target in
// t = ln x (C behaves like x^{nu/2} near 0, so this converges in a few steps
// however deep the tail); upper tail: Newton on 1 - C(x) - target in x.  Both
// keep the iterate inside a bracket and bisect when Newton leaves it.
AICDF_HD double ncx2_quantile(double target, bool upper, double z, double nu, double lam, int *status) {
  double T, f;
  const double x0 = ncx2_sankaran(z, nu, lam);
  const Ncx2Range rg = ncx2_range(lam, status);
  int it = 0;
  if (!upper) {
    const double lt = log(target);
    double t = log(x0), lo = -1e300, hi = 1e300;  // bracket in t = ln x
    for (; it < 100; ++it) {
      const double x = exp(t);
      ncx2_tail_pdf(x, nu, lam, rg, false, &T, &f, status);
      double tn;
      if (!(T > 0.0)) {  // C underflowed: x far too small
        lo = t;
        tn = hi < 1e300 ? 0.5 * (lo + hi) : t + 2.0;
      } else {
        const double r = log(T) - lt;  // > 0 when x is too large
        if (r > 0.0) hi = t;
        else lo = t;
        const double d = x * f / T;   // d ln C / d ln x
        tn = (d > 0.0) ? t - r / d : 0.5 * (lo + hi);
        if (!(tn > lo && tn < hi)) tn = (lo > -1e300 && hi < 1e300) ? 0.5 * (lo + hi) : (r > 0.0 ? t - 2.0 : t + 2.0);
      }
      const double dt = fabs(tn - t);
      t = tn;
      if (dt <= 1e-13 || (hi - lo) <= 1e-14) break;
    }
    if (it == 100) *status |= kNcx2NoConverge;
    return exp(t);
  }
  double x = x0;
  double lo = 0.0, hi = -1.0;  // hi < 0: no upper bound yet
  for (; it < 100; ++it) {
    ncx2_tail_pdf(x, nu, lam, rg, true, &T, &f, status);
    const double r = target - T;  // = C(x) - u, > 0 when x is too large
    if (r > 0.0) hi = x;
    else lo = x;
    double xn = (f > 0.0) ? x - r / f : -1.0;
    if (hi < 0.0) {
      if (!(xn > lo)) xn = 2.0 * x + 1.0;
    } else if (!(xn > lo && xn < hi)) {
      xn = 0.5 * (lo + hi);
    }
    const double dx = fabs(xn - x);
    x = xn;
    if (dx <= 1e-13 * x || (hi > 0.0 && hi - lo <= 1e-14 * hi)) break;
  }
  if (it == 100) *status |= kNcx2NoConverge;
  return x;
}

// Quantile C^{-1}_nu(u; lambda) for 0 < u < 1 (FP64; 1 - u is exact for the
// FP32 uniforms the paths use).
__device__ __forceinline__ double ncx2_ppf(double u, double nu, double lam, int *status) {
  if (!(u > 0.0)) return 0.0;
  if (!(u < 1.0)) return __longlong_as_double(0x7ff0000000000000ll);
  const bool upper = u > 0.5;
  return ncx2_quantile(upper ? 1.0 - u : u, upper, normcdfinv(u), nu, lam, status);
}

}  // namespace aicdf
