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

// Stopping thresholds of the series, the continued fraction and the modified
// Lentz guard, per arithmetic (the FP32 form serves as the first phase of the
// device quantile, which an FP64 step then polishes).
template <class T>
struct Ncx2Eps;
template <>
struct Ncx2Eps<double> {
  static constexpr double series = 1e-17, cf = 1e-16, tiny = 1e-300, lg_min = -700.0;
};
template <>
struct Ncx2Eps<float> {
  static constexpr float series = 3e-8f, cf = 1e-7f, tiny = 1e-30f, lg_min = -80.0f;
};

// log Gamma(s), s > 0: shift to s >= 12 (one log of the product), then the
// Stirling series through the s^-11 term (truncation error < 1e-16).
template <class T>
AICDF_HD T lgamma_pos(T s) {
  T prod = T(1);
  while (s < T(12)) {  // at most 12 iterations for s > 0
    prod *= s;
    s += T(1);
  }
  const T r = T(1) / s, r2 = r * r;
  const T series =
      r * (T(1.0 / 12.0) -
           r2 * (T(1.0 / 360.0) -
                 r2 * (T(1.0 / 1260.0) -
                       r2 * (T(1.0 / 1680.0) - r2 * (T(1.0 / 1188.0) - r2 * T(691.0 / 360360.0))))));
  return (s - T(0.5)) * log(s) - s + T(0.91893853320467274178) + series - log(prod);
}

// P(s, y), Q(s, y) and g(s) = y^s e^-y / Gamma(s+1): the series for y < s + 1
// (gives P), the continued fraction for Q otherwise (modified Lentz).
template <class T>
AICDF_HD void gamma_pq(T s, T y, T *P, T *Q, T *g, int *status) {
  const T lg = s * log(y) - y - lgamma_pos<T>(s + T(1));
  *g = exp(lg);
  if (y < s + T(1)) {
    // terms y^k / ((s+1)...(s+k)), two per division
    T term = T(1), sum = T(1), d = s;
    int it = 0;
    for (; it < 2000; it += 2) {
      const T d1 = d + T(1), d2 = d + T(2);
      const T inv = T(1) / (d1 * d2);
      const T t1 = term * y * d2 * inv;  // term y / d1
      term = t1 * y * d1 * inv;          // t1 y / d2
      sum += t1 + term;
      d = d2;
      if (term < sum * Ncx2Eps<T>::series) break;
    }
    if (it == 2000) *status |= kNcx2NoConverge;
    *P = fmin(*g * sum, T(1));
    *Q = T(1) - *P;
    return;
  }
  const T tiny = Ncx2Eps<T>::tiny;
  T b = y + T(1) - s, c = T(1) / tiny, dd = T(1) / b, h = dd;
  int i = 1;
  for (; i < 2000; ++i) {
    const T an = -T(i) * (T(i) - s);
    b += T(2);
    dd = an * dd + b;
    if (fabs(dd) < tiny) dd = tiny;
    c = b + an / c;
    if (fabs(c) < tiny) c = tiny;
    dd = T(1) / dd;
    const T del = dd * c;
    h *= del;
    if (fabs(del - T(1)) < Ncx2Eps<T>::cf) break;
  }
  if (i == 2000) *status |= kNcx2NoConverge;
  *Q = fmin((*g) * s * h, T(1));  // e^-y y^s / Gamma(s) = g s
  *P = T(1) - *Q;
}

// Poisson range [jlo, jhi] of the mixture weights Pois(j; lambda/2) down to
// the weight `cut`, walked from the mode, with the weights at both ends.  Every
// term of the CDF or its tail is at most its weight, so a cut of 1e-8 times
// the probability sought keeps 1e-8 of it (and 1e-20 is used at least).  A
// quantile computes it once.
template <class T>
struct Ncx2Range {
  int jlo, jhi;
  T plo, phi;
};

template <class T>
AICDF_HD Ncx2Range<T> ncx2_range(T lam, T cut, int *status) {
  Ncx2Range<T> r{0, 0, T(1), T(1)};
  const T m = T(0.5) * lam;
  if (m > T(0)) {
    const int j0 = (int)floor(m);
    const T p0 = exp(-m + T(j0) * log(m) - lgamma_pos<T>(T(j0) + T(1)));
    const T rm = T(1) / m;
    T p = p0;
    int j = j0, it = 0;
    for (; j > 0 && p > cut && it < 100000; ++it) {
      p *= T(j) * rm;
      --j;
    }
    if (it == 100000) *status |= kNcx2NoConverge;
    r.jlo = j;
    r.plo = p;
    p = p0;
    j = j0;
    for (it = 0; p > cut && it < 100000; ++it) {
      p *= m / T(j + 1);
      ++j;
    }
    if (it == 100000) *status |= kNcx2NoConverge;
    r.jhi = j;
    r.phi = p;
  }
  return r;
}

// Lower CDF (upper = false) or upper tail (upper = true) of chi'^2_nu(lambda)
// at x, and the density, over the Poisson range rg of lambda.  With D1 also
// the density's derivative: the central chi-squared density f_s (s = nu/2 + j)
// has f_s' = f_s ((s - 1)/y - 1)/2, so f' = (sum p_j f_j (s_j - 1))/(2y) - f/2.
template <class T, bool D1 = false>
AICDF_HD void ncx2_tail_pdf(T x, T nu, T lam, const Ncx2Range<T> &rg, bool upper, T *Tout, T *f, int *status,
                            T *fprime = nullptr) {
  if (x <= T(0)) {
    *Tout = upper ? T(1) : T(0);
    *f = T(0);
    if (D1) *fprime = T(0);
    return;
  }
  const T y = T(0.5) * x, a = T(0.5) * nu, m = T(0.5) * lam;
  const T ry = T(1) / y, h2y = T(0.5) * ry;  // loop-invariant reciprocals
  const T ly = log(y);
  const int jlo = rg.jlo, jhi = rg.jhi;
  T acc = T(0), dens = T(0), dm = T(0);  // dm: sum p_j f_j (s_j - 1), with D1
  // The recurrences multiply g_j = y^{s_j} e^{-y} / Gamma(s_j + 1) step by step,
  // so a start whose g underflows would leave every term 0.  The start is moved
  // (in log space) to the first j where g is representable; the skipped terms
  // have P (lower) or Q (upper) below that underflow level and drop out.
  if (!upper) {
    const T rm = T(1) / m;  // only used when jhi > jlo, i.e. m > 0
    int js = jhi;
    T p = rg.phi;
    T lg = (a + T(js)) * ly - y - lgamma_pos<T>(a + T(js) + T(1));
    while (lg < Ncx2Eps<T>::lg_min && js > jlo) {
      lg += log((a + T(js)) * ry);  // g_{j-1} = g_j (a + j) / y
      p *= T(js) * rm;
      --js;
    }
    T P, Q, g;
    T sj = a + T(js), jd = T(js);  // s_j and j, stepped by exact unit decrements
    gamma_pq<T>(sj, y, &P, &Q, &g, status);
    acc = p * P;
    dens = p * g * sj;  // sum p_j g_j s_j; times 1/(2y) at the end
    if (D1) dm = dens * (sj - T(1));
    for (int j = js; j > jlo; --j) {
      g *= sj * ry;  // g_{j-1} = g_j s_j / y
      P += g;        // P(s_{j-1})
      p *= jd * rm;  // p_{j-1} = p_j j / m
      sj -= T(1);
      jd -= T(1);
      acc = fma(p, P, acc);
      const T t = p * g * sj;
      dens += t;
      if (D1) dm = fma(t, sj - T(1), dm);
    }
  } else {
    int js = jlo;
    T p = rg.plo;
    T lg = (a + T(js)) * ly - y - lgamma_pos<T>(a + T(js) + T(1));
    while (lg < Ncx2Eps<T>::lg_min && js < jhi) {
      lg += ly - log(a + T(js + 1));  // g_{j+1} = g_j y / (a + j + 1)
      p *= m / T(js + 1);
      ++js;
    }
    T P, Q, g;
    T sj = a + T(js), jd = T(js);
    gamma_pq<T>(sj, y, &P, &Q, &g, status);
    acc = p * Q;
    dens = p * g * sj;
    if (D1) dm = dens * (sj - T(1));
    for (int j = js; j < jhi; ++j) {
      jd += T(1);  // j + 1
      sj += T(1);  // s_{j+1}
      // g_{j+1} = g_j y / s_{j+1} and p_{j+1} = p_j m / (j + 1), with one
      // division: d = 1 / ((j + 1) s_{j+1})
      const T d = T(1) / (jd * sj);
      Q += g;  // Q(s_{j+1})
      g *= y * jd * d;
      p *= m * sj * d;
      acc = fma(p, Q, acc);
      const T t = p * g * sj;
      dens += t;
      if (D1) dm = fma(t, sj - T(1), dm);
    }
  }
  dens *= h2y;
  *Tout = fmin(acc, T(1));
  *f = dens;
  if (D1) *fprime = dm * h2y * h2y - T(0.5) * dens;
}

// Sankaran's approximation of the quantile (Section 5.1; with sqrt(2 c2) in
// the normal term) at the normal quantile z = Phi^{-1}(u), used as the start.
template <class T = double>
AICDF_HD T ncx2_sankaran(T z, T nu, T lam) {
  const T k = nu, h0 = k + lam, h2 = k + T(2) * lam;
  const T c1 = T(1) - T(2.0 / 3.0) * h0 * (k + T(3) * lam) / (h2 * h2);
  const T c2 = h2 / (h0 * h0);
  const T c3 = (c1 - T(1)) * (T(1) - T(3) * c1);
  const T base = T(1) + c1 * c2 * (c1 - T(1) + T(0.5) * (T(2) - c1) * c2 * c3) +
                 c1 * sqrt(T(2) * c2) * (T(1) + T(0.5) * c2 * c3) * z;
  if (!(base > T(0)) || !(fabs(c1) > T(1e-3))) return h0;  // outside its range: start at the mean
  const T r = h0 * pow(base, T(1) / c1);
  return (r > T(0) && isfinite(r)) ? r : h0;
}

// The x with C(x) = target (upper = false) or 1 - C(x) = target (upper = true),
// 0 < target <= 1/2, from the start x0 (Sankaran's approximation), in the
// arithmetic T with relative tolerance tol.  Lower tail: Newton on
// ln C(e^t) - ln target in t = ln x (C behaves like x^{nu/2} near 0, so this
// converges in a few steps however deep the tail); upper tail: Newton on
// 1 - C(x) - target in x.  Both keep the iterate inside a bracket and bisect
// when Newton leaves it.
template <class T>
AICDF_HD T ncx2_solve(T target, bool upper, T x0, T nu, T lam, T tol, const Ncx2Range<T> &rg, int *status) {
  T Tv, f;
  const T big = T(1e30);
  int it = 0;
  if (!upper) {
    const T lt = log(target);
    T t = log(x0), lo = -big, hi = big;  // bracket in t = ln x
    for (; it < 100; ++it) {
      const T x = exp(t);
      ncx2_tail_pdf<T>(x, nu, lam, rg, false, &Tv, &f, status);
      T tn;
      if (!(Tv > T(0))) {  // C underflowed: x far too small
        lo = t;
        tn = hi < big ? T(0.5) * (lo + hi) : t + T(2);
      } else {
        const T r = log(Tv) - lt;  // > 0 when x is too large
        if (r > T(0)) hi = t;
        else lo = t;
        const T d = x * f / Tv;   // d ln C / d ln x
        // converged: take the last Newton step as it is (a step that rounds to
        // nothing must not meet the bracket test below, which would jump away)
        if (d > T(0) && fabs(r / d) <= tol) {
          t -= r / d;
          break;
        }
        tn = (d > T(0)) ? t - r / d : T(0.5) * (lo + hi);
        if (!(tn > lo && tn < hi)) tn = (lo > -big && hi < big) ? T(0.5) * (lo + hi) : (r > T(0) ? t - T(2) : t + T(2));
      }
      const T dt = fabs(tn - t);
      t = tn;
      if (dt <= tol || (hi - lo) <= T(0.1) * tol) break;
    }
    if (it == 100) *status |= kNcx2NoConverge;
    return exp(t);
  }
  T x = x0;
  T lo = T(0), hi = T(-1);  // hi < 0: no upper bound yet
  for (; it < 100; ++it) {
    ncx2_tail_pdf<T>(x, nu, lam, rg, true, &Tv, &f, status);
    const T r = target - Tv;  // = C(x) - u, > 0 when x is too large
    if (r > T(0)) hi = x;
    else lo = x;
    if (f > T(0) && fabs(r / f) <= tol * x) {  // converged (see the lower tail)
      x -= r / f;
      break;
    }
    T xn = (f > T(0)) ? x - r / f : T(-1);
    if (hi < T(0)) {
      if (!(xn > lo)) xn = T(2) * x + T(1);
    } else if (!(xn > lo && xn < hi)) {
      xn = T(0.5) * (lo + hi);
    }
    const T dx = fabs(xn - x);
    x = xn;
    if (dx <= tol * x || (hi > T(0) && hi - lo <= T(0.1) * tol * hi)) break;
  }
  if (it == 100) *status |= kNcx2NoConverge;
  return x;
}

// The Poisson range of a quantile at `target`: weights down to
// min(1e-20, 1e-8 target) of the probability sought.
template <class T>
AICDF_HD Ncx2Range<T> ncx2_quantile_range(T lam, T target, int *status) {
  return ncx2_range<T>(lam, fmin(T(1e-20), T(1e-8) * target), status);
}

template <class T>
AICDF_HD T ncx2_solve(T target, bool upper, T x0, T nu, T lam, T tol, int *status) {
  return ncx2_solve<T>(target, upper, x0, nu, lam, tol, ncx2_quantile_range<T>(lam, target, status), status);
}

// FP64 quantile from Sankaran's start at the normal quantile z of the same
// probability (the host table build and the device fallback).
AICDF_HD double ncx2_quantile(double target, bool upper, double z, double nu, double lam, int *status) {
  return ncx2_solve<double>(target, upper, ncx2_sankaran(z, nu, lam), nu, lam, 1e-13, status);
}

// Quantile C^{-1}_nu(u; lambda) for 0 < u < 1 (FP64 result; 1 - u is exact
// for the FP32 uniforms the paths use).  FP64 runs at 1/64 of the FP32 rate on
// this GPU, so the root is first found in FP32 (its evaluation noise leaves it
// within ~1e-5), then polished in FP64 by Halley steps on G(x) = C(x) - u:
// dx = d / (1 - d f' / (2 f)) with the Newton step d = G / f and f' from the
// same pass over the mixture.  Halley's error is cubic in the step, so a step
// with |d| <= 1e-5 x and |d f' / (2 f)| <= 1e-3 leaves ~1e-15 x plus the FP64
// evaluation's own noise: one FP64 evaluation for ~97% of calls (two or three
// otherwise), against 2.3-2.8 for Newton steps, with the same agreement with
// the full FP64 solve (<= 2e-13 relative for nu >= 0.889, host-checked on
// 20k cases per nu).  Should the FP32 phase fail (a range limit, no
// convergence; about 0.1% of calls) or the polish not settle, the full FP64
// solve runs.
__device__ __forceinline__ double ncx2_ppf(double u, double nu, double lam, int *status) {
  if (!(u > 0.0)) return 0.0;
  if (!(u < 1.0)) return __longlong_as_double(0x7ff0000000000000ll);
  const bool upper = u > 0.5;
  const double target = upper ? 1.0 - u : u;
  // the start only needs to be near the root: FP32
  const float x0 = ncx2_sankaran<float>(normcdfinvf((float)u), (float)nu, (float)lam);
  int st32 = 0;
  const Ncx2Range<float> rg32 = ncx2_quantile_range<float>((float)lam, (float)target, &st32);
  const float x32 = ncx2_solve<float>((float)target, upper, fmaxf(x0, 1e-30f), (float)nu, (float)lam, 1e-6f,
                                      rg32, &st32);
  if (st32 == 0 && x32 > 1e-30f && x32 < 1e30f) {
    // the polish sums over the FP32 phase's Poisson range (an FP32 rounding
    // at its ends moves weights of ~1e-20 of the probability), with the end
    // weights Pois(j; lambda/2) recomputed in FP64
    Ncx2Range<double> rg{rg32.jlo, rg32.jhi, 1.0, 1.0};
    if (lam > 0.0) {  // the lower tail starts from the top weight, the upper from the bottom one
      const double m = 0.5 * lam;
      const int j = upper ? rg.jlo : rg.jhi;
      const double w = exp(-m + j * log(m) - lgamma_pos<double>(j + 1.0));
      (upper ? rg.plo : rg.phi) = w;
    }
    double x = (double)x32;
    for (int k = 0; k < 3; ++k) {
      double Tv, f, fp;
      ncx2_tail_pdf<double, true>(x, nu, lam, rg, upper, &Tv, &f, status, &fp);
      if (!(f > 0.0)) break;
      const double r = upper ? target - Tv : Tv - target;  // G = C(x) - u; G' = f, G'' = f'
      const double d = r / f;
      if (!(fabs(d) <= 1e-3 * x)) break;  // not in the polish's range: fall back
      const double c = 0.5 * d * fp / f;
      x -= fabs(c) < 0.5 ? d / (1.0 - c) : d;  // far from the root: a Newton step
      if (fabs(d) <= 1e-5 * x && fabs(c) <= 1e-3) return x;
    }
  }
  return ncx2_solve<double>(target, upper, (double)x0, nu, lam, 1e-13, status);
}

}  // namespace aicdf
