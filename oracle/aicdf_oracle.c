/*
 * aicdf_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Written from the paper (Giles & Sheridan-Methven, arXiv 2012.09715) and the
 * published definitions it relies on.  Nothing here is shared with the GPU
 * library.  Only the tests, the smoke check and the benchmark's CPU baseline
 * may load it.
 *
 * Pins (checked by the CPU test suite against things other than this file):
 *   or_philox4      word-size-generic; the W=64 instance is checked against
 *                   numpy.random.Philox, an independent implementation.
 *   or_phiinv       symmetry, round trip through erfc, scipy.special.ndtri,
 *                   mpmath.
 *   or_pwc_table    the truncated values printed in the piecewise constant
 *                   listing (Section 3.2), independent quadrature, Theorem 2.1
 *                   conditions, the Corollary 2.3 tail bound.
 *   or_pwl_table    the truncated listing coefficients (Section 3.3), the
 *                   closed form of the singular interval (proof of Theorem 2.4),
 *                   mpmath quadrature of the normal equations, the Peano bound.
 *   samplers        brute force over the uniform grid near every interval edge.
 *   or_mlmc_level   exact Euler-Maruyama moments for P(X)=X, the Black-Scholes
 *                   price, the CIR mean; Milstein: the GBM step-factor moments
 *                   E[X_N^k], k <= 3, for exact and approximate variates, the
 *                   strong-order-1 decay of the two-way variance (GBM and CIR),
 *                   and the CIR mean with exact and approximate variates.
 *   or_mlmc_alloc   the speed-ups printed in Table 2 and Table 6.
 *   ncx2            lambda = 0 closed forms, moments, scipy.stats.ncx2.ppf.
 *   mlp             central finite differences.
 */
#include "aicdf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ========================================================================== */
/* Philox4xW-R (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy */
/* as 1, 2, 3", SC'11).  One round: two W x W -> 2W multiplies, the high      */
/* halves xor-ed with the other counter words and the round key; the key is   */
/* bumped by the Weyl constants between rounds.                               */
/* ========================================================================== */
static void mulhilo(int w, uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  if (w == 32) {
    uint64_t p = (a & 0xffffffffull) * (b & 0xffffffffull);
    *hi = p >> 32;
    *lo = p & 0xffffffffull;
  } else {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
  }
}

void or_philox4(int w, int rounds, const uint64_t ctr[4], const uint64_t key[2],
                uint64_t out[4]) {
  const uint64_t mask = (w == 32) ? 0xffffffffull : ~0ull;
  const uint64_t M0 = (w == 32) ? 0xD2511F53ull : 0xD2E7470EE14C6C93ull;
  const uint64_t M1 = (w == 32) ? 0xCD9E8D57ull : 0xCA5A826395121157ull;
  const uint64_t W0 = (w == 32) ? 0x9E3779B9ull : 0x9E3779B97F4A7C15ull;
  const uint64_t W1 = (w == 32) ? 0xBB67AE85ull : 0xBB67AE8584CAA73Bull;
  uint64_t c0 = ctr[0] & mask, c1 = ctr[1] & mask, c2 = ctr[2] & mask, c3 = ctr[3] & mask;
  uint64_t k0 = key[0] & mask, k1 = key[1] & mask;
  for (int r = 0; r < rounds; ++r) {
    if (r > 0) {
      k0 = (k0 + W0) & mask;
      k1 = (k1 + W1) & mask;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo(w, M0, c0, &hi0, &lo0);
    mulhilo(w, M1, c2, &hi1, &lo1);
    uint64_t n0 = (hi1 ^ c1 ^ k0) & mask;
    uint64_t n1 = lo1;
    uint64_t n2 = (hi0 ^ c3 ^ k1) & mask;
    uint64_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double or_u01(uint32_t x) {
  /* midpoint of the k-th of 2^23 equal cells: the top bit of x picks the half
   * of (0, 1) and the low 22 bits m the cell, counted from 0 in the lower half
   * and from 1 in the upper half (k = m, or k = 2^23 - 1 - m) */
  const uint32_t m = x & 0x3FFFFFu;
  const uint32_t k = (x >> 31) ? 0x7FFFFFu - m : m;
  return ((double)k + 0.5) / 8388608.0;
}

void or_uniforms(uint64_t seed, uint64_t offset, int64_t n, float *u) {
  const uint64_t key[2] = {seed & 0xffffffffull, seed >> 32};
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    uint64_t s = offset + (uint64_t)i;
    uint64_t j = s / 4;
    uint64_t ctr[4] = {j & 0xffffffffull, j >> 32, 0, 0};
    uint64_t out[4];
    or_philox4(32, 10, ctr, key, out);
    u[i] = (float)or_u01((uint32_t)out[s % 4]);
  }
}

/* Truncated-bit uniforms (Section 1, Section 2.2: a uniform carried to B bits
 * and offset to its cell midpoint).  Philox call j gives four words; each word
 * holds F = floor(32/B) B-bit fields.  Sample s of the stream is field h of
 * word t of call j with s = 4F j + 4h + t, and u = (m + 1/2) 2^-B for the
 * field value m. */
void or_uniforms_bits(uint64_t seed, uint64_t offset, int64_t n, int bits, float *u) {
  const uint64_t key[2] = {seed & 0xffffffffull, seed >> 32};
  const uint64_t F = (uint64_t)(32 / bits), per = 4 * F;
  const uint64_t mask = (1ull << bits) - 1;
  for (int64_t i = 0; i < n; ++i) {
    uint64_t s = offset + (uint64_t)i;
    uint64_t j = s / per, r = s % per, h = r / 4, t = r % 4;
    uint64_t ctr[4] = {j & 0xffffffffull, j >> 32, 0, 0};
    uint64_t out[4];
    or_philox4(32, 10, ctr, key, out);
    uint64_t m = (out[t] >> (h * (uint64_t)bits)) & mask;
    u[i] = (float)(((double)m + 0.5) / (double)(1ull << bits));
  }
}

/* ========================================================================== */
/* Gaussian: phi, Phi, and the exact inverse Phi^{-1} (Section 2)             */
/* ========================================================================== */
double or_phi(double z) { return exp(-0.5 * z * z) / sqrt(2.0 * M_PI); }

double or_Phi(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

/* F(z) - v, computed without cancellation: erfc form in the lower tail,
 * erf form near the centre (where v - 1/2 is exact). */
static double cdf_minus(double z, double v) {
  if (v < 0.25) return 0.5 * erfc(-z / sqrt(2.0)) - v;
  return 0.5 * erf(z / sqrt(2.0)) - (v - 0.5);
}

/* Phi^{-1}(v) for 0 < v <= 1/2: bisection on [-40, 0] to bracket the root to
 * ~1e-13, then Newton steps z -= (Phi(z) - v)/phi(z) until the step is below
 * 4 ulp of z. */
static double phiinv_lower(double v) {
  if (v == 0.5) return 0.0;
  double lo = -40.0, hi = 0.0;
  for (int it = 0; it < 50; ++it) {
    double mid = 0.5 * (lo + hi);
    if (cdf_minus(mid, v) > 0.0) hi = mid; else lo = mid;
  }
  double z = 0.5 * (lo + hi);
  for (int it = 0; it < 30; ++it) {
    double f = cdf_minus(z, v);
    double d = or_phi(z);
    if (d == 0.0) break;
    double step = f / d;
    double zn = z - step;
    if (zn < lo) zn = lo;
    if (zn > hi) zn = hi;
    double dz = fabs(zn - z);
    z = zn;
    if (dz <= 4.0 * 2.220446049250313e-16 * fabs(z) || dz < 1e-300) break;
  }
  return z;
}

double or_phiinv(double u) {
  if (isnan(u) || u < 0.0 || u > 1.0) return NAN;
  if (u == 0.0) return -INFINITY;
  if (u == 1.0) return INFINITY;
  if (u <= 0.5) return phiinv_lower(u);
  return -phiinv_lower(1.0 - u); /* 1 - u is exact for u in [1/2, 1] */
}

void or_phiinv_n(const float *u, int64_t n, double *z) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) z[i] = or_phiinv((double)u[i]);
}

/* ========================================================================== */
/* Piecewise constant tables (Section 2.2, Corollary 2.3)                     */
/* ========================================================================== */
int or_pwc_table(int n, int construction, double *q) {
  if (n < 2) return -1;
  for (int k = 0; k < n; ++k) {
    double ulo = (double)k / n, uhi = (double)(k + 1) / n;
    if (construction == 0) {
      /* Z^E_k = E(Z | Phi(Z) in I_k) = n * int_{z_k}^{z_{k+1}} z phi(z) dz
       *       = n * (phi(z_k) - phi(z_{k+1})), phi(+-inf) = 0. */
      double pa = (k == 0) ? 0.0 : or_phi(or_phiinv(ulo));
      double pb = (k == n - 1) ? 0.0 : or_phi(or_phiinv(uhi));
      q[k] = n * (pa - pb);
    } else if (construction == 1) {
      q[k] = or_phiinv(0.5 * (ulo + uhi)); /* Z^C: centre of the interval */
    } else if (construction == 2) {
      /* Z^I: the endpoint nearest 1/2 (inner endpoint) */
      if (ulo >= 0.5) q[k] = or_phiinv(ulo);
      else if (uhi < 0.5) q[k] = or_phiinv(uhi);
      else q[k] = 0.0; /* interval straddles 1/2 (only for n = 2): endpoint 1/2 */
    } else if (construction == 3) {
      /* Z^V: Z^E rescaled to unit variance (moment matching, Section 1); for
       * n = 2 the values are +-1, the Rademacher variables. */
      double pa = (k == 0) ? 0.0 : or_phi(or_phiinv(ulo));
      double pb = (k == n - 1) ? 0.0 : or_phi(or_phiinv(uhi));
      q[k] = n * (pa - pb);
    } else {
      return -1;
    }
  }
  if (construction == 3) {
    double m2 = 0.0;
    for (int k = 0; k < n; ++k) m2 += q[k] * q[k] / n;
    for (int k = 0; k < n; ++k) q[k] /= sqrt(m2);
  }
  return 0;
}

/* ||Q - Phi^{-1}||_2^2 = int Phi^{-1}^2 - 2 sum_k Q_k int_{I_k} Phi^{-1} + sum_k Q_k^2 / n,
 * with int_0^1 Phi^{-1}(u)^2 du = 1 and int_{I_k} Phi^{-1} = phi(z_k) - phi(z_{k+1}). */
double or_pwc_l2err2(int n, const double *q) {
  double acc = 1.0;
  for (int k = 0; k < n; ++k) {
    double pa = (k == 0) ? 0.0 : or_phi(or_phiinv((double)k / n));
    double pb = (k == n - 1) ? 0.0 : or_phi(or_phiinv((double)(k + 1) / n));
    double m0 = pa - pb;
    acc += -2.0 * q[k] * m0 + q[k] * q[k] / n;
  }
  return acc;
}

/* ========================================================================== */
/* Piecewise linear tables on geometric intervals (Section 2.3, Theorem 2.4)  */
/* I_k = [r^k/2, r^{k-1}/2) for k < K, I_K = (0, r^{K-1}/2).                 */
/* ========================================================================== */
static void pwl_interval(int k, int K, double r, double *a, double *b) {
  *b = 0.5 * pow(r, k - 1);
  *a = (k == K) ? 0.0 : 0.5 * pow(r, k);
}

/* M0 = int_a^b Phi^{-1}(u) du and M1 = int_a^b u Phi^{-1}(u) du, by the change
 * of variables u = Phi(z): int z phi = -phi, int Phi(z) z phi(z) dz =
 * -Phi phi + int phi^2, int phi^2 = Phi(sqrt2 z) / (2 sqrt(pi)). */
static void pwl_moments(double a, double b, double *M0, double *M1) {
  double za = (a == 0.0) ? -INFINITY : or_phiinv(a);
  double zb = or_phiinv(b);
  double pa = (a == 0.0) ? 0.0 : or_phi(za);
  double pb = or_phi(zb);
  double Pa2 = (a == 0.0) ? 0.0 : or_Phi(sqrt(2.0) * za);
  double Pb2 = or_Phi(sqrt(2.0) * zb);
  *M0 = pa - pb;
  *M1 = a * pa - b * pb + (Pb2 - Pa2) / (2.0 * sqrt(M_PI));
}

int or_pwl_table(int K, double r, double *alpha, double *beta) {
  if (K < 1 || !(r > 0.0 && r < 1.0)) return -1;
  alpha[0] = 0.0; /* row 0 handles u = 1/2 (Phi^{-1}(1/2) = 0) */
  beta[0] = 0.0;
  for (int k = 1; k <= K; ++k) {
    double a, b, M0, M1;
    pwl_interval(k, K, r, &a, &b);
    pwl_moments(a, b, &M0, &M1);
    /* normal equations of the L2 fit (proof of Theorem 2.4):
     *   alpha (b-a)         + beta (b^2-a^2)/2 = M0
     *   alpha (b^2-a^2)/2   + beta (b^3-a^3)/3 = M1     -- Cramer's rule */
    double s11 = b - a, s12 = 0.5 * (b * b - a * a), s22 = (b * b * b - a * a * a) / 3.0;
    double det = s11 * s22 - s12 * s12;
    alpha[k] = (M0 * s22 - M1 * s12) / det;
    beta[k] = (s11 * M1 - s12 * M0) / det;
  }
  return 0;
}

/* ||D - Phi^{-1}||_2^2 = 1 - 2 sum int D Phi^{-1} + sum int D^2, over both halves
 * (antisymmetry doubles the lower half). */
double or_pwl_l2err2(int K, double r, const double *alpha, const double *beta) {
  double cross = 0.0, sq = 0.0;
  for (int k = 1; k <= K; ++k) {
    double a, b, M0, M1;
    pwl_interval(k, K, r, &a, &b);
    pwl_moments(a, b, &M0, &M1);
    double al = alpha[k], be = beta[k];
    cross += al * M0 + be * M1;
    sq += al * al * (b - a) + al * be * (b * b - a * a) + be * be * (b * b * b - a * a * a) / 3.0;
  }
  return 1.0 - 2.0 * (2.0 * cross) + 2.0 * sq;
}

int or_pwl_index(double v, int K, double r) {
  if (v >= 0.5) return 0;
  for (int k = 1; k < K; ++k) {
    double a, b;
    pwl_interval(k, K, r, &a, &b);
    if (v >= a && v < b) return k;
  }
  return K;
}

/* ========================================================================== */
/* Piecewise polynomials on the dyadic intervals (Section 2.3, "best L2       */
/* polynomial on each interval"): normal equations in the local variable s,   */
/* moments by Gauss-Legendre quadrature.                                      */
/* ========================================================================== */
#define OR_GL 48
static void gauss_legendre(int n, double *x, double *w) {
  /* nodes on [-1, 1]: Newton on P_n from the Chebyshev-like start */
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* M_j = int_{I_k} s^j Phi^{-1}(u) du, j = 0..3 */
static void pwp_moments(int k, int K, double *M) {
  double x[OR_GL], w[OR_GL];
  gauss_legendre(OR_GL, x, w);
  for (int j = 0; j < 4; ++j) M[j] = 0.0;
  const double b = ldexp(1.0, -k);
  if (k < K) {
    const double a = 0.5 * b, h = b - a;
    for (int i = 0; i < OR_GL; ++i) {
      const double s = 0.5 * (x[i] + 1.0), u = a + h * s, f = or_phiinv(u), wi = 0.5 * w[i] * h;
      double sp = 1.0;
      for (int j = 0; j < 4; ++j) {
        M[j] += wi * sp * f;
        sp *= s;
      }
    }
  } else {
    /* singular interval: u = Phi(z), z in (-38, z_b], 16 equal panels */
    const double zb = or_phiinv(b), zl = -38.0;
    const int panels = 16;
    for (int p = 0; p < panels; ++p) {
      const double z0 = zl + (zb - zl) * p / panels, z1 = zl + (zb - zl) * (p + 1) / panels;
      for (int i = 0; i < OR_GL; ++i) {
        const double z = 0.5 * (z1 - z0) * x[i] + 0.5 * (z1 + z0);
        const double s = or_Phi(z) / b, wi = 0.5 * (z1 - z0) * w[i] * z * or_phi(z);
        double sp = 1.0;
        for (int j = 0; j < 4; ++j) {
          M[j] += wi * sp;
          sp *= s;
        }
      }
    }
  }
}

double or_pwp_table(int K, int deg, double *coef) {
  if (K < 1 || deg < 1 || deg > 3) return NAN;
  for (int i = 0; i < 4 * (K + 1); ++i) coef[i] = 0.0;
  double proj = 0.0;
  for (int k = 1; k <= K; ++k) {
    const double b = ldexp(1.0, -k);
    const double h = (k < K) ? 0.5 * b : b;
    double M[4], G[4][5];
    pwp_moments(k, K, M);
    const int n = deg + 1;
    /* Gram matrix: int_{I_k} s^i s^j du = h / (i + j + 1) */
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) G[i][j] = h / (i + j + 1.0);
      G[i][n] = M[i];
    }
    /* Gaussian elimination with partial pivoting */
    for (int c = 0; c < n; ++c) {
      int piv = c;
      for (int r = c + 1; r < n; ++r)
        if (fabs(G[r][c]) > fabs(G[piv][c])) piv = r;
      for (int j = 0; j <= n; ++j) {
        double t = G[c][j];
        G[c][j] = G[piv][j];
        G[piv][j] = t;
      }
      for (int r = c + 1; r < n; ++r) {
        double f = G[r][c] / G[c][c];
        for (int j = c; j <= n; ++j) G[r][j] -= f * G[c][j];
      }
    }
    for (int r = n - 1; r >= 0; --r) {
      double s = G[r][n];
      for (int j = r + 1; j < n; ++j) s -= G[r][j] * coef[4 * k + j];
      coef[4 * k + r] = s / G[r][r];
    }
    for (int j = 0; j < n; ++j) proj += coef[4 * k + j] * M[j];
  }
  /* projection: int D Phi^{-1} = int D^2 per interval; both halves */
  return 1.0 - 2.0 * proj;
}

/* The piecewise polynomial approximation at one uniform (NaN outside [0, 1]). */
static double pwp_value(const float *coef, int K, float uf) {
  double x = (double)uf;
  if (!(x >= 0.0 && x <= 1.0)) return NAN;
  int lower = x < 0.5;
  double v = lower ? x : 1.0 - x;
  int k = or_pwl_index(v, K, 0.5);
  double s = 0.0;
  if (k > 0) {
    const double b = ldexp(1.0, -k);
    s = (k < K) ? (v - 0.5 * b) / (0.5 * b) : v / b;
  }
  double z = 0.0;
  for (int j = 3; j >= 0; --j) z = z * s + (double)coef[4 * k + j];
  return lower ? z : -z;
}

void or_sample_pwp(const float *coef, int K, const float *u, int64_t n, double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = pwp_value(coef, K, u[i]);
}

/* ========================================================================== */
/* Samplers (Section 3.2 piecewise constant; Section 3.3 / Algorithm 1)       */
/* ========================================================================== */
/* One uniform: the value and the interval index (-1 and NaN outside [0, 1]). */
static double pwc_value(const float *table, int n_table, float uf, int32_t *m_out) {
  double x = (double)uf;
  if (!(x >= 0.0 && x <= 1.0)) {
    *m_out = -1;
    return NAN;
  }
  /* interval [m/N, (m+1)/N) containing x; x = 1 goes to the last interval */
  int m = (int)floor(x * n_table);
  if (m > n_table - 1) m = n_table - 1;
  *m_out = m;
  return (double)table[m];
}

static double pwl_value(const float *alpha, const float *beta, int K, float uf, int32_t *k_out) {
  double x = (double)uf;
  if (!(x >= 0.0 && x <= 1.0)) {
    *k_out = -1;
    return NAN;
  }
  int lower = x < 0.5;                  /* predicate                       */
  double v = lower ? x : 1.0 - x;       /* reflect about 1/2 (exact)        */
  int k = or_pwl_index(v, K, 0.5);      /* dyadic interval of v             */
  double z = (double)alpha[k] + (double)beta[k] * v;
  *k_out = k;
  return lower ? z : -z;                /* restore the sign (u=1/2 -> -0)   */
}

/* The samplers spread their independent elements over the OpenMP threads. */
void or_sample_pwc(const float *table, int n_table, const float *u, int64_t n,
                   double *out, int32_t *idx) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int32_t m;
    out[i] = pwc_value(table, n_table, u[i], &m);
    if (idx) idx[i] = m;
  }
}

void or_sample_pwl(const float *alpha, const float *beta, int K, const float *u, int64_t n,
                   double *out, int32_t *idx) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int32_t k;
    out[i] = pwl_value(alpha, beta, K, u[i], &k);
    if (idx) idx[i] = k;
  }
}

/* ========================================================================== */
/* Multilevel Monte Carlo level (Section 4: Euler-Maruyama with exact and     */
/* approximate variates from the same uniform; coarse increments are pairwise */
/* sums of the fine ones; Section 4.1 estimators).                            */
/* ========================================================================== */
static double approx_variate(const or_sde_params *prm, const float *alpha, const float *beta,
                             int K, float u) {
  int32_t k;
  if (prm->approx == OR_APPROX_PWC) return pwc_value(alpha, K, u, &k);
  if (prm->approx == OR_APPROX_PWP) return pwp_value(alpha, K, u);
  return pwl_value(alpha, beta, K, u, &k);
}

/* one step of the scheme with Brownian increment dW over time dt */
static double sde_step(const or_sde_params *p, double x, double dt, double dW) {
  if (p->model == OR_MODEL_GBM) {
    double y = x + p->mu * x * dt + p->sigma * x * dW;
    if (p->scheme == OR_SCHEME_MILSTEIN) y += 0.5 * p->sigma * p->sigma * x * (dW * dW - dt);
    return y;
  } else {
    /* CIR, truncated scheme: sqrt(x) -> sqrt(|x|) (Higham & Mao) */
    double y = x + p->kappa * (p->theta - x) * dt + p->sigma * sqrt(fabs(x)) * dW;
    if (p->scheme == OR_SCHEME_MILSTEIN) y += 0.25 * p->sigma * p->sigma * (dW * dW - dt);
    return y;
  }
}

static double payoff(const or_sde_params *p, double x) {
  if (p->payoff == OR_PAYOFF_CALL) return p->discount * (x > p->K ? x - p->K : 0.0);
  return p->discount * x;
}

static double path_value(const or_sde_params *prm, const float *alpha, const float *beta,
                         int K, int level, int kind, uint64_t p, uint64_t seed, uint32_t tag) {
  const uint64_t key[2] = {seed & 0xffffffffull, seed >> 32};
  const int64_t nf = (int64_t)1 << level;
  const double dtf = prm->T / (double)nf;
  const double sdt = sqrt(dtf);
  double xf_e = prm->X0, xc_e = prm->X0, xf_a = prm->X0, xc_a = prm->X0;
  double zc_e = 0.0, zc_a = 0.0; /* running pair sums of fine variates */
  for (int64_t s = 0; s < nf; ++s) {
    /* levels 0 and 1 use fewer than four words per path: G = 4 / 2^level
     * paths share the call of group q = p / G, path p taking words
     * (p mod G) 2^level + s; from level 2 on, path p owns its calls */
    uint64_t q = p, c = (uint64_t)(s / 4), word = (uint64_t)(s % 4);
    if (level < 2) {
      const uint64_t G = 4u >> level;
      q = p / G;
      c = 0;
      word = (p % G) * (uint64_t)nf + (uint64_t)s;
    }
    uint64_t ctr[4] = {c, q & 0xffffffffull, q >> 32, tag};
    uint64_t out[4];
    or_philox4(32, 10, ctr, key, out);
    float u = (float)or_u01((uint32_t)out[word]);
    double ze = or_phiinv((double)u);
    double za = approx_variate(prm, alpha, beta, K, u);
    xf_e = sde_step(prm, xf_e, dtf, sdt * ze);
    xf_a = sde_step(prm, xf_a, dtf, sdt * za);
    zc_e += ze;
    zc_a += za;
    if (level > 0 && (s & 1)) {
      xc_e = sde_step(prm, xc_e, 2.0 * dtf, sdt * zc_e);
      xc_a = sde_step(prm, xc_a, 2.0 * dtf, sdt * zc_a);
      zc_e = 0.0;
      zc_a = 0.0;
    }
  }
  double pf_e = payoff(prm, xf_e), pf_a = payoff(prm, xf_a);
  double pc_e = level > 0 ? payoff(prm, xc_e) : 0.0; /* P_{-1} := 0 */
  double pc_a = level > 0 ? payoff(prm, xc_a) : 0.0;
  switch (kind) {
    case OR_KIND_APPROX2: return pf_a - pc_a;
    case OR_KIND_CORR4: return pf_e - pc_e - pf_a + pc_a;
    case OR_KIND_EXACT2: return pf_e - pc_e;
    case OR_KIND_PLAIN: return pf_e;
    case OR_KIND_PLAIN_APPROX: return pf_a;
    default: return NAN;
  }
}

void or_mlmc_paths(const or_sde_params *prm, const float *alpha, const float *beta, int K,
                   int level, int kind, uint64_t n_paths, uint64_t path_offset,
                   uint64_t seed, uint32_t tag, double *y) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < (int64_t)n_paths; ++i)
    y[i] = path_value(prm, alpha, beta, K, level, kind, path_offset + (uint64_t)i, seed, tag);
}

void or_mlmc_level(const or_sde_params *prm, const float *alpha, const float *beta, int K,
                   int level, int kind, uint64_t n_paths, uint64_t path_offset,
                   uint64_t seed, uint32_t tag, double sums[5]) {
  double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : s1, s2, s3, s4)
  for (int64_t i = 0; i < (int64_t)n_paths; ++i) {
    double y = path_value(prm, alpha, beta, K, level, kind, path_offset + (uint64_t)i, seed, tag);
    s1 += y;
    s2 += y * y;
    s3 += y * y * y;
    s4 += y * y * y * y;
  }
  sums[0] = s1;
  sums[1] = s2;
  sums[2] = s3;
  sums[3] = s4;
  sums[4] = (double)n_paths;
}

/* ========================================================================== */
/* Cost model (Section 4.1): Lagrange-optimal path counts for a set of        */
/* estimator terms with variances v and costs c; returns total time T.        */
/* ========================================================================== */
double or_mlmc_alloc(int nterms, const double *v, const double *c, double eps, double *m) {
  double s = 0.0;
  for (int i = 0; i < nterms; ++i) s += sqrt(v[i] * c[i]);
  double T = 2.0 / (eps * eps) * s * s;
  for (int i = 0; i < nterms; ++i) m[i] = sqrt(2.0 * T * v[i] / c[i]) / eps;
  return T;
}

/* ========================================================================== */
/* Non-central chi-squared (Section 5): CDF as a Poisson mixture of central   */
/* chi-squared CDFs (Abramowitz & Stegun 26.4.25); quantile by root finding.  */
/* ========================================================================== */
/* regularised lower incomplete gamma P(a, x): series for x < a + 1, else the
 * continued fraction for Q = 1 - P (modified Lentz). */
double or_gammp(double a, double x) {
  if (x <= 0.0) return 0.0;
  if (isinf(x)) return 1.0;
  double lpre = -x + a * log(x) - lgamma(a);
  if (x < a + 1.0) {
    double ap = a, del = 1.0 / a, sum = del;
    for (int n = 0; n < 100000; ++n) {
      ap += 1.0;
      del *= x / ap;
      sum += del;
      if (fabs(del) < fabs(sum) * 1e-17) break;
    }
    return sum * exp(lpre);
  } else {
    const double tiny = 1e-300;
    double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, h = d;
    for (int i = 1; i < 100000; ++i) {
      double an = -i * (i - a);
      b += 2.0;
      d = an * d + b;
      if (fabs(d) < tiny) d = tiny;
      c = b + an / c;
      if (fabs(c) < tiny) c = tiny;
      d = 1.0 / d;
      double del = d * c;
      h *= del;
      if (fabs(del - 1.0) < 1e-17) break;
    }
    return 1.0 - exp(lpre) * h;
  }
}

static double pois_logw(int64_t j, double m) { /* log of e^{-m} m^j / j! */
  if (m == 0.0) return j == 0 ? 0.0 : -INFINITY;
  return -m + (double)j * log(m) - lgamma((double)j + 1.0);
}

/* regularised upper incomplete gamma Q(a, x) = 1 - P(a, x), computed
 * directly from the continued fraction for x >= a + 1 (no cancellation in
 * the upper tail) */
static double gammq(double a, double x) {
  if (x <= 0.0) return 1.0;
  if (isinf(x)) return 0.0;
  if (x < a + 1.0) return 1.0 - or_gammp(a, x);
  const double lpre = -x + a * log(x) - lgamma(a), tiny = 1e-300;
  double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, h = d;
  for (int i = 1; i < 100000; ++i) {
    double an = -i * (i - a);
    b += 2.0;
    d = an * d + b;
    if (fabs(d) < tiny) d = tiny;
    c = b + an / c;
    if (fabs(c) < tiny) c = tiny;
    d = 1.0 / d;
    double del = d * c;
    h *= del;
    if (fabs(del - 1.0) < 1e-17) break;
  }
  return exp(lpre) * h;
}

/* sum over j of Pois(j; lam/2) * f(j), outward from the mode; f = CDF (0),
 * density (1) or upper tail (2) of the central chi^2 with nu + 2j degrees of
 * freedom.  f <= 1 for the CDF and the tail, and the density is <= 1/2 for
 * nu + 2j >= 2, so a side is cut once its Poisson weight is below 1e-17 of
 * the running sum (the neglected terms then sum to about 1e-17 relative,
 * however small the sum itself is); for nu < 2 the j = 0 density, unbounded
 * near x = 0, is always added. */
static double ncx2_f(double x, double a, int pdf) {
  if (pdf == 1) return (x <= 0.0) ? 0.0 : exp((a - 1.0) * log(0.5 * x) - 0.5 * x - lgamma(a)) * 0.5;
  if (pdf == 2) return gammq(a, 0.5 * x);
  return or_gammp(a, 0.5 * x);
}

static double ncx2_mix(double x, double nu, double lam, int pdf) {
  double m = 0.5 * lam;
  int64_t j0 = (int64_t)floor(m);
  double total = 0.0;
  for (int64_t j = j0;; ++j) {           /* upward from the mode */
    double w = exp(pois_logw(j, m));
    total += w * ncx2_f(x, 0.5 * nu + (double)j, pdf);
    if (w == 0.0 || w < 1e-17 * total) break;
    if (j > j0 + 100000000) break;
  }
  for (int64_t j = j0 - 1; j >= 0; --j) { /* downward to 0 */
    double w = exp(pois_logw(j, m));
    total += w * ncx2_f(x, 0.5 * nu + (double)j, pdf);
    if ((w == 0.0 || w < 1e-17 * total) && j > 0) {
      if (pdf == 1 && nu < 2.0) total += exp(pois_logw(0, m)) * ncx2_f(x, 0.5 * nu, pdf);
      break;
    }
  }
  return total;
}

double or_ncx2_cdf(double x, double nu, double lam) {
  if (x <= 0.0) return 0.0;
  return ncx2_mix(x, nu, lam, 0);
}

double or_ncx2_pdf(double x, double nu, double lam) {
  if (x <= 0.0) return 0.0;
  return ncx2_mix(x, nu, lam, 1);
}

/* quantile: bracket [lo, hi] with F(lo) <= u <= F(hi), then Newton steps kept
 * inside the bracket (bisection when Newton leaves it), to 1e-14 relative. */
double or_ncx2_ppf(double u, double nu, double lam) {
  if (isnan(u) || u < 0.0 || u > 1.0) return NAN;
  if (u == 0.0) return 0.0;
  if (u == 1.0) return INFINITY;
  double mean = nu + lam, sd = sqrt(2.0 * (nu + 2.0 * lam));
  double lo = 0.0, hi = mean + 10.0 * sd;
  while (or_ncx2_cdf(hi, nu, lam) < u && hi < 1e300) { lo = hi; hi *= 2.0; }
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 500; ++it) {
    double F = or_ncx2_cdf(x, nu, lam) - u;
    if (F > 0.0) hi = x; else lo = x;
    double f = or_ncx2_pdf(x, nu, lam);
    double xn = (f > 0.0) ? x - F / f : 0.5 * (lo + hi);
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    double dx = fabs(xn - x);
    x = xn;
    if (dx <= 1e-14 * fabs(x) || hi - lo <= 1e-15 * fabs(x)) break;
  }
  return x;
}

double or_ncx2_sf(double x, double nu, double lam) {
  if (x <= 0.0) return 1.0;
  return ncx2_mix(x, nu, lam, 2);
}

/* upper-tail quantile: the x with 1 - F(x) = v, solved on the upper tail
 * itself so that v down to the smallest doubles keeps full relative accuracy */
double or_ncx2_isf(double v, double nu, double lam) {
  if (isnan(v) || v < 0.0 || v > 1.0) return NAN;
  if (v == 0.0) return INFINITY;
  if (v == 1.0) return 0.0;
  double mean = nu + lam, sd = sqrt(2.0 * (nu + 2.0 * lam));
  double lo = 0.0, hi = mean + 10.0 * sd;
  while (or_ncx2_sf(hi, nu, lam) > v && hi < 1e300) { lo = hi; hi *= 2.0; }
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 500; ++it) {
    double G = or_ncx2_sf(x, nu, lam) - v;   /* decreasing in x */
    if (G < 0.0) hi = x; else lo = x;
    double f = or_ncx2_pdf(x, nu, lam);
    double xn = (f > 0.0) ? x + G / f : 0.5 * (lo + hi);
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    double dx = fabs(xn - x);
    x = xn;
    if (dx <= 1e-14 * fabs(x) || hi - lo <= 1e-15 * fabs(x)) break;
  }
  return x;
}

/* P_x(U; y) = sqrt(x / 4y) ( (y/x) C^{-1}_x(U; (1-y)x/y) - 1 )  (Section 5.1) */
double or_ncx2_P(double u, double x, double y) {
  double lam = (1.0 - y) * x / y;
  double c = or_ncx2_ppf(u, x, lam);
  return sqrt(x / (4.0 * y)) * ((y / x) * c - 1.0);
}

/* ========================================================================== */
/* Section 5.1: piecewise polynomial approximation of P_nu(.; y).  Knots y_i  */
/* with sqrt(y_i) = i/(n-1) equally spaced (y_0 = 0: the Gaussian limit       */
/* Phi^{-1}; y_{n-1} = 1: the central chi^2 limit), separate fits on the two   */
/* halves u <= 1/2 and u > 1/2 (the law is not antisymmetric), K dyadic       */
/* intervals per half in v = min(u, 1-u), the L2-optimal polynomial of degree */
/* deg in the local variable s on each; linear interpolation between knots   */
/* in sqrt(y).  Row 0 of each half holds the value at u = 1/2.               */
/* ========================================================================== */
/* P_nu(u; y) at u = v (lower half) or u = 1 - v (upper half) */
static double ncx2_half_P(double v, int upper, double nu, double y) {
  if (y <= 0.0) return upper ? -or_phiinv(v) : or_phiinv(v);
  if (!upper) return or_ncx2_P(v, nu, y);
  const double c = or_ncx2_isf(v, nu, (1.0 - y) * nu / y);
  return sqrt(nu / (4.0 * y)) * ((y / nu) * c - 1.0);
}

/* int_{I_k} s^j g(v) dv, j = 0..3, for g = P on one half.  Regular intervals:
 * 24-point Gauss-Legendre; the singular interval (0, 2^-K): 40 geometric
 * panels [b 2^-(p+1), b 2^-p] of 8 points (the rest, below b 2^-40, is
 * dropped: |P| grows at most logarithmically there). */
#define NCX2_GL 24
#define NCX2_GLS 8
#define NCX2_PANELS 40
static void ncx2_moments(int k, int K, int upper, double nu, double y, double *M) {
  double x[NCX2_GL], w[NCX2_GL], xs[NCX2_GLS], ws[NCX2_GLS];
  gauss_legendre(NCX2_GL, x, w);
  gauss_legendre(NCX2_GLS, xs, ws);
  for (int j = 0; j < 4; ++j) M[j] = 0.0;
  const double b = ldexp(1.0, -k);
  const int np = (k < K) ? 1 : NCX2_PANELS, nq = (k < K) ? NCX2_GL : NCX2_GLS;
  for (int p = 0; p < np; ++p) {
    const double hi = (k < K) ? b : ldexp(b, -p), lo = 0.5 * hi, h = hi - lo;
    for (int i = 0; i < nq; ++i) {
      const double xi = (k < K) ? x[i] : xs[i], wi = 0.5 * ((k < K) ? w[i] : ws[i]) * h;
      const double v = lo + 0.5 * (xi + 1.0) * h;
      const double s = (k < K) ? (v - lo) / h : v / b;
      const double f = ncx2_half_P(v, upper, nu, y);
      double sp = 1.0;
      for (int j = 0; j < 4; ++j) {
        M[j] += wi * sp * f;
        sp *= s;
      }
    }
  }
}

/* L2 fit of degree deg on interval k from the moments (Gram h/(i+j+1)) */
static void poly_fit(int k, int K, int deg, const double *M, double *c) {
  const double b = ldexp(1.0, -k), h = (k < K) ? 0.5 * b : b;
  const int n = deg + 1;
  double G[4][5];
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) G[i][j] = h / (i + j + 1.0);
    G[i][n] = M[i];
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(G[r][col]) > fabs(G[piv][col])) piv = r;
    for (int j = 0; j <= n; ++j) {
      double t = G[col][j];
      G[col][j] = G[piv][j];
      G[piv][j] = t;
    }
    for (int r = col + 1; r < n; ++r) {
      double f = G[r][col] / G[col][col];
      for (int j = col; j <= n; ++j) G[r][j] -= f * G[col][j];
    }
  }
  for (int j = 0; j < 4; ++j) c[j] = 0.0;
  for (int r = n - 1; r >= 0; --r) {
    double acc = G[r][n];
    for (int j = r + 1; j < n; ++j) acc -= G[r][j] * c[j];
    c[r] = acc / G[r][r];
  }
}

int or_ncx2_poly_table(double nu, int K, int n_knots, int deg, double *coef) {
  if (!(nu > 0.0) || K < 1 || K > 31 || n_knots < 2 || deg < 1 || deg > 3) return -1;
  /* every (knot, half, interval) fit is independent */
  const int nfit = n_knots * 2 * (K + 1);
#pragma omp parallel for schedule(dynamic, 1)
  for (int f = 0; f < nfit; ++f) {
    const int k = f % (K + 1), half = (f / (K + 1)) % 2, i = f / (2 * (K + 1));
    const double r = (double)i / (n_knots - 1), y = r * r;
    double *c = coef + (size_t)f * 4;
    if (k == 0) {
      c[0] = ncx2_half_P(0.5, 0, nu, y);
      c[1] = c[2] = c[3] = 0.0;
    } else {
      double M[4];
      ncx2_moments(k, K, half, nu, y, M);
      poly_fit(k, K, deg, M, c);
    }
  }
  return 0;
}

/* P~_nu(u; y) from a table (coef as laid out by or_ncx2_poly_table) */
double or_ncx2_poly_P(const double *coef, int K, int n_knots, double u, double y) {
  const int upper = u > 0.5;
  const double v = upper ? 1.0 - u : u;
  const int k = or_pwl_index(v, K, 0.5);
  double s = 0.0;
  if (k > 0) {
    const double b = ldexp(1.0, -k);
    s = (k < K) ? (v - 0.5 * b) / (0.5 * b) : v / b;
  }
  double t = sqrt(y) * (n_knots - 1);
  int i = (int)floor(t);
  if (i > n_knots - 2) i = n_knots - 2;
  if (i < 0) i = 0;
  const double f = t - i;
  double p[2];
  for (int q = 0; q < 2; ++q) {
    const double *c = coef + (size_t)(((i + q) * 2 + upper) * (K + 1) + k) * 4;
    p[q] = ((c[3] * s + c[2]) * s + c[1]) * s + c[0];
  }
  return (1.0 - f) * p[0] + f * p[1];
}

/* C~^{-1}_nu(u; lambda) = lambda + nu + 2 sqrt(lambda + nu) P~_nu(u; nu/(lambda + nu)) */
double or_ncx2_poly_ppf(const double *coef, double nu, int K, int n_knots, double u, double lam) {
  const double h = lam + nu;
  return h + 2.0 * sqrt(h) * or_ncx2_poly_P(coef, K, n_knots, u, nu / h);
}

/* RMSE sqrt(int_0^1 (C~^{-1} - C^{-1})^2 du) by the same quadrature as the fit
 * (each half, each dyadic interval, the singular ones on geometric panels). */
double or_ncx2_poly_rmse(const double *coef, double nu, int K, int n_knots, double lam) {
  double x[NCX2_GL], w[NCX2_GL], xs[NCX2_GLS], ws[NCX2_GLS];
  gauss_legendre(NCX2_GL, x, w);
  gauss_legendre(NCX2_GLS, xs, ws);
  double acc = 0.0;
  const int nseg = 2 * (K - 1 + NCX2_PANELS);  /* per half: K-1 regular intervals + panels */
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : acc)
  for (int g = 0; g < nseg; ++g) {
    const int half = g / (nseg / 2), r = g % (nseg / 2);
    const int k = (r < K - 1) ? r + 1 : K, p = (r < K - 1) ? 0 : r - (K - 1);
    const double b = ldexp(1.0, -k);
    const double hi = (k < K) ? b : ldexp(b, -p), lo = 0.5 * hi, h = hi - lo;
    const int nq = (k < K) ? NCX2_GL : NCX2_GLS;
    for (int i = 0; i < nq; ++i) {
      const double xi = (k < K) ? x[i] : xs[i], wi = 0.5 * ((k < K) ? w[i] : ws[i]) * h;
      const double v = lo + 0.5 * (xi + 1.0) * h, u = half ? 1.0 - v : v;
      const double ex = half ? or_ncx2_isf(v, nu, lam) : or_ncx2_ppf(v, nu, lam);
      const double d = or_ncx2_poly_ppf(coef, nu, K, n_knots, u, lam) - ex;
      acc += wi * d * d;
    }
  }
  return sqrt(acc);
}

/* ========================================================================== */
/* MLP surrogate reference: y = w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3       */
/* ========================================================================== */
void or_mlp_forward(int H, const double *W1, const double *b1, const double *W2,
                    const double *b2, const double *w3, const double *b3,
                    const double *x, int64_t n, double *y) {
  double *h1 = (double *)malloc(sizeof(double) * H);
  double *h2 = (double *)malloc(sizeof(double) * H);
  for (int64_t i = 0; i < n; ++i) {
    for (int j = 0; j < H; ++j)
      h1[j] = tanh(W1[2 * j] * x[2 * i] + W1[2 * j + 1] * x[2 * i + 1] + b1[j]);
    for (int j = 0; j < H; ++j) {
      double s = b2[j];
      for (int k = 0; k < H; ++k) s += W2[j * H + k] * h1[k];
      h2[j] = tanh(s);
    }
    double o = b3[0];
    for (int j = 0; j < H; ++j) o += w3[j] * h2[j];
    y[i] = o;
  }
  free(h1);
  free(h2);
}

double or_mlp_grad(int H, const double *W1, const double *b1, const double *W2,
                   const double *b2, const double *w3, const double *b3,
                   const double *x, const double *t, int64_t n,
                   double *gW1, double *gb1, double *gW2, double *gb2, double *gw3,
                   double *gb3) {
  memset(gW1, 0, sizeof(double) * 2 * H);
  memset(gb1, 0, sizeof(double) * H);
  memset(gW2, 0, sizeof(double) * H * H);
  memset(gb2, 0, sizeof(double) * H);
  memset(gw3, 0, sizeof(double) * H);
  gb3[0] = 0.0;
  double *h1 = (double *)malloc(sizeof(double) * H);
  double *h2 = (double *)malloc(sizeof(double) * H);
  double *d2 = (double *)malloc(sizeof(double) * H);
  double loss = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double x0 = x[2 * i], x1 = x[2 * i + 1];
    for (int j = 0; j < H; ++j) h1[j] = tanh(W1[2 * j] * x0 + W1[2 * j + 1] * x1 + b1[j]);
    for (int j = 0; j < H; ++j) {
      double s = b2[j];
      for (int k = 0; k < H; ++k) s += W2[j * H + k] * h1[k];
      h2[j] = tanh(s);
    }
    double o = b3[0];
    for (int j = 0; j < H; ++j) o += w3[j] * h2[j];
    double e = o - t[i];
    loss += e * e;
    double dout = 2.0 * e / (double)n; /* d(mean sq)/d out */
    gb3[0] += dout;
    for (int j = 0; j < H; ++j) {
      gw3[j] += dout * h2[j];
      d2[j] = dout * w3[j] * (1.0 - h2[j] * h2[j]);
      gb2[j] += d2[j];
    }
    for (int j = 0; j < H; ++j)
      for (int k = 0; k < H; ++k) gW2[j * H + k] += d2[j] * h1[k];
    for (int k = 0; k < H; ++k) {
      double s = 0.0;
      for (int j = 0; j < H; ++j) s += W2[j * H + k] * d2[j];
      double d1 = s * (1.0 - h1[k] * h1[k]);
      gb1[k] += d1;
      gW1[2 * k] += d1 * x0;
      gW1[2 * k + 1] += d1 * x1;
    }
  }
  free(h1);
  free(h2);
  free(d2);
  return loss / (double)n;
}
