/*
 * aicdf_oracle.h -- plain, slow, FP64 CPU oracle for the approximate
 * inverse-CDF method of Giles & Sheridan-Methven, "Approximating inverse
 * cumulative distribution functions to produce approximate random variables".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The GPU library shares
 * no code, header, table or constant generator with it.
 *
 * Every function cites the section / equation / algorithm of the paper it
 * follows.  Floating point is FP64 unless the paper fixes the precision (the
 * samplers take FP32 uniforms and FP32-rounded coefficients, as the paper's
 * single precision implementation does, but do their arithmetic in FP64).
 *
 * Parity status per function is listed in the header of aicdf_oracle.c.
 */
#ifndef AICDF_ORACLE_H
#define AICDF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- uniforms: Philox4xW-R (Salmon et al., SC'11), W in {32, 64} ---------- */
void or_philox4(int wbits, int rounds, const uint64_t ctr[4], const uint64_t key[2],
                uint64_t out[4]);
/* u = (2*(x & 0x7FFFFF)+1) * 2^-24 : 2^23-point midpoint grid, open and symmetric. */
double or_u01(uint32_t x);
/* Standalone sampling stream: sample i uses Philox call j=(offset+i)/4 with
 * ctr=(j mod 2^32, j>>32, 0, 0), key=(seed mod 2^32, seed>>32), word (offset+i)%4. */
void or_uniforms(uint64_t seed, uint64_t offset, int64_t n, float *u);
/* Truncated-bit stream, B = bits in [1, 23]: F = floor(32/B) fields per word;
 * sample s = 4F j + 4h + t is field h (bits hB..hB+B-1) of word t of call j
 * (counter and key as above); u = (m + 1/2) 2^-B. */
void or_uniforms_bits(uint64_t seed, uint64_t offset, int64_t n, int bits, float *u);

/* ---- Gaussian ---------------------------------------------------------------- */
double or_phi(double z);            /* density */
double or_Phi(double z);            /* CDF     */
double or_phiinv(double u);         /* exact inverse CDF: bisection + Newton on erfc */
void   or_phiinv_n(const float *u, int64_t n, double *z);

/* ---- tables (Section 2.2, Corollary 2.3; Section 2.3, Theorem 2.4) --------- */
/* construction: 0 = conditional mean Z^E, 1 = centre Z^C, 2 = inner endpoint Z^I,
 * 3 = Z^E rescaled to unit variance (n = 2: Rademacher +-1) */
int    or_pwc_table(int n, int construction, double *q);
double or_pwc_l2err2(int n, const double *q);          /* ||Q - Phi^-1||_2^2 */
/* K intervals with decay rate r; alpha/beta get K+1 rows, row 0 = (0,0). */
int    or_pwl_table(int K, double r, double *alpha, double *beta);
double or_pwl_l2err2(int K, double r, const double *alpha, const double *beta);
/* interval index of v in (0,1/2] for decay rate r (0 for v = 1/2) */
int    or_pwl_index(double v, int K, double r);

/* Piecewise polynomials of degree deg (1..3) on the K dyadic intervals of
 * (0, 1/2) (Section 2.3: the best L2 polynomial on each interval), in the
 * local variable s in [0, 1): s = (v - a)/(b - a) on I_k = [a, b), k < K, and
 * s = v / b on I_K = (0, b).  coef[4 k + j] multiplies s^j (rows 1..K; row 0
 * zero, unused coefficients zero).  Returns ||D - Phi^{-1}||_2^2 over (0, 1). */
double or_pwp_table(int K, int deg, double *coef);
void or_sample_pwp(const float *coef, int K, const float *u, int64_t n, double *out);

/* ---- samplers (Section 3.2 listing semantics; Algorithm 1) ---------------- */
void or_sample_pwc(const float *table, int n_table, const float *u, int64_t n,
                   double *out, int32_t *idx);
void or_sample_pwl(const float *alpha, const float *beta, int K, const float *u,
                   int64_t n, double *out, int32_t *idx);

/* ---- multilevel Monte Carlo level (Section 4, Section 4.1) ---------------- */
enum { OR_KIND_APPROX2 = 0, OR_KIND_CORR4 = 1, OR_KIND_EXACT2 = 2, OR_KIND_PLAIN = 3,
       OR_KIND_PLAIN_APPROX = 4 };
enum { OR_MODEL_GBM = 0, OR_MODEL_CIR = 1 };
enum { OR_SCHEME_EM = 0, OR_SCHEME_MILSTEIN = 1 };
enum { OR_PAYOFF_X = 0, OR_PAYOFF_CALL = 1 };
enum { OR_APPROX_PWL = 0, OR_APPROX_PWC = 1, OR_APPROX_PWP = 2 };

typedef struct {
  int model, scheme, payoff, approx;
  double X0, T, K;        /* initial value, horizon, strike               */
  double mu, sigma;       /* GBM: drift, volatility                       */
  double kappa, theta;    /* CIR: mean reversion rate, level (sigma above) */
  double discount;        /* payoff multiplier, e.g. exp(-rT)             */
} or_sde_params;

/* Power sums over paths p = path_offset .. path_offset+n_paths-1 of Y for the
 * level estimator of the given kind (Section 4.1: sample mean and variance,
 * plus the third and fourth power sums behind the kurtosis).
 * sums = {sum Y, sum Y^2, sum Y^3, sum Y^4, n}.
 * Uniform for fine step s of path p: Philox4x32-10 with key = (seed mod 2^32,
 * seed>>32); for level >= 2, ctr = (s/4, p mod 2^32, p>>32, tag) and word s%4;
 * for levels 0 and 1 (2^level < 4 fine steps) G = 4/2^level paths share one
 * call: ctr = (0, q mod 2^32, q>>32, tag) with q = p/G, word (p mod G) 2^level + s.
 * approx tables: PWL (alpha, beta, K), PWC (alpha = table, K = n_table) or
 * PWP (alpha = (K+1) x 4 polynomial coefficients, K). */
void or_mlmc_level(const or_sde_params *prm, const float *alpha, const float *beta, int K,
                   int level, int kind, uint64_t n_paths, uint64_t path_offset,
                   uint64_t seed, uint32_t tag, double sums[5]);
/* single path values (for tests): writes Y of each path */
void or_mlmc_paths(const or_sde_params *prm, const float *alpha, const float *beta, int K,
                   int level, int kind, uint64_t n_paths, uint64_t path_offset,
                   uint64_t seed, uint32_t tag, double *y);

/* ---- cost model (Section 4.1) --------------------------------------------- */
/* Optimal path counts m_l = eps^-1 sqrt(2 T v_l / c_l), T = 2 eps^-2 (sum sqrt(v c))^2 */
double or_mlmc_alloc(int nterms, const double *v, const double *c, double eps, double *m);

/* ---- non-central chi-squared (Section 5) ---------------------------------- */
double or_gammp(double a, double x);                     /* regularised lower gamma */
double or_ncx2_cdf(double x, double nu, double lam);
double or_ncx2_pdf(double x, double nu, double lam);
double or_ncx2_ppf(double u, double nu, double lam);     /* root finding on the CDF */
double or_ncx2_sf(double x, double nu, double lam);      /* 1 - CDF, summed directly */
double or_ncx2_isf(double v, double nu, double lam);     /* x with 1 - CDF(x) = v */
/* P_x(U; y) of Section 5.1 and its inverse map C^{-1}_nu(U; lambda) */
double or_ncx2_P(double u, double x, double y);
/* Section 5.1 piecewise polynomial approximation of P_nu(.; y): n_knots knots
 * with sqrt(y) equally spaced on [0, 1], two halves, K dyadic intervals per
 * half (v = min(u, 1-u)), L2 polynomial of degree deg in the local variable s.
 * coef[(((i*2 + half)*(K+1)) + k)*4 + j] multiplies s^j (half 1: u > 1/2);
 * row 0 of each half = [P(1/2; y_i), 0, 0, 0]. */
int    or_ncx2_poly_table(double nu, int K, int n_knots, int deg, double *coef);
double or_ncx2_poly_P(const double *coef, int K, int n_knots, double u, double y);
double or_ncx2_poly_ppf(const double *coef, double nu, int K, int n_knots, double u, double lam);
double or_ncx2_poly_rmse(const double *coef, double nu, int K, int n_knots, double lam);

/* ---- MLP surrogate 2 -> H -> H -> 1, tanh (FP64 reference) ----------------- */
/* weights: W1[H][2], b1[H], W2[H][H], b2[H], w3[H], b3[1] (row-major, out x in) */
void or_mlp_forward(int H, const double *W1, const double *b1, const double *W2,
                    const double *b2, const double *w3, const double *b3,
                    const double *x /* n x 2 */, int64_t n, double *y);
/* gradient of L = mean_i (y_i - t_i)^2 with respect to all parameters;
 * returns L.  grads laid out like the weights. */
double or_mlp_grad(int H, const double *W1, const double *b1, const double *W2,
                   const double *b2, const double *w3, const double *b3,
                   const double *x, const double *t, int64_t n,
                   double *gW1, double *gb1, double *gW2, double *gb2, double *gw3,
                   double *gb3);

#ifdef __cplusplus
}
#endif
#endif
