/*
 * aicdf.h -- C ABI of libaicdf, a GB300 (sm_103a) library for approximate
 * random variables produced from cheap approximations to the inverse
 * cumulative distribution function, after Giles & Sheridan-Methven,
 * "Approximating inverse cumulative distribution functions to produce
 * approximate random variables" (arXiv 2012.09715).
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are device pointers; *_host are host pointers.
 *     The caller owns every buffer and stream; the library owns handles.
 *   - Calls that take a stream are asynchronous on it unless stated.
 *   - Errors are returned as aicdf_status; nothing throws across the ABI.
 *     Arguments are checked before anything is launched.  A CUDA error from a
 *     launch is reported as AICDF_ERR_CUDA (aicdf_last_cuda_error() gives the
 *     cudaError_t value).
 *   - Uniforms.  Where the library draws uniforms itself it uses
 *     Philox4x32-10 (Salmon et al., SC'11) with key (seed mod 2^32, seed>>32)
 *     and maps a 32-bit word x to the midpoint u = (2k+1) * 2^-24 of one of
 *     2^23 equal cells: with m = x mod 2^22 (its low 22 bits), k = m when bit
 *     31 is clear (u < 1/2) and k = 2^23 - 1 - m when it is set (u > 1/2);
 *     bits 22..30 are unused.  u lies in [2^-24, 1-2^-24], is never 1/2, and
 *     u and 1-u are both exact in FP32.
 */
#ifndef AICDF_H
#define AICDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (binary compatible with cudaStream_t); NULL = legacy stream. */
typedef struct CUstream_st *aicdf_stream_t;

typedef enum {
  AICDF_OK = 0,
  AICDF_ERR_ARG = 1,          /* bad argument (null, size, alignment, range)   */
  AICDF_ERR_CUDA = 2,         /* a CUDA runtime call or launch failed          */
  AICDF_ERR_NOCONVERGE = 3,   /* an iteration hit its cap                      */
  AICDF_ERR_DOMAIN = 4,       /* parameters outside the model's domain         */
  AICDF_ERR_STATE = 5,        /* handle in the wrong state                     */
  AICDF_ERR_NOMEM = 6,        /* host allocation failed                        */
  AICDF_ERR_UNSUPPORTED = 7   /* valid request that this build does not serve  */
} aicdf_status;

const char *aicdf_status_str(aicdf_status s);
int aicdf_last_cuda_error(void);
/* Library version as major*10000 + minor*100 + patch. */
int aicdf_version(void);

/* ===================================================================== */
/* Approximation tables (host objects; built in FP64)                     */
/* ===================================================================== */
typedef enum {
  AICDF_PWC = 0, AICDF_PWL = 1, AICDF_EXACT = 2, AICDF_EXACT_LIB = 3, AICDF_PWP = 4
} aicdf_method;
typedef enum { AICDF_Z_E = 0, AICDF_Z_C = 1, AICDF_Z_I = 2, AICDF_Z_V = 3 } aicdf_construction;
typedef struct aicdf_table_s *aicdf_table;

/* Build an approximation table on the host in FP64.
 *
 * AICDF_PWC (Section 2.2, Theorem 2.1, Corollary 2.3): n equal intervals
 *   [m/n, (m+1)/n), n a power of two in [2, 4096]; constants by construction
 *   Z^E (conditional mean E(Z | Phi(Z) in I_m), the paper's choice),
 *   Z^C (Phi^{-1} of the interval centre), Z^I (the endpoint nearest 1/2)
 *   or Z^V (Z^E rescaled to unit mean square, a moment-matched variant as in
 *   Section 1; n = 2 gives the Rademacher values -1, +1).
 * AICDF_PWL (Section 2.3, Theorem 2.4 with the dyadic rate r = 1/2,
 *   Section 3.3): n = K intervals in (0, 1/2), I_k = [2^-(k+1), 2^-k) for
 *   k < K and I_K = (0, 2^-K), K in [1, 31]; each line is the L2-optimal fit
 *   on its interval (the normal equations of the proof of Theorem 2.4).  The
 *   table holds K+1 rows; row 0 is zero so that u = 1/2 maps to 0 (Section
 *   3.3).  construction must be AICDF_Z_E (ignored).
 * AICDF_PWP (Section 2.3, the piecewise polynomial generalisation; Fig. 2
 *   uses cubics): n = K dyadic intervals as for PWL, construction = the
 *   degree d in 1..3; on each interval the L2-optimal polynomial of degree d
 *   in the local variable s in [0, 1): s = (v - a)/(b - a) on I_k = [a, b),
 *   k < K (the fraction of v's FP32 significand), and s = v / b on I_K = (0, b).
 *   The table holds K+1 rows of 4 coefficients (powers s^0..s^3; row 0 and the
 *   powers above d are zero).
 * On success *out owns the table; release it with aicdf_table_destroy. */
aicdf_status aicdf_table_build(int method, int n, int construction, aicdf_table *out);
void aicdf_table_destroy(aicdf_table t);
/* Copy the FP64 coefficients to the host.  PWC: c0 = the n constants, c1
 * unused (may be NULL).  PWL: c0 = intercepts alpha[0..K], c1 = gradients
 * beta[0..K].  PWP: c0 = 4(K+1) coefficients, c0[4k + j] multiplying s^j on
 * interval k; c1 unused.  cap = capacity of each array; *n_out = entries
 * written. */
aicdf_status aicdf_table_get(aicdf_table t, double *c0, double *c1, int cap, int *n_out);
/* method (AICDF_PWC / AICDF_PWL / AICDF_PWP) and size (n or K) of a table */
aicdf_status aicdf_table_info(aicdf_table t, int *method, int *n);

/* ===================================================================== */
/* Sampling (Section 3: the inverse transform with Q, D or exact Phi^{-1}) */
/* ===================================================================== */
typedef enum { AICDF_F32 = 0, AICDF_F16 = 1 } aicdf_dtype;

/* out_dev[i] = approx(u_i) for i < n, where
 *   method AICDF_PWC : Q(u) = table[min(floor(n_table u), n_table-1)]  (Section 3.2)
 *   method AICDF_PWL : Algorithm 1 -- reflect about 1/2, interval index from
 *                      the FP32 exponent bits, one FMA, restore the sign
 *                      (u = 1/2 gives -0, as the piecewise linear C
 *                      listing of Section 3.3 does)
 *   method AICDF_PWP : the piecewise polynomial of the table's interval,
 *                      evaluated by Horner's rule in v = min(u, 1 - u) on the
 *                      row re-expanded in v (FP64, rounded once to FP32;
 *                      the same polynomial up to that rounding: within
 *                      ~3 2^-24 sum_j |d_j| v^j of the s form), sign
 *                      restored as for PWL
 *   method AICDF_EXACT     : the library's FP32 Phi^{-1} (max rel. error < 1e-6)
 *   method AICDF_EXACT_LIB : CUDA's normcdfinvf, for comparison
 * Uniforms: if u_dev != NULL, u_i = u_dev[i] (FP32, any value; u outside
 * [0, 1] or NaN gives NaN; u = 0 / 1 give the end values: -inf / +inf for the
 * exact methods, the end constants for PWC/PWL).  If u_dev == NULL, u_i is
 * the library's Philox uniform for sample index offset + i: Philox call
 * j = (offset+i)/4 with counter (j mod 2^32, j>>32, 0, 0), word (offset+i)%4.
 * table must be NULL for the exact methods and a table of the matching method
 * otherwise.  out_dtype: AICDF_F32, or AICDF_F16 (round-to-nearest-even of
 * the FP32 result).  out_dev must be aligned to its element size; 16-byte
 * alignment enables the vectorised path.  Asynchronous on stream. */
aicdf_status aicdf_sample(aicdf_table table, int method, const float *u_dev, uint64_t seed,
                          uint64_t offset, size_t n, void *out_dev, int out_dtype,
                          aicdf_stream_t stream);

/* Same samples as aicdf_sample with u_dev == NULL, delivered to HOST memory:
 * the library generates chunks into the caller's device staging buffer
 * (staging_bytes >= 2 MiB, 256-byte aligned; split in four parts when it
 * holds at least 4 MiB, else two) and overlaps the generation of one chunk
 * with the device-to-host copies of the previous ones (two copy streams).
 * If host_out is page-locked memory the device can address, the kernel
 * stores the samples into it directly over the host link and the staging
 * buffer is left untouched.  Synchronous: returns when host_out is complete. */
aicdf_status aicdf_sample_to_host(aicdf_table table, int method, uint64_t seed,
                                  uint64_t offset, size_t n, void *host_out, int out_dtype,
                                  void *staging_dev, size_t staging_bytes,
                                  aicdf_stream_t stream);

/* Truncated-bit sampling (Section 1 and Section 2.2: uniforms carried to a
 * fixed number of bits and offset to the cell midpoint).  Each Philox call j
 * (counter (j mod 2^32, j>>32, 0, 0), key as in aicdf_sample) yields four
 * 32-bit words of F = 32/bits fields each; sample s of the stream
 * (s = offset + i) is field h of word t of call j, s = 4F j + 4h + t, and
 * its uniform is u = (m + 1/2) 2^-bits for the field value m.  The sample is
 * the method's value at that u, as in aicdf_sample: PWC reads cell
 * floor(n_table u); EXACT gives the midpoint piecewise constant approximation
 * on 2^bits equal intervals.  bits: 8 or 16 (others AICDF_ERR_UNSUPPORTED).
 * Fewer Philox calls per sample than aicdf_sample (1/8 or 1/16 of a call).
 * out_dev must be aligned to its element size; with 32-byte alignment and
 * offset a multiple of 4F the vectorised path runs.  Asynchronous on stream. */
aicdf_status aicdf_sample_bits(aicdf_table table, int method, int bits, uint64_t seed,
                               uint64_t offset, size_t n, void *out_dev, int out_dtype,
                               aicdf_stream_t stream);

/* ===================================================================== */
/* Multilevel Monte Carlo levels (Section 4, Section 4.1)                 */
/* ===================================================================== */
typedef enum { AICDF_MODEL_GBM = 0, AICDF_MODEL_CIR = 1 } aicdf_model;
typedef enum { AICDF_SCHEME_EM = 0, AICDF_SCHEME_MILSTEIN = 1 } aicdf_scheme;
/* Payoffs P of a path: X_T; discount (X_T - K)^+; ASIAN: discount times the
 * arithmetic average of the path's 2^level post-step values X_1 .. X_N, the
 * path-dependent functional of Section 5.2 (accepted by the CIR per-step
 * calls aicdf_cir_level and aicdf_cir_level_table only; the level kernels
 * return AICDF_ERR_ARG for it). */
typedef enum { AICDF_PAYOFF_X = 0, AICDF_PAYOFF_CALL = 1, AICDF_PAYOFF_ASIAN = 2 } aicdf_payoff;
/* Level estimator kinds.  With P^ (exact variates) and P~ (approximate
 * variates from the same uniforms), fine level l and coarse level l-1
 * (P_{-1} := 0):
 *   APPROX2      Y = P~_l - P~_{l-1}                     (two-way, approximate)
 *   CORR4        Y = P^_l - P^_{l-1} - P~_l + P~_{l-1}   (four-way correction)
 *   EXACT2       Y = P^_l - P^_{l-1}                     (regular MLMC)
 *   PLAIN        Y = P^_l                                (plain Monte Carlo)
 *   PLAIN_APPROX Y = P~_l                                                     */
typedef enum {
  AICDF_KIND_APPROX2 = 0, AICDF_KIND_CORR4 = 1, AICDF_KIND_EXACT2 = 2,
  AICDF_KIND_PLAIN = 3, AICDF_KIND_PLAIN_APPROX = 4
} aicdf_kind;

typedef struct {
  int model;        /* aicdf_model                                         */
  int scheme;       /* aicdf_scheme                                        */
  int payoff;       /* aicdf_payoff: P = discount * X_T or discount*(X_T-K)^+ */
  int reserved;
  double X0, T, K;  /* initial value, horizon, strike                      */
  double mu;        /* GBM drift                                           */
  double sigma;     /* volatility (GBM) / diffusion coefficient (CIR)      */
  double kappa;     /* CIR mean-reversion rate                             */
  double theta;     /* CIR mean-reversion level                            */
  double discount;  /* payoff multiplier, e.g. exp(-rT)                    */
} aicdf_sde_params;

/* Level sums: every call below that returns the sums of one estimator term
 * writes AICDF_SUMS_PER_TERM FP64 values, [sum Y, sum Y^2, sum Y^3, sum Y^4,
 * n] over its paths -- the sample mean and variance of the Section 4.1
 * estimators, plus the third and fourth power sums from which the term's
 * kurtosis (the reliability of its variance estimate) follows.  Sums of Y and
 * Y^2 are exact FP64 sums of per-chunk FP32 partial sums (chunks of ~16 paths
 * per thread, ~32 at levels 0 and 1, each chunk's FP32 sum within 31 2^-24
 * of its sum of |Y|); those of Y^3 and Y^4 are FP32 running sums over each thread's
 * k paths, reduced across threads in FP64 (relative error at most (k-1) 2^-24,
 * typically sqrt(k) 2^-24, with k = n_paths / (resident threads) -- ~4e-6 for
 * a 10^9-path level; |Y| below ~1e-9 underflows Y^4 in FP32). */
#define AICDF_SUMS_PER_TERM 5

/* Sums over paths p = path_offset .. path_offset+n_paths-1 of the powers of Y for the
 * level estimator `kind` at `level` (2^level fine steps of size T/2^level;
 * the coarse path takes 2^(level-1) steps with the pairwise sums of the fine
 * Brownian increments, Section 4.1).  Fine step s of path p draws its uniform
 * from Philox4x32-10 keyed by seed: for level >= 2 with counter
 * (s/4, p mod 2^32, p>>32, tag), word s%4; for levels 0 and 1, where a path
 * has fewer than four steps, G = 4/2^level paths share one call: counter
 * (0, q mod 2^32, q>>32, tag) with q = p/G, word (p mod G) 2^level + s.  The
 * exact and approximate variates of a step use that same uniform (Section
 * 4.1).  approx: a PWL or PWP (K <= 15) or PWC (n <= 1024) table.
 * Models: GBM dX = mu X dt + sigma X dW; CIR dX = kappa(theta-X)dt +
 * sigma sqrt(X) dW with sqrt(|X|) (truncated scheme).  Schemes: Euler-
 * Maruyama (Section 4) or Milstein.
 * Writes sums_dev[0..4] = (sum Y, sum Y^2, sum Y^3, sum Y^4, n) (FP64).
 * workspace_dev: caller-owned device scratch of at least
 * aicdf_mlmc_level_workspace_bytes() bytes (per-block partial sums), not
 * shared with a concurrent call.  Deterministic: the same arguments give
 * bit-identical sums on the same GPU model.  Asynchronous on stream. */
size_t aicdf_mlmc_level_workspace_bytes(void);
aicdf_status aicdf_mlmc_level(const aicdf_sde_params *params, aicdf_table approx, int level,
                              int kind, uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                              uint32_t tag, double *sums_dev, void *workspace_dev,
                              size_t workspace_bytes, aicdf_stream_t stream);

/* aicdf_mlmc_level for callers that cannot allocate device memory.  The paper
 * has no counterpart; this is a library convenience.
 *
 * Who needs it: code that must not call cudaMalloc -- for example a plugin
 * running inside a host application that owns all device memory through its
 * own pool and does not let components allocate outside it, or a latency-
 * critical loop that cannot afford cudaMalloc/cudaFree and the device
 * synchronisation they imply.  Such callers cannot provide the scratch
 * workspace that aicdf_mlmc_level asks for.
 *
 * Same arguments and results as aicdf_mlmc_level, without the workspace: the
 * per-block partial sums go to a fixed array inside the library (2048
 * partials of four FP64 sums, 64 KiB, held on every GPU that loads the
 * library until the process exits).  The caller still passes the output
 * sums_dev (AICDF_SUMS_PER_TERM values).  The call allocates nothing.  Its
 * first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process, so make
 * the first call on each device before any stream capture, and do not call
 * it on a device after cudaDeviceReset there (the reset unloads the array and
 * the kept address goes stale).  A launch that would need more than 2048 thread blocks is
 * refused with AICDF_ERR_UNSUPPORTED (the library sizes the grid itself; this
 * does not happen on GPUs with up to 256 SMs).  All calls share the one
 * array: two calls that can run at the same time on the GPU (different
 * streams, no ordering between them) race and give wrong sums; serialise
 * them.  Nothing carries over between calls: every slot a call reads it has
 * written first.  Asynchronous on stream. */
aicdf_status aicdf_mlmc_level_noalloc(const aicdf_sde_params *params, aicdf_table approx,
                                      int level, int kind, uint64_t n_paths, uint64_t path_offset,
                                      uint64_t seed, uint32_t tag, double *sums_dev,
                                      aicdf_stream_t stream);

/* Optimal sample allocation (Section 4.1): for nterms estimator terms with
 * variances v[i] and costs c[i] and target RMSE eps, the Lagrange-optimal
 * counts m[i] = eps^-1 sqrt(2 T v_i / c_i) with total time
 * T = 2 eps^-2 (sum_i sqrt(v_i c_i))^2; returns T in *total.  Host only. */
aicdf_status aicdf_mlmc_allocate(int nterms, const double *v, const double *c, double eps,
                                 double *m, double *total);


/* ===================================================================== */
/* Batched MLMC terms in one persistent launch                            */
/* ===================================================================== */
/* One estimator term: `n_paths` paths (indices path_offset ...) of kind
 * `kind` at `level` for parameter set `set`, Philox stream `tag`.  Its sums
 * are defined exactly as for aicdf_mlmc_level with the same arguments. */
typedef struct {
  uint32_t set;
  int32_t level;
  int32_t kind;
  uint32_t tag;
  uint64_t n_paths;
  uint64_t path_offset;
} aicdf_batch_term;

/* Launch schedule: terms are cut into tiles of equal work: tile_paths (a
 * multiple of 32, >= block_threads) paths of a level-0 two-way term, and
 * proportionally fewer paths (by 2^level + 4 path-steps, x1.8 for the
 * four-way kind; at least block_threads) for costlier terms.  Each CTA of
 * block_threads threads (64/128/256) takes tiles from a shared counter,
 * largest first; blocks_per_sm = 0 uses the occupancy maximum.  var16 = 1 rounds every approximate variate to FP16
 * before it drives a path (FP16 approximate variates); exact variates stay FP32. */
typedef struct {
  int tile_paths;
  int block_threads;
  int blocks_per_sm;
  int var16;
} aicdf_schedule;

typedef struct aicdf_batch_s *aicdf_batch;

/* Describe a batch: n_sets parameter sets and n_terms terms over them, one
 * approximation table (PWL K <= 15 or PWC n <= 1024) and one seed.  Host only. */
aicdf_status aicdf_batch_create(const aicdf_sde_params *sets, int n_sets,
                                const aicdf_batch_term *terms, int n_terms, aicdf_table approx,
                                uint64_t seed, aicdf_batch *out);
void aicdf_batch_destroy(aicdf_batch b);
/* Device workspace a schedule needs (0 for an invalid schedule). */
size_t aicdf_batch_workspace_bytes(aicdf_batch b, const aicdf_schedule *s);
/* Run every term: sums_dev[5t .. 5t+4] = (sum Y, sum Y^2, sum Y^3, sum Y^4, n)
 * of term t (FP64).
 * The tile list of the schedule is uploaded into the workspace whenever
 * another schedule or batch used that workspace since (or never), and the
 * counter reset, the persistent kernel and the per-term reduction are
 * captured into a CUDA graph on the first run with a given (schedule,
 * workspace, sums); later runs replay it.  Only the library may write the
 * workspace between runs.
 * Deterministic: sums do not depend on which CTA ran which tile.
 * Asynchronous on stream (the first run synchronises it once). */
aicdf_status aicdf_batch_run(aicdf_batch b, const aicdf_schedule *s, double *sums_dev,
                             void *workspace_dev, size_t workspace_bytes, aicdf_stream_t stream);
/* Tiles and grid of the last run of schedule s. */
aicdf_status aicdf_batch_info(aicdf_batch b, const aicdf_schedule *s, int *n_items, int *grid);
/* Time candidate schedules (block 128/256 x tile 2..128 blocks) that fit the
 * workspace on this GPU and return the fastest (median of 3 graph replays).
 * If cache_path is given, a result cached there for this GPU model and batch
 * is returned without timing, and a new result is appended to it. */
aicdf_status aicdf_batch_autotune(aicdf_batch b, int var16, double *sums_dev,
                                  void *workspace_dev, size_t workspace_bytes,
                                  aicdf_stream_t stream, const char *cache_path,
                                  aicdf_schedule *best, double *best_ms);

/* ===================================================================== */
/* Non-central chi-squared (Section 5)                                     */
/* ===================================================================== */
/* Exact quantiles C^{-1}_nu(u_i; lambda_i) in FP64 for i < n: root finding on
 * the CDF written as the Poisson mixture of central chi-squared CDFs
 * (Section 5), Newton steps inside a bracket from Sankaran's approximation
 * (Section 5.1).  Every loop is capped; a cap that is hit ORs 1 into
 * *status_dev (device int, caller-cleared).  u outside (0, 1): 0 or +inf. */
aicdf_status aicdf_ncx2_ppf(const float *u_dev, const double *lam_dev, double nu, size_t n,
                            double *out_dev, int *status_dev, aicdf_stream_t stream);
/* Training targets for the surrogate: sample i takes u and ln(lambda) ~
 * U(loglam_lo, loglam_hi) from words 0 and 1 of Philox block i (counter
 * (i mod 2^32, i>>32, 0, tag)) and the exact rescaled quantile
 * P = (C^{-1}_nu(u; lambda) - lambda - nu) / (2 sqrt(lambda + nu)), i.e.
 * P_nu(u; nu/(lambda+nu)) of Section 5.1.  Writes u, lambda, P (FP32). */
aicdf_status aicdf_ncx2_targets(double nu, float loglam_lo, float loglam_hi, uint64_t seed,
                                uint32_t tag, size_t n, float *u_dev, float *lam_dev, float *p_dev,
                                int *status_dev, aicdf_stream_t stream);

/* ===================================================================== */
/* Learned surrogate of P_nu(U; y) (Section 5.1 rescaling)                 */
/* ===================================================================== */
/* A learned surrogate of P_nu(U; y), y = nu / (lambda + nu) (the rescaled
 * quantile of Section 5.1), for one fixed nu:
 *   P~(u, lambda) = Phi^{-1}(u) + sqrt(y) N(x0, x1),
 *   x0 = s(u)/3, s(u) = sign(u-1/2) sqrt(-2 ln(2 min(u,1-u))),  x1 = 2 sqrt(y) - 1,
 * with N a 2 -> 64 -> 64 -> 1 tanh network; then
 * C~^{-1}_nu(u; lambda) = lambda + nu + 2 sqrt(lambda + nu) P~.  P tends to
 * Phi^{-1}(u) as y -> 0 with P - Phi^{-1} = O(sqrt(y)), so N learns the bounded
 * correction (P - Phi^{-1}) / sqrt(y) over every lambda >= 0 (x1 covers
 * [-1, 1) as lambda runs over [0, inf)); Phi^{-1} is the library's FP32
 * inverse.  The 64 x 64 layer runs on the tensor cores in BF16 with FP32
 * accumulation (tcgen05 MMAs into tensor memory for evaluation and training;
 * the CIR path kernel's in-loop evaluation uses warp-level MMAs); FP32 master
 * weights.  The handle owns its device buffers (allocated at create).
 * Parameter blob layout (FP32): W1[64][2] | b1[64] | W2[64 out][64 in]
 * | b2[64] | w3[64] | b3, aicdf_surrogate_param_count() floats. */
typedef struct aicdf_surrogate_s *aicdf_surrogate;
aicdf_status aicdf_surrogate_create(double nu, uint64_t seed, aicdf_surrogate *out);
void aicdf_surrogate_destroy(aicdf_surrogate s);
int aicdf_surrogate_param_count(void);
aicdf_status aicdf_surrogate_get_params(aicdf_surrogate s, float *host, int cap);
/* Replaces the weights and resets the optimiser state. */
aicdf_status aicdf_surrogate_set_params(aicdf_surrogate s, const float *host, int n);
/* Save the trained network (nu and the parameter blob, not the optimiser
 * state) to a host file, and create a handle from such a file (on the
 * current device); AICDF_ERR_ARG if the file cannot be written or read or is
 * not a saved surrogate.  Host I/O, synchronous. */
aicdf_status aicdf_surrogate_save(aicdf_surrogate s, const char *path);
aicdf_status aicdf_surrogate_load(const char *path, aicdf_surrogate *out);
/* p_out_dev[i] = P~(u_dev[i], lam_dev[i]).  Should a tensor-core product not
 * signal completion within the kernel's bounded wait (a fault of the device,
 * not of the inputs), the affected outputs are NaN. */
aicdf_status aicdf_surrogate_eval(aicdf_surrogate s, const float *u_dev, const float *lam_dev,
                                  size_t n, float *p_out_dev, aicdf_stream_t stream);
/* The network is fitted to g_i = (target_i - Phi^{-1}(u_i)) / sqrt(y_i) for
 * targets of P: gradient of L = mean_i (N_i - g_i)^2 (= mean_i (P~_i -
 * target_i)^2 / y_i, the squared error of P~ in the units that a CIR step
 * carries equally at every lambda) over the n samples, into
 * grad_dev[0 .. param_count) (same layout as the parameters), with the sum of
 * (N_i - g_i)^2 at grad_dev[param_count]; n <= 2^24. */
aicdf_status aicdf_surrogate_grad(aicdf_surrogate s, const float *u_dev, const float *lam_dev,
                                  const float *target_dev, size_t n, float *grad_dev,
                                  aicdf_stream_t stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the batch; writes the
 * batch's L to *loss_dev if loss_dev is not NULL. */
aicdf_status aicdf_surrogate_train_step(aicdf_surrogate s, const float *u_dev, const float *lam_dev,
                                        const float *target_dev, size_t n, float lr,
                                        float *loss_dev, aicdf_stream_t stream);
/* epochs passes over n samples in batches of `batch` (the tail that does not
 * fill a batch is skipped), step size decaying geometrically from lr to
 * lr_final; the last batch's L goes to *loss_dev.  One epoch's launches are
 * captured as a CUDA graph and replayed per epoch (the step sizes come from a
 * device step counter), so the call must not itself be made during a stream
 * capture.  The samples' network inputs and g_i are formed once per call into
 * a device buffer of 16 bytes a sample that the surrogate keeps (and grows for
 * a larger n) until aicdf_surrogate_destroy; should that allocation fail, every
 * gradient launch forms them itself, with the same result. */
aicdf_status aicdf_surrogate_train(aicdf_surrogate s, const float *u_dev, const float *lam_dev,
                                   const float *target_dev, size_t n, size_t batch, int epochs,
                                   float lr, float lr_final, float *loss_dev, aicdf_stream_t stream);

/* ===================================================================== */
/* CIR with exact and approximate non-central chi-squared steps (Section 5.2) */
/* ===================================================================== */
/* Kinds of Y for one path of 2^level steps of size h = T/2^level; every step
 * draws one uniform U (Philox counter (s/4, p mod 2^32, p>>32, tag), word
 * s%4) and both sides use the same U:
 *   EXACT       P(X^_T), X^' = c C^{-1}_nu(U; X^ e^{-kappa h}/c)  (FP64 root finder)
 *   SURROGATE   P(X~_T), X~' = c max(C~^{-1}_nu(U; lambda~), 0)   (learned P~)
 *   DIFF        P(X^_T) - P(X~_T)                                  (same steps)
 *   GAUSS       as SURROGATE with P~ replaced by Phi^{-1}(U), the y -> 0
 *               limit of P (Section 5.1): the approximation without the network
 *   DIFF_GAUSS  P(X^_T) - P(X~_T) for GAUSS
 * with c = sigma^2 (1 - e^{-kappa h}) / (4 kappa), nu = 4 kappa theta / sigma^2. */
typedef enum {
  AICDF_CIR_EXACT = 0, AICDF_CIR_SURROGATE = 1, AICDF_CIR_DIFF = 2,
  AICDF_CIR_GAUSS = 3, AICDF_CIR_DIFF_GAUSS = 4,
  AICDF_CIR_TABLE = 5, AICDF_CIR_DIFF_TABLE = 6  /* aicdf_cir_level_table only */
} aicdf_cir_kind;

/* Sums of Y, Y^2, Y^3, Y^4 and n (FP64, sums_dev[0..4]) over paths
 * path_offset .. path_offset+n_paths-1 of
 * a CIR model (params->model = AICDF_MODEL_CIR, payoff X or call; level <=
 * 12).  sur: a surrogate trained for this nu (required by SURROGATE and
 * DIFF, else may be NULL).  workspace: as for aicdf_mlmc_level.  Root-finder
 * caps hit OR 1 into *status_dev.  Asynchronous on stream. */
aicdf_status aicdf_cir_level(const aicdf_sde_params *params, aicdf_surrogate sur, int level,
                             int kind, uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                             uint32_t tag, double *sums_dev, void *workspace_dev,
                             size_t workspace_bytes, int *status_dev, aicdf_stream_t stream);

/* ===================================================================== */
/* Tabulated non-central chi-squared inverse (Section 5.1)               */
/* ===================================================================== */
/* For a fixed nu, with y = nu / (lambda + nu) and
 *   P_nu(U; y) = sqrt(nu / 4y) ((y / nu) C^{-1}_nu(U; (1 - y) nu / y) - 1),
 * the approximation is C~^{-1}_nu(U; lambda) = h + 2 sqrt(h) P~(U; y), h = lambda + nu,
 * where P~ interpolates linearly in sqrt(y) between tables at n_knots knots
 * sqrt(y_i) = i / (n_knots - 1) (y = 0: the Gaussian limit Phi^{-1}; y = 1: the
 * central chi^2).  Each knot holds two tables, for u <= 1/2 and u > 1/2, each
 * the L2-optimal polynomial of the given degree (1..3) on the K dyadic
 * intervals of v = min(u, 1 - u) in the local variable s (as for AICDF_PWP);
 * row 0 of each half is the value at u = 1/2.  The paper's Table 5 uses
 * K = 16 and 16 knots.  Built on the host in FP64 (exact quantiles from the
 * library's root finder; about a second); *out owns the table.
 * Errors: AICDF_ERR_ARG for nu <= 0, K outside 1..30, n_knots outside 2..64
 * or degree outside 1..3; AICDF_ERR_DOMAIN if a quantile did not converge. */
typedef struct aicdf_ncx2_table_s *aicdf_ncx2_table;
aicdf_status aicdf_ncx2_table_build(double nu, int K, int n_knots, int degree, aicdf_ncx2_table *out);
void aicdf_ncx2_table_destroy(aicdf_ncx2_table t);
aicdf_status aicdf_ncx2_table_info(aicdf_ncx2_table t, double *nu, int *K, int *n_knots, int *degree);
/* FP64 coefficients, layout [knot][half][row 0..K][power 0..3] (half 1: u > 1/2);
 * cap in doubles; with coef == NULL only *n_out is set. */
aicdf_status aicdf_ncx2_table_get(aicdf_ncx2_table t, double *coef, size_t cap, size_t *n_out);
/* out_dev[i] = C~^{-1}_nu(u_dev[i]; lam_dev[i]) in FP32 (device arrays of n;
 * NaN for u outside [0, 1] or lambda < 0, NaN or inf).  The kernels take the
 * table as a launch parameter: n_knots * 2 * (K + 1) <= 1024, else
 * AICDF_ERR_UNSUPPORTED.  Asynchronous on stream. */
aicdf_status aicdf_ncx2_table_eval(aicdf_ncx2_table t, const float *u_dev, const float *lam_dev, size_t n,
                                   float *out_dev, aicdf_stream_t stream);
/* aicdf_cir_level with the tabulated approximation in place of the
 * surrogate: kinds AICDF_CIR_EXACT, AICDF_CIR_TABLE (P(X~_T) with
 * X~' = c max(C~^{-1}_nu(U; lambda~), 0)) and AICDF_CIR_DIFF_TABLE
 * (P(X^_T) - P(X~_T), same uniforms).  The table's nu must equal
 * 4 kappa theta / sigma^2 (AICDF_ERR_DOMAIN otherwise). */
aicdf_status aicdf_cir_level_table(const aicdf_sde_params *params, aicdf_ncx2_table table, int level,
                                   int kind, uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                                   uint32_t tag, double *sums_dev, void *workspace_dev,
                                   size_t workspace_bytes, int *status_dev, aicdf_stream_t stream);

/* ===================================================================== */
/* MLMC driver (Section 4.1): estimate E[P] to a target RMSE               */
/* ===================================================================== */
typedef enum {
  AICDF_EST_NESTED = 0,   /* theta~ : per level APPROX2 + CORR4 terms (independent streams) */
  AICDF_EST_REGULAR = 1,  /* theta^ : per level EXACT2 terms                              */
  AICDF_EST_PLAIN = 2,    /* plain Monte Carlo with exact variates at the finest level     */
  AICDF_EST_ADAPTIVE = 3  /* per level the cheaper of the nested pair and an EXACT2 term:
                             the pair is piloted; where (sqrt(V2 c2) + sqrt(V4 c4))^2 >
                             V2 c_exact2 (Section 4.1's cost model) it is dropped and an
                             EXACT2 term on its own stream replaces it (a library
                             extension of the paper's nested estimator)                 */
} aicdf_estimator;

#define AICDF_MAX_LEVELS 24

typedef struct {
  double eps;             /* target RMSE: variance eps^2/2 and bias^2 <= eps^2/2        */
  int estimator;          /* aicdf_estimator                                              */
  int L_min, L_max;       /* first and last admissible finest level                      */
  int fixed_L;            /* >= 0: use exactly this finest level (no bias test)           */
  uint64_t n_pilot;       /* pilot paths per new term at levels <= L_min (0: 10^4),
                             halved for each level above L_min (at least 128;
                             plain Monte Carlo keeps n_pilot); a
                             nested estimator's four-way terms, with their far
                             smaller variance, start from max(128, n_pilot / 16)
                             (at most n_pilot)                                            */
  uint64_t seed;
  double weak_order;      /* alpha in the bias estimate |E Y_L| / (2^alpha - 1)           */
} aicdf_mlmc_opts;

typedef struct {
  double estimate;        /* sum over terms of the sample means                          */
  double variance;        /* estimated variance of the estimator                         */
  double bias;            /* bias estimate from the finest level                          */
  double gpu_ms;          /* device time of all path launches (CUDA events)               */
  double wall_ms;         /* host wall time of the whole run                              */
  int L;                  /* finest level used                                            */
  int converged;          /* 1 if the bias test passed (or fixed_L was given)             */
  int n_terms;            /* terms per level: 2 (nested) or 1                            */
  int launches;           /* path-kernel launches issued                                  */
  /* per level l and term t (t = 0: APPROX2 / EXACT2 / PLAIN, t = 1: CORR4) */
  uint64_t paths[AICDF_MAX_LEVELS][2];
  double mean[AICDF_MAX_LEVELS][2];
  double var[AICDF_MAX_LEVELS][2];
  double kurt[AICDF_MAX_LEVELS][2];     /* kurtosis E(Y-EY)^4 / Var(Y)^2 of the term          */
  double cost_ns[AICDF_MAX_LEVELS][2];  /* measured device ns per path                     */
  int exact_level[AICDF_MAX_LEVELS];    /* AICDF_EST_ADAPTIVE: 1 where level l uses an EXACT2
                                           term (slot 0) in place of the nested pair         */
} aicdf_mlmc_result;

/* Run one estimator to RMSE opts->eps.  Each term draws uniforms from its own
 * Philox stream (tag = 1 + 64*estimator + 2*l + t; an adaptive estimator's
 * EXACT2 replacement at level l: 1 + 64*estimator + 42 + l), extending the stream with
 * path_offset as more paths are added, so the result is reproducible from the
 * seed.  Path counts follow the optimal allocation of Section 4.1 from the
 * measured variances and per-path device times.  A term whose share f of
 * the estimator's variance sum_i V_i / n_i is not small keeps at least
 * (k - 1) (4 f)^2 paths, k its measured kurtosis, so that its variance
 * estimate moves the estimator's by no more than about 25% of its share (a
 * library choice; the paper takes the variances as known).  While the bias estimate
 * exceeds eps/sqrt(2), levels are added (up to L_max; converged = 0 if it is
 * reached): as many at once as the weak order predicts are needed,
 * ceil(log2(bias / (eps/sqrt(2))) / weak_order), at least one.  workspace_dev: at least aicdf_mlmc_run_workspace_bytes().
 * Synchronous on stream. */
size_t aicdf_mlmc_run_workspace_bytes(void);
aicdf_status aicdf_mlmc_run(const aicdf_sde_params *params, aicdf_table approx,
                            const aicdf_mlmc_opts *opts, aicdf_mlmc_result *result,
                            void *workspace_dev, size_t workspace_bytes, aicdf_stream_t stream);

/* aicdf_mlmc_run for n_sets independent parameter sets at once.  Each set
 * follows the same procedure with its own variances, costs and bias test;
 * every round is one batched launch holding the new paths of all sets (a
 * small set costs no launch of its own).  Set s draws from its own streams
 * (tag = 256 s + 1 + 64*estimator + 2*l + t).  results[s] as for
 * aicdf_mlmc_run, except that gpu_ms, wall_ms and launches are those of the
 * whole run.  workspace_dev: at least aicdf_mlmc_run_sets_workspace_bytes(n_sets).
 * Synchronous on stream. */
size_t aicdf_mlmc_run_sets_workspace_bytes(int n_sets);
aicdf_status aicdf_mlmc_run_sets(const aicdf_sde_params *sets, int n_sets, aicdf_table approx,
                                 const aicdf_mlmc_opts *opts, aicdf_mlmc_result *results,
                                 void *workspace_dev, size_t workspace_bytes, aicdf_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* AICDF_H */
