// Device primitives shared by the sampling and path kernels.
//
//  * Philox4x32-10 (Salmon et al., SC'11) with the round keys precomputed on
//    the host: the key schedule is the same for every thread of a launch, so
//    the xor with the round key reads a kernel-parameter (constant bank) word.
//  * v01 / u01: the 32-bit word -> uniform map: the top bit picks the half of
//    (0, 1) and the low 22 bits m the cell, v = min(u, 1-u) = (2m+1) 2^-24 and
//    u = v or 1 - v, both exact in FP32.
//  * pwl_eval: Algorithm 1 (Section 3.3) with the 2 x 16 coefficients held in
//    registers across the warp and fetched by __shfl_sync -- the GPU form of
//    keeping the table in one 512-bit vector register (Section 3.3).
//  * pwc_eval: the lookup of Section 3.2, table staged in shared memory.
//  * phiinv_f32: exact FP32 inverse Gaussian CDF (Giles' erfinv formulation,
//    coefficients fitted by fit_phiinv.py), FP64 branch in the far tail.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>

#include "phiinv_coefs.h"

namespace aicdf {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr uint32_t PHILOX_M0 = 0xD2511F53u;
constexpr uint32_t PHILOX_M1 = 0xCD9E8D57u;
constexpr uint32_t PHILOX_W0 = 0x9E3779B9u;
constexpr uint32_t PHILOX_W1 = 0xBB67AE85u;

// Round keys of Philox4x32-10 for one seed: k0[r] = lo(seed) + r*W0,
// k1[r] = hi(seed) + r*W1 (mod 2^32).
struct PhiloxKeys {
  uint32_t k0[10];
  uint32_t k1[10];
};

inline PhiloxKeys make_keys(uint64_t seed) {
  PhiloxKeys k;
  uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    k.k0[r] = a;
    k.k1[r] = b;
    a += PHILOX_W0;
    b += PHILOX_W1;
  }
  return k;
}

// One Philox round: the two 32 x 32 -> 64 products are written as 64-bit
// multiplies, so each is a single wide multiply giving both halves.
__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t k0, uint32_t k1) {
  const uint64_t p0 = (uint64_t)PHILOX_M0 * c.x, p1 = (uint64_t)PHILOX_M1 * c.z;
  return make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
}

__device__ __forceinline__ uint4 philox(uint4 c, const PhiloxKeys &k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) c = philox_round(c, k.k0[r], k.k1[r]);
  return c;
}

// NC independent Philox calls advanced round by round together, so that the
// multiplies of different calls overlap (one call alone is a serial chain of
// 10 dependent rounds).
template <int NC>
__device__ __forceinline__ void philox_n(uint4 (&c)[NC], const PhiloxKeys &k) {
#pragma unroll
  for (int r = 0; r < 10; ++r)
#pragma unroll
    for (int q = 0; q < NC; ++q) c[q] = philox_round(c[q], k.k0[r], k.k1[r]);
}

// The library's uniform from a Philox word x: the sign bit picks the half of
// (0, 1) and the low 22 bits m the cell within it.  v = (1 + m 2^-23) -
// (1 - 2^-24) = (2m+1) 2^-24 (one logic op and one exact add) is min(u, 1-u)
// in (0, 1/2); u = v when bit 31 is clear and 1 - v (exact) when it is set.
// So u is the midpoint (2k+1) 2^-24 of cell k of 2^23 equal cells, k = m or
// 2^23 - 1 - m, and never 1/2; bits 22..30 are unused.  The samplers' word
// forms take v and the sign bit as they stand, with no compare or reflection.
__device__ __forceinline__ float v01(uint32_t x) {
  return __uint_as_float(0x3F800000u | (x & 0x3FFFFFu)) - 0x1.fffffep-1f;
}
__device__ __forceinline__ float u01(uint32_t x) {
  const float v = v01(x);
  return (x & 0x80000000u) ? 1.0f - v : v;
}

// Truncated-bit uniform: cell m of 2^B, u = (m + 1/2) 2^-B = (1 + m 2^-B) -
// (1 - 2^-(B+1)); the significand holds m exactly and the subtraction is exact
// (its result needs at most B + 1 bits).  Such u lie on the 2^-24 grid, so the
// grid forms below apply to them as they stand.
template <int B>
__device__ __forceinline__ float ubits(uint32_t m) {
  static_assert(B >= 1 && B <= 23, "field width");
  constexpr float c = 1.0f - 1.0f / (float)(2u << B);
  return __uint_as_float(0x3F800000u | (m << (23 - B))) - c;
}

// u - 1/2 of the same cell in one exact add: (1 + m 2^-B) - (3/2 - 2^-(B+1));
// the constant is exact in FP32 for B <= 22 and the result needs B + 1 bits.
template <int B>
__device__ __forceinline__ float tbits(uint32_t m) {
  static_assert(B >= 1 && B <= 22, "field width");
  constexpr float c = 1.5f - 1.0f / (float)(2u << B);
  return __uint_as_float(0x3F800000u | (m << (23 - B))) - c;
}

// ---------------------------------------------------------------------------
// Algorithm 1 for uniforms on the 2^-24 grid (the library's own uniforms).
// On the grid, u - 1/2 and 1/2 - |u - 1/2| are exact, so v = min(u, 1-u) costs
// two adds.  v in [2^-24, 1/2] has biased exponent e in [103, 126] and row
// 126 - e; since the shuffle reads lane (e mod 32) = e - 96, lane L holds row
// min(30 - L, K) and the exponent is the lane index as it stands (no bias
// subtraction, no cap).  The sign is restored by one xor with the complement
// of the sign of u - 1/2 (u = 1/2 gives -0, as the piecewise linear C listing
// of Section 3.3 does).
struct PwlRows {
  float a, b;
};

__device__ __forceinline__ PwlRows pwl_lane_rows(const float *alpha, const float *beta, int K) {
  const int r = min(max(30 - (int)(threadIdx.x & 31), 0), K);
  PwlRows c;
  c.a = alpha[r];
  c.b = beta[r];
  return c;
}

// Must be called by all 32 lanes of the warp.  Equals pwl_eval_grid(u01(x)).
__device__ __forceinline__ float pwl_eval_word(uint32_t x, const PwlRows &c) {
  const float v = v01(x);
  const uint32_t e = __float_as_uint(v) >> 23;  // the shuffle uses e mod 32
  const float a = __shfl_sync(0xffffffffu, c.a, e);
  const float b = __shfl_sync(0xffffffffu, c.b, e);
  return __uint_as_float(__float_as_uint(fmaf(b, v, a)) ^ (x & 0x80000000u));
}

// Must be called by all 32 lanes of the warp; t = u - 1/2 (exact).
__device__ __forceinline__ float pwl_eval_t(float t, const PwlRows &c) {
  const float v = 0.5f - fabsf(t);
  const uint32_t e = __float_as_uint(v) >> 23;  // the shuffle uses e mod 32
  const float a = __shfl_sync(0xffffffffu, c.a, e);
  const float b = __shfl_sync(0xffffffffu, c.b, e);
  const float z = fmaf(b, v, a);
  return __uint_as_float(__float_as_uint(z) ^ (~__float_as_uint(t) & 0x80000000u));
}
__device__ __forceinline__ float pwl_eval_grid(float u, const PwlRows &c) { return pwl_eval_t(u - 0.5f, c); }

// ---------------------------------------------------------------------------
// Piecewise polynomial (degree <= 3) on the dyadic intervals.  The table's
// rows are polynomials in the local variable s of each interval (the fraction
// of v's significand on I_k = [2^-(k+1), 2^-k), s = 2^(k+1) v - 1; s = 2^K v on
// the singular interval); the kernels receive each row re-expanded in v itself
// (d_j, built on the host from the FP32 s-coefficients in FP64), so that one
// Horner pass in v needs neither s nor a test for the singular row.  The rows
// are staged in shared memory for one 16-byte load per variate (four
// coefficients; four shuffles of lane-held rows cost more): entry i < 512
// holds row min(126 - i, K) (unsigned, so every i > 126 -- v >= 1, a set sign
// bit, NaN -- takes the singular row K, and -0 lands there like +0), indexed
// by the top 9 bits of v (its sign and biased exponent).  tab: [4 powers][16
// rows].  All threads of the block must call the stager.
constexpr int kPwpStagedRows = 512;
__device__ __forceinline__ void pwp_stage_rows(const float *tab, int K, float4 *rows) {
  for (int i = threadIdx.x; i < kPwpStagedRows; i += blockDim.x) {
    const int r = (int)min(126u - (uint32_t)i, (uint32_t)K);
    rows[i] = make_float4(tab[r], tab[16 + r], tab[32 + r], tab[48 + r]);
  }
  __syncthreads();
}
__device__ __forceinline__ float pwp_horner(float v, const float4 *rows) {
  const float4 d = rows[__float_as_uint(v) >> 23];
  return fmaf(fmaf(fmaf(d.w, v, d.z), v, d.y), v, d.x);
}
// The library's uniform of word x (v and the sign straight from the bits).
__device__ __forceinline__ float pwp_staged_word(uint32_t x, const float4 *rows) {
  const float z = pwp_horner(v01(x), rows);
  return __uint_as_float(__float_as_uint(z) ^ (x & 0x80000000u));
}
// Grid uniforms, t = u - 1/2 (exact).
__device__ __forceinline__ float pwp_staged_t(float t, const float4 *rows) {
  const float z = pwp_horner(0.5f - fabsf(t), rows);
  return __uint_as_float(__float_as_uint(z) ^ (~__float_as_uint(t) & 0x80000000u));
}
// Any FP32 u (caller uniforms): reflection by 1 - u.
__device__ __forceinline__ float pwp_staged(float u, const float4 *rows) {
  const bool lower = u < 0.5f;
  const float z = pwp_horner(lower ? u : 1.0f - u, rows);
  return lower ? z : -z;
}

// Piecewise constant with n = 2^q intervals (q >= 1) for the uniform of word
// x: u = (2k+1) 2^-24 with k = m (bit 31 clear) or 2^23 - 1 - m (set), m = low
// 22 bits, so floor(n u) = k >> (23 - q) is j = m >> (23 - q) below 1/2 and
// n - 1 - j above.  The word forms index a word-order copy of the table,
// W[j] = T[j] and W[n/2 + j] = T[n - 1 - j] (j < n/2), at slot j + (n/2) bit31:
// the low q - 1 bits of x >> (23 - q) joined to bit q - 1 of x >> (32 - q), one
// select.
struct PwcWord {
  uint32_t shift, shift_top, lo;  // 23 - q, 32 - q, n/2 - 1
};
__host__ __device__ inline PwcWord pwc_word(uint32_t q) { return PwcWord{23u - q, 32u - q, (1u << (q - 1)) - 1u}; }
__device__ __forceinline__ uint32_t pwc_slot_from_word(uint32_t x, const PwcWord &p) {
  return ((x >> p.shift) & p.lo) | ((x >> p.shift_top) & ~p.lo);
}
// The row of T held at slot i of the word-order copy.
__device__ __forceinline__ int pwc_word_row(int i, int n) { return i < n / 2 ? i : n - 1 - (i - n / 2); }

// ---------------------------------------------------------------------------
// Algorithm 1.  Lane L of every warp holds the coefficients of row (L & 15);
// lanes 0..15 hold them negated (used for u >= 1/2), lanes 16..31 as they are
// (u < 1/2), so the sign restore is folded into the row choice.
struct PwlLane {
  float a, b;
};

__device__ __forceinline__ PwlLane pwl_lane_coefs(const float *alpha, const float *beta) {
  const int lane = threadIdx.x & 31;
  PwlLane c;
  c.a = alpha[lane & 15];
  c.b = beta[lane & 15];
  if (lane < 16) {
    c.a = -c.a;
    c.b = -c.b;
  }
  return c;
}

// Must be called by all 32 lanes of the warp (the shuffles are warp-wide).
__device__ __forceinline__ float pwl_eval(float u, const PwlLane &c, unsigned kmax) {
  const bool lower = u < 0.5f;                           // predicate
  const float v = lower ? u : 1.0f - u;                  // reflect (exact)
  const uint32_t e = __float_as_uint(v) >> 23;           // exponent bits
  uint32_t idx = min(126u - e, kmax);                    // bias offset, cap
  idx |= lower ? 16u : 0u;                               // sign via the row
  const float a = __shfl_sync(FULL_MASK, c.a, idx);
  const float b = __shfl_sync(FULL_MASK, c.b, idx);
  return fmaf(b, v, a);                                  // one FMA
}

// Piecewise constant: n a power of two, table in shared memory.
__device__ __forceinline__ float pwc_eval(float u, const float *s_tab, float nf, int nmax) {
  const int m = min(__float2int_rz(u * nf), nmax);       // floor(n u), capped
  return s_tab[max(m, 0)];
}

// ---------------------------------------------------------------------------
// Exact inverse Gaussian CDF in FP32.  With v = min(u, 1-u), x = 2v-1 and
// w = -ln(4v(1-v)), Phi^{-1}(v) = x g(w); g is a fitted polynomial in w (w < W0)
// or in sqrt(w) (W0 <= w <= W1).  Below v ~ 1.7e-8 (and for v = 0, NaN) an
// FP64 branch runs three Newton steps on ln Phi(z) = ln v.
static __device__ __noinline__ float phiinv_far_tail_f64(float vf) {
  const double v = (double)vf;
  if (!(v > 0.0)) return v == 0.0 ? -__int_as_float(0x7f800000) : __int_as_float(0x7fc00000);
  const double L = -2.0 * log(v);
  double z = -sqrt(L - log(6.283185307179586 * L));      // asymptotic start
#pragma unroll 1
  for (int it = 0; it < 3; ++it) {
    const double P = 0.5 * erfc(-z * 0.7071067811865476);
    const double d = 0.3989422804014327 * exp(-0.5 * z * z);
    z -= (log(P) - log(v)) * P / d;
  }
  return (float)z;
}

__device__ __forceinline__ float phiinv_f32(float u) {
  const bool lower = u < 0.5f;
  const float v = lower ? u : 1.0f - u;
  const float x = fmaf(2.0f, v, -1.0f);
  const float w = -__logf(4.0f * v * (1.0f - v));
  float z;
  if (w < AICDF_PHIINV_W0) {
    z = x * aicdf_phiinv_poly_central(w - AICDF_PHIINV_WC);
  } else if (w <= AICDF_PHIINV_W1) {
    z = x * aicdf_phiinv_poly_tail(sqrtf(w) - AICDF_PHIINV_S0);
  } else {
    z = phiinv_far_tail_f64(v);
  }
  return lower ? z : -z;
}

// The same for uniforms on the 2^-24 grid (the library's own, and the
// truncated-bit cells): v >= 2^-24 keeps w <= 24 ln 2 - ln 4 < W1, so the FP64
// far-tail branch is never taken and is left out -- identical results, and no
// call site in the callers' unrolled loops (6% more exact samples per second).
// Lower half: v in (0, 1/2] -> Phi^-1(v) <= 0.
__device__ __forceinline__ float phiinv_f32_half(float v) {
  const float x = fmaf(2.0f, v, -1.0f);
  const float w = -__logf(4.0f * v * (1.0f - v));
  return w < AICDF_PHIINV_W0 ? x * aicdf_phiinv_poly_central(w - AICDF_PHIINV_WC)
                             : x * aicdf_phiinv_poly_tail(sqrtf(w) - AICDF_PHIINV_S0);
}
__device__ __forceinline__ float phiinv_f32_grid(float u) {
  const bool lower = u < 0.5f;
  const float z = phiinv_f32_half(lower ? u : 1.0f - u);
  return lower ? z : -z;
}
// The same for a word x: equals phiinv_f32_grid(u01(x)) (v < 1/2, so z != 0).
__device__ __forceinline__ float phiinv_f32_word(uint32_t x) {
  return __uint_as_float(__float_as_uint(phiinv_f32_half(v01(x))) ^ (x & 0x80000000u));
}

__device__ __forceinline__ bool in_unit(float u) { return u >= 0.0f && u <= 1.0f; }

}  // namespace aicdf
