// Device evaluation of the Section 5.1 approximation of the non-central
// chi-squared inverse CDF for a fixed nu:
//   C~^{-1}_nu(u; lambda) = h + 2 sqrt(h) P~(u; y),  h = lambda + nu,  y = nu / h,
// where P~ interpolates linearly in sqrt(y) between tables at knots
// sqrt(y_i) = i / (n_knots - 1).  Each knot holds two tables (u <= 1/2 and
// u > 1/2), each a polynomial of degree <= 3 per dyadic interval of
// v = min(u, 1 - u) in the local variable s, as for the Gaussian tables:
// s is the fraction of v's significand on I_k = [2^-(k+1), 2^-k), k < K, and
// v 2^K on the singular interval (0, 2^-K); row 0 is the value at u = 1/2.
#pragma once

#include <cstdint>

namespace aicdf {

constexpr int kNcx2TabMaxRows = 1024;  // n_knots * 2 * (K + 1) float4 rows (16 KiB)

struct Ncx2TabArgs {
  int K, n_knots;
  float nu, scale_k;  // scale_k = 2^K
  float4 rows[kNcx2TabMaxRows];  // [knot][half][row] -> (c0, c1, c2, c3)
};

// rows: the table (staged in shared memory by the caller)
__device__ __forceinline__ float ncx2_table_P(const float4 *rows, int K, int n_knots, float scale_k, float u,
                                              float sqrt_y) {
  const bool upper = u > 0.5f;
  const float v = upper ? 1.0f - u : u;
  // 126 - e wraps past K for a set sign bit (u = -0), as in pwl_eval
  const uint32_t k = min(126u - (__float_as_uint(v) >> 23), (uint32_t)K);
  const float frac = __uint_as_float((__float_as_uint(v) & 0x7FFFFFu) | 0x3F800000u) - 1.0f;
  const float s = k == (uint32_t)K ? v * scale_k : frac;
  const float t = sqrt_y * (float)(n_knots - 1);
  const int i = min(max((int)t, 0), n_knots - 2);
  const float f = t - (float)i;
  const float4 c0 = rows[(i * 2 + (int)upper) * (K + 1) + (int)k];
  const float4 c1 = rows[((i + 1) * 2 + (int)upper) * (K + 1) + (int)k];
  const float p0 = fmaf(fmaf(fmaf(c0.w, s, c0.z), s, c0.y), s, c0.x);
  const float p1 = fmaf(fmaf(fmaf(c1.w, s, c1.z), s, c1.y), s, c1.x);
  return fmaf(f, p1 - p0, p0);
}

// C~^{-1}_nu(u; lambda), lambda >= 0
__device__ __forceinline__ float ncx2_table_ppf(const float4 *rows, int K, int n_knots, float nu, float scale_k,
                                                float u, float lam) {
  const float h = lam + nu;
  const float p = ncx2_table_P(rows, K, n_knots, scale_k, u, sqrtf(nu / h));
  return fmaf(2.0f * sqrtf(h), p, h);
}

}  // namespace aicdf
