// Section 5.1: piecewise polynomial approximation of the non-central
// chi-squared inverse CDF for a fixed nu -- host FP64 table build and the
// device evaluation entry point.
//
// With y = nu / (lambda + nu), the scaled quantile
//   P_nu(U; y) = sqrt(nu / 4y) ((y / nu) C^{-1}_nu(U; (1 - y) nu / y) - 1)
// tends to Phi^{-1}(U) as y -> 0 and to C^{-1}_nu(U) / (2 sqrt nu) - sqrt(nu) / 2
// (the central law) as y -> 1.  Tables of P_nu(.; y_i) are built at knots
// equally spaced in sqrt(y), separately for u <= 1/2 and u > 1/2 (the law is
// not antisymmetric), each the L2-optimal polynomial of degree d on every
// dyadic interval of v = min(u, 1 - u); P~ interpolates linearly in sqrt(y).
//
// The projection on each interval uses the shifted Legendre basis (no linear
// system): Gauss-Legendre in v on the regular intervals and, on the singular
// interval (0, b), the substitution v = b e^{-w} (s = e^{-w}, w in [0, 36],
// where b e^{-36} < 1e-15 b: the part below holds no measurable L2 mass).
// The exact quantile is the library's FP64 root finder, solved on the tail
// probability itself (C = v below 1/2, 1 - C = v above) so that small v keep
// their relative accuracy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "aicdf_internal.h"
#include "ncx2.cuh"
#include "ncx2_table.cuh"
#include "quad.h"

struct aicdf_ncx2_table_s {
  uint32_t magic;
  double nu;
  int K, n_knots, degree;
  std::vector<double> coef;  // [knot][half][row][4], FP64
  std::vector<float> coef32;
};

namespace aicdf {

constexpr uint32_t kNcx2TableMagic = 0x4E435854u;  // "NCXT"

static bool ncx2_table_ok(const aicdf_ncx2_table_s *t) { return t && t->magic == kNcx2TableMagic; }

// P_nu at v on one half (upper: u = 1 - v) for knot y; y = 0 is the Gaussian limit.
static double knot_P(double v, bool upper, double nu, double y, int *status) {
  if (y <= 0.0) return upper ? -host_phiinv(v) : host_phiinv(v);
  const double lam = (1.0 - y) * nu / y;
  const double z = upper ? -host_phiinv(v) : host_phiinv(v);
  const double x = ncx2_quantile(v, upper, z, nu, lam, status);
  return std::sqrt(nu / (4.0 * y)) * ((y / nu) * x - 1.0);
}

static void build_knot(aicdf_ncx2_table_s *t, int i, int *status) {
  const int K = t->K;
  const double r = (double)i / (t->n_knots - 1), y = r * r, nu = t->nu;
  std::vector<double> gx, gw;
  gl_nodes(24, gx, gw);
  const double mid = knot_P(0.5, false, nu, y, status);
  for (int half = 0; half < 2; ++half) {
    double *rows = &t->coef[(size_t)((i * 2 + half) * (K + 1)) * 4];
    rows[0] = mid;
    rows[1] = rows[2] = rows[3] = 0.0;
    for (int k = 1; k <= K; ++k) {
      const double b = std::ldexp(1.0, -k);
      LegendreProjector pr;
      if (k < K) {
        const double a = 0.5 * b, h = b - a;
        for (size_t q = 0; q < gx.size(); ++q) {
          const double s = 0.5 * (gx[q] + 1.0);
          pr.add(s, knot_P(a + h * s, half == 1, nu, y, status), 0.5 * gw[q]);
        }
      } else {
        const int panels = 24;
        const double wmax = 36.0;
        for (int p = 0; p < panels; ++p) {
          const double w0 = wmax * p / panels, w1 = wmax * (p + 1) / panels;
          for (size_t q = 0; q < gx.size(); ++q) {
            const double wv = 0.5 * (w1 - w0) * gx[q] + 0.5 * (w1 + w0);
            const double s = std::exp(-wv);
            pr.add(s, knot_P(b * s, half == 1, nu, y, status), 0.5 * (w1 - w0) * gw[q] * s);
          }
        }
      }
      pr.monomials(t->degree, rows + 4 * k);
    }
  }
}

// Fill the kernel-parameter copy of a table.
aicdf_status pack_ncx2_table(const aicdf_ncx2_table_s *t, Ncx2TabArgs *a) {
  if (!ncx2_table_ok(t)) return AICDF_ERR_ARG;
  const int nrows = t->n_knots * 2 * (t->K + 1);
  if (nrows > kNcx2TabMaxRows) return AICDF_ERR_UNSUPPORTED;
  a->K = t->K;
  a->n_knots = t->n_knots;
  a->nu = (float)t->nu;
  a->scale_k = std::ldexp(1.0f, t->K);
  for (int r = 0; r < nrows; ++r)
    a->rows[r] = make_float4(t->coef32[4 * r], t->coef32[4 * r + 1], t->coef32[4 * r + 2], t->coef32[4 * r + 3]);
  return AICDF_OK;
}

double ncx2_table_nu(const aicdf_ncx2_table_s *t) { return t->nu; }

__global__ void __launch_bounds__(256) k_ncx2_table_eval(const __grid_constant__ Ncx2TabArgs a,
                                                          const float *__restrict__ u,
                                                          const float *__restrict__ lam, uint64_t n,
                                                          float *__restrict__ out) {
  __shared__ float4 s_rows[kNcx2TabMaxRows];
  const int nrows = a.n_knots * 2 * (a.K + 1);
  for (int r = threadIdx.x; r < nrows; r += blockDim.x) s_rows[r] = a.rows[r];
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float ui = u[i], li = lam[i];
    float y = ncx2_table_ppf(s_rows, a.K, a.n_knots, a.nu, a.scale_k, ui, li);
    if (!(ui >= 0.0f && ui <= 1.0f) || !(li >= 0.0f) || isinf(li)) y = __int_as_float(0x7fc00000);
    out[i] = y;
  }
}

}  // namespace aicdf

using namespace aicdf;

extern "C" aicdf_status aicdf_ncx2_table_build(double nu, int K, int n_knots, int degree,
                                               aicdf_ncx2_table *out) {
  if (!out) return AICDF_ERR_ARG;
  *out = nullptr;
  if (!(nu > 0.0) || !std::isfinite(nu) || K < 1 || K > 30 || n_knots < 2 || n_knots > 64 || degree < 1 ||
      degree > 3)
    return AICDF_ERR_ARG;
  aicdf_ncx2_table_s *t = new (std::nothrow) aicdf_ncx2_table_s();
  if (!t) return AICDF_ERR_NOMEM;
  t->magic = kNcx2TableMagic;
  t->nu = nu;
  t->K = K;
  t->n_knots = n_knots;
  t->degree = degree;
  t->coef.assign((size_t)n_knots * 2 * (K + 1) * 4, 0.0);
  // knots are independent: one host thread each
  std::vector<int> status(n_knots, 0);
  std::vector<std::thread> pool;
  for (int i = 0; i < n_knots; ++i) pool.emplace_back(build_knot, t, i, &status[i]);
  for (auto &th : pool) th.join();
  t->coef32.assign(t->coef.begin(), t->coef.end());
  int any = 0;
  for (int s : status) any |= s;
  if (any) {
    delete t;
    return AICDF_ERR_DOMAIN;  // the exact quantile did not converge at a quadrature node
  }
  *out = t;
  return AICDF_OK;
}

extern "C" void aicdf_ncx2_table_destroy(aicdf_ncx2_table t) {
  if (ncx2_table_ok(t)) {
    t->magic = 0;
    delete t;
  }
}

extern "C" aicdf_status aicdf_ncx2_table_info(aicdf_ncx2_table t, double *nu, int *K, int *n_knots, int *degree) {
  if (!ncx2_table_ok(t)) return AICDF_ERR_ARG;
  if (nu) *nu = t->nu;
  if (K) *K = t->K;
  if (n_knots) *n_knots = t->n_knots;
  if (degree) *degree = t->degree;
  return AICDF_OK;
}

extern "C" aicdf_status aicdf_ncx2_table_get(aicdf_ncx2_table t, double *coef, size_t cap, size_t *n_out) {
  if (!ncx2_table_ok(t)) return AICDF_ERR_ARG;
  if (n_out) *n_out = t->coef.size();
  if (!coef) return AICDF_OK;
  if (cap < t->coef.size()) return AICDF_ERR_ARG;
  std::memcpy(coef, t->coef.data(), t->coef.size() * sizeof(double));
  return AICDF_OK;
}

extern "C" aicdf_status aicdf_ncx2_table_eval(aicdf_ncx2_table t, const float *u_dev, const float *lam_dev, size_t n,
                                              float *out_dev, aicdf_stream_t stream) {
  static thread_local Ncx2TabArgs a;  // 16 KiB: keep it off the stack
  aicdf_status s = pack_ncx2_table(t, &a);
  if (s != AICDF_OK) return s;
  if (n == 0) return AICDF_OK;
  if (!u_dev || !lam_dev || !out_dev || ((uintptr_t)u_dev % 4) || ((uintptr_t)lam_dev % 4) ||
      ((uintptr_t)out_dev % 4))
    return AICDF_ERR_ARG;
  const uint64_t want = (n + 255) / 256;
  const uint64_t cap = (uint64_t)sm_count() * resident_blocks((const void *)k_ncx2_table_eval, 256);
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min(want, cap));
  k_ncx2_table_eval<<<grid, 256, 0, (cudaStream_t)stream>>>(a, u_dev, lam_dev, n, out_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error((int)e);
    return AICDF_ERR_CUDA;
  }
  return AICDF_OK;
}
