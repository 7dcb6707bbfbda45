// CIR paths with exact non-central chi-squared transitions vs approximate ones
// driven by the same uniforms (Section 5.2).
//
// Over a step h the CIR law is X' = c chi'^2_nu(lambda) with c = sigma^2 (1 - e^{-kappa h}) /
// (4 kappa), nu = 4 kappa theta / sigma^2 and lambda = X e^{-kappa h} / c (the
// horizon-T law of Section 5.2 applied per step).  Exact: X' = c C^{-1}_nu(U; lambda)
// by the FP64 root finder.  Approximate: X' = c max(C~^{-1}_nu(U; lambda), 0) with
// C~^{-1} = lambda + nu + 2 sqrt(lambda + nu) P~ and P~ either the learned
// surrogate P~ = Phi^{-1}(U) + sqrt(y) N (tensor-core MLP, one warp = 32
// paths; y = nu / (lambda + nu)) or, for comparison, the limit P ->
// Phi^{-1}(U) of Section 5.1.  As in the paper's CIR experiment the
// two-way difference uses the same time step on both sides.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "aicdf_internal.h"
#include "device_common.cuh"
#include "mlmc_path.cuh"
#include "mlp_device.cuh"
#include "ncx2.cuh"
#include "ncx2_table.cuh"

namespace aicdf {

constexpr int kCirThreads = 256;

struct CirArgs {
  PhiloxKeys keys;
  const float *params;  // surrogate weights (may be null for kinds without it)
  uint64_t n_paths, path_offset;
  uint32_t tag;
  uint32_t lanes;       // active lanes per warp (1..32)
  int level, kind, payoff;
  double nu, c, e;      // chi^2 scale, degrees of freedom, e^{-kappa h}
  float X0, K, discount;
};

struct NoTab {};

// APPROX: 0 none, 1 surrogate, 2 Gaussian limit, 3 table (TabT = Ncx2TabArgs)
template <bool EXACT, int APPROX, class TabT>
__global__ void __launch_bounds__(kCirThreads)
    k_cir(const __grid_constant__ CirArgs a, const __grid_constant__ TabT tab, Moments *__restrict__ partials,
          int *__restrict__ status) {
  __shared__ __align__(16) MlpSmem s;
  __shared__ __align__(16) __nv_bfloat16 hs[APPROX == 1 ? kCirThreads / 32 : 1][32 * kHPad];
  __shared__ Moments s_red[kCirThreads / 32];
  __shared__ float4 s_rows[APPROX == 3 ? kNcx2TabMaxRows : 1];
  if constexpr (APPROX == 1) {
    mlp_stage(a.params, s);
    __syncthreads();
  }
  if constexpr (APPROX == 3) {
    const int nrows = tab.n_knots * 2 * (tab.K + 1);
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) s_rows[r] = tab.rows[r];
    __syncthreads();
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nsteps = 1 << a.level;
  const float cf = (float)a.c, nuf = (float)a.nu, ratio = (float)(a.e / a.c);
  // a warp takes a.lanes consecutive paths per iteration (32 unless the term
  // is small; the surrogate's warp-wide MLP always runs all 32 lanes)
  const uint64_t L = APPROX == 1 ? 32u : a.lanes;
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t stride = (((uint64_t)gridDim.x * blockDim.x) >> 5) * L;
  int st = 0;
  PathSums acc;
  chunked_loop(gw * L, a.n_paths, stride, kChunkPaths, acc, [&](uint64_t base) {  // warp-uniform
    const uint64_t i = base + lane;
    const bool active = (uint64_t)lane < L && i < a.n_paths;
    const uint64_t p = a.path_offset + i;
    double xe = a.X0, se = 0.0;  // the path and (ASIAN) the sum of its post-step values
    float xa = a.X0, sa = 0.f;
    const PhiloxPath pp = philox_path((uint32_t)p, (uint32_t)(p >> 32), a.keys);
    for (int s4 = 0; s4 < nsteps && (active || APPROX == 1); s4 += 4) {
      const uint4 r = philox_path_call((uint32_t)(s4 >> 2), a.tag, pp, a.keys);
      const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (s4 + t < nsteps) {
          const float u = u01(w[t]);
          if (EXACT) {
            const double lam = xe * a.e / a.c;
            xe = a.c * ncx2_ppf((double)u, a.nu, lam, &st);
            se += xe;
          }
          if (APPROX != 0) {
            const float lam = fmaxf(xa, 0.f) * ratio;
            float pt;
            if constexpr (APPROX == 1) {
              const float sy = mlp_sqrt_y(lam, nuf);
              pt = fmaf(sy, mlp_forward_warp(s, mlp_feature_u(u), mlp_feature_y(sy), hs[warp]), phiinv_f32_grid(u));
            } else if constexpr (APPROX == 3) {
              pt = ncx2_table_P(s_rows, tab.K, tab.n_knots, tab.scale_k, u, sqrtf(nuf / (lam + nuf)));
            } else {
              pt = phiinv_f32_grid(u);
            }
            const float h = lam + nuf;
            xa = cf * fmaxf(fmaf(2.0f * sqrtf(h), pt, h), 0.f);
            sa += xa;
          }
        }
      }
    }
    float y;
    const float inv_n = 1.0f / (float)nsteps;  // exact: nsteps is a power of two
    const float pe = a.payoff == AICDF_PAYOFF_CALL    ? a.discount * fmaxf((float)xe - a.K, 0.f)
                     : a.payoff == AICDF_PAYOFF_ASIAN ? a.discount * ((float)se * inv_n)
                                                      : a.discount * (float)xe;
    const float pa = a.payoff == AICDF_PAYOFF_CALL    ? a.discount * fmaxf(xa - a.K, 0.f)
                     : a.payoff == AICDF_PAYOFF_ASIAN ? a.discount * (sa * inv_n)
                                                      : a.discount * xa;
    if (EXACT && APPROX != 0) y = pe - pa;
    else if (EXACT) y = pe;
    else y = pa;
    acc.add(y, active);
  });
  const Moments tot = block_reduce_moments(acc.total(), s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
  if (st) atomicOr(status, st);
}

using CirFn = void (*)(CirArgs, NoTab, Moments *, int *);
using CirTabFn = void (*)(CirArgs, Ncx2TabArgs, Moments *, int *);

static CirFn select_cir(int kind) {
  switch (kind) {
    case AICDF_CIR_EXACT: return k_cir<true, 0, NoTab>;
    case AICDF_CIR_SURROGATE: return k_cir<false, 1, NoTab>;
    case AICDF_CIR_DIFF: return k_cir<true, 1, NoTab>;
    case AICDF_CIR_GAUSS: return k_cir<false, 2, NoTab>;
    default: return k_cir<true, 2, NoTab>;
  }
}

const float *surrogate_params(aicdf_surrogate s);
double surrogate_nu(aicdf_surrogate s);
bool surrogate_ok(aicdf_surrogate s);
aicdf_status pack_ncx2_table(const aicdf_ncx2_table_s *t, Ncx2TabArgs *a);
double ncx2_table_nu(const aicdf_ncx2_table_s *t);

// Argument checks and the per-level constants shared by both entry points.
static aicdf_status cir_setup(const aicdf_sde_params *prm, int level, uint64_t n_paths, uint64_t path_offset,
                              uint64_t seed, uint32_t tag, int kind, double *sums_dev, void *workspace_dev,
                              size_t workspace_bytes, int *status_dev, CirArgs *a) {
  if (!prm || prm->model != AICDF_MODEL_CIR) return AICDF_ERR_ARG;
  if (level < 0 || level > 12) return AICDF_ERR_ARG;
  if (n_paths == 0 || path_offset + n_paths < path_offset) return AICDF_ERR_ARG;
  if (!sums_dev || ((uintptr_t)sums_dev % 8) || !status_dev) return AICDF_ERR_ARG;
  if (!workspace_dev || ((uintptr_t)workspace_dev % 16) || workspace_bytes < aicdf_mlmc_level_workspace_bytes())
    return AICDF_ERR_ARG;
  if (prm->payoff != AICDF_PAYOFF_X && prm->payoff != AICDF_PAYOFF_CALL && prm->payoff != AICDF_PAYOFF_ASIAN)
    return AICDF_ERR_ARG;
  if (!(prm->kappa > 0.0) || !(prm->theta > 0.0) || !(prm->sigma > 0.0) || !(prm->T > 0.0) ||
      !(prm->X0 >= 0.0) || !std::isfinite(prm->X0 + prm->T + prm->K + prm->discount))
    return AICDF_ERR_DOMAIN;
  std::memset(a, 0, sizeof(*a));
  const double h = prm->T / std::ldexp(1.0, level);
  a->keys = make_keys(seed);
  a->n_paths = n_paths;
  a->path_offset = path_offset;
  a->tag = tag;
  a->level = level;
  a->kind = kind;
  a->payoff = prm->payoff;
  a->nu = 4.0 * prm->kappa * prm->theta / (prm->sigma * prm->sigma);
  a->e = std::exp(-prm->kappa * h);
  a->c = prm->sigma * prm->sigma * (-std::expm1(-prm->kappa * h)) / (4.0 * prm->kappa);
  a->X0 = (float)prm->X0;
  a->K = (float)prm->K;
  a->discount = (float)prm->discount;
  return AICDF_OK;
}

// Launch shape.  With paths to fill every SM with full blocks: 256 threads,
// 32 paths per warp.  A smaller term is spread over all SMs, and -- for the
// kinds without the warp-wide MLP -- over all four SM sub-partitions too: one
// warp of 128-thread blocks per sub-partition, each warp taking
// ceil(n / (4 SMs)) paths on that many lanes.  An exact step is a serial chain
// of FP64 operations, and each sub-partition has its own share of the SM's
// FP64 rate, so a small exact term finishes up to 4x sooner that way.
template <class Fn, class TabT>
static aicdf_status cir_launch(Fn k, CirArgs a, const TabT &tab, bool warp_mlp, uint64_t n_paths,
                               void *workspace_dev, double *sums_dev, int *status_dev, cudaStream_t st) {
  const uint64_t sms = (uint64_t)sm_count();
  constexpr uint64_t kSubPartitions = 4;
  int threads = kCirThreads;
  a.lanes = 32;
  uint64_t want;
  if (!warp_mlp && n_paths < sms * kSubPartitions * 32) {
    a.lanes = (uint32_t)((n_paths + sms * kSubPartitions - 1) / (sms * kSubPartitions));  // 1..32
    threads = 128;
    const uint64_t warps = (n_paths + a.lanes - 1) / a.lanes;
    want = (warps + 3) / 4;
  } else {
    if (n_paths < sms * kCirThreads) {
      const uint64_t per_sm = (n_paths + sms - 1) / sms;
      threads = (int)std::min<uint64_t>(kCirThreads, std::max<uint64_t>(32, (per_sm + 31) / 32 * 32));
    }
    want = (n_paths + threads - 1) / threads;
  }
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(
      want, std::min<uint64_t>(sms * resident_blocks((const void *)k, threads), 4096)));
  Moments *parts = reinterpret_cast<Moments *>(workspace_dev);
  k<<<grid, threads, 0, st>>>(a, tab, parts, status_dev);
  launch_reduce_partials(parts, grid, (double)n_paths, sums_dev, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error((int)e);
    return AICDF_ERR_CUDA;
  }
  return AICDF_OK;
}

}  // namespace aicdf

using namespace aicdf;

extern "C" aicdf_status aicdf_cir_level(const aicdf_sde_params *prm, aicdf_surrogate sur, int level, int kind,
                                        uint64_t n_paths, uint64_t path_offset, uint64_t seed, uint32_t tag,
                                        double *sums_dev, void *workspace_dev, size_t workspace_bytes,
                                        int *status_dev, aicdf_stream_t stream) {
  if (kind < AICDF_CIR_EXACT || kind > AICDF_CIR_DIFF_GAUSS) return AICDF_ERR_ARG;
  CirArgs a;
  aicdf_status s = cir_setup(prm, level, n_paths, path_offset, seed, tag, kind, sums_dev, workspace_dev,
                             workspace_bytes, status_dev, &a);
  if (s != AICDF_OK) return s;
  if (kind == AICDF_CIR_SURROGATE || kind == AICDF_CIR_DIFF) {
    if (!surrogate_ok(sur)) return AICDF_ERR_ARG;
    if (std::fabs(surrogate_nu(sur) - a.nu) > 1e-9 * a.nu) return AICDF_ERR_DOMAIN;  // trained for another nu
    a.params = surrogate_params(sur);
  }
  const bool mlp = kind == AICDF_CIR_SURROGATE || kind == AICDF_CIR_DIFF;
  return cir_launch(select_cir(kind), a, NoTab{}, mlp, n_paths, workspace_dev, sums_dev, status_dev,
                    (cudaStream_t)stream);
}

extern "C" aicdf_status aicdf_cir_level_table(const aicdf_sde_params *prm, aicdf_ncx2_table table, int level,
                                              int kind, uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                                              uint32_t tag, double *sums_dev, void *workspace_dev,
                                              size_t workspace_bytes, int *status_dev, aicdf_stream_t stream) {
  if (kind != AICDF_CIR_EXACT && kind != AICDF_CIR_TABLE && kind != AICDF_CIR_DIFF_TABLE) return AICDF_ERR_ARG;
  CirArgs a;
  aicdf_status s = cir_setup(prm, level, n_paths, path_offset, seed, tag, kind, sums_dev, workspace_dev,
                             workspace_bytes, status_dev, &a);
  if (s != AICDF_OK) return s;
  static thread_local Ncx2TabArgs tab;  // 16 KiB: keep it off the stack
  s = pack_ncx2_table(table, &tab);
  if (s != AICDF_OK) return s;
  if (std::fabs(ncx2_table_nu(table) - a.nu) > 1e-9 * a.nu) return AICDF_ERR_DOMAIN;  // built for another nu
  CirTabFn k = kind == AICDF_CIR_EXACT ? k_cir<true, 0, Ncx2TabArgs>
               : kind == AICDF_CIR_TABLE ? k_cir<false, 3, Ncx2TabArgs>
                                         : k_cir<true, 3, Ncx2TabArgs>;
  return cir_launch(k, a, tab, false, n_paths, workspace_dev, sums_dev, status_dev, (cudaStream_t)stream);
}
