// Fused nested-MLMC level kernel (Section 4, Section 4.1).
//
// One thread simulates one path at a time, entirely in registers: every fine
// step draws one Philox uniform U, and from that same U the exact variate
// Z = Phi^{-1}(U) and/or the approximate variate Z~ = D(U) (or Q(U)); the fine
// exact and approximate states advance with Z and Z~, and every second step
// the coarse states advance with the pairwise sums (Section 4.1: coarse
// Wiener increments are pairwise sums of the fine ones).  The payoff
// difference Y of the requested estimator kind is accumulated per thread in
// FP32 over a chunk of paths and flushed to FP64; warps reduce in FP64 by
// shuffles, blocks write one FP64 partial each, and a second one-block
// kernel adds the partials in a fixed order, so sums are deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "aicdf_internal.h"
#include "device_common.cuh"
#include "mlmc_path.cuh"

namespace aicdf {

constexpr int kLevelThreads = 256;
constexpr int kMaxLevelBlocks = 4096;
constexpr int kFlushEvery = 16;  // paths per FP32 chunk before the FP64 flush

template <bool NE, bool NA, int AP, int MODEL, int SCHEME>
__global__ void __launch_bounds__(kLevelThreads)
    k_mlmc_level(const __grid_constant__ LevelArgs a, double2 *__restrict__ partials) {
  __shared__ float s_tab[AP == AICDF_PWC ? 1024 : 1];
  __shared__ double2 s_red[kLevelThreads / 32];
  const ApproxTable<AP> ap(a.tab, a.ntab, s_tab);
  const PathConsts pc = make_path_consts(a);
  const int lane = threadIdx.x & 31;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  float f1 = 0.f, f2 = 0.f;
  double d1 = 0.0, d2 = 0.0;
  int chunk = 0;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < a.n_paths;
       base += stride) {
    const uint64_t i = base + lane;
    const uint64_t p = a.path_offset + i;
    const float y = path_y<NE, NA, AP, MODEL, SCHEME>(a, pc, ap, p);
    if (i < a.n_paths) {
      f1 += y;
      f2 = fmaf(y, y, f2);
    }
    if (++chunk == kFlushEvery) {
      d1 += (double)f1;
      d2 += (double)f2;
      f1 = f2 = 0.f;
      chunk = 0;
    }
  }
  d1 += (double)f1;
  d2 += (double)f2;
  const double2 t = block_reduce2(d1, d2, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// Fixed-order sum of the per-block partials (one block).
__global__ void __launch_bounds__(256) k_reduce_partials(const double2 *__restrict__ partials,
                                                         int nparts, double count,
                                                         double *__restrict__ sums) {
  __shared__ double2 s_red[256 / 32];
  double d1 = 0.0, d2 = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    d1 += partials[i].x;
    d2 += partials[i].y;
  }
  const double2 t = block_reduce2(d1, d2, s_red);
  if (threadIdx.x == 0) {
    sums[0] = t.x;
    sums[1] = t.y;
    sums[2] = count;
  }
}

using LevelFn = void (*)(LevelArgs, double2 *);

template <bool NE, bool NA, int AP>
LevelFn pick_ms(int model, int scheme) {
  if (model == AICDF_MODEL_GBM)
    return scheme == AICDF_SCHEME_EM ? (LevelFn)k_mlmc_level<NE, NA, AP, AICDF_MODEL_GBM, AICDF_SCHEME_EM>
                                     : (LevelFn)k_mlmc_level<NE, NA, AP, AICDF_MODEL_GBM, AICDF_SCHEME_MILSTEIN>;
  return scheme == AICDF_SCHEME_EM ? (LevelFn)k_mlmc_level<NE, NA, AP, AICDF_MODEL_CIR, AICDF_SCHEME_EM>
                                   : (LevelFn)k_mlmc_level<NE, NA, AP, AICDF_MODEL_CIR, AICDF_SCHEME_MILSTEIN>;
}

template <bool NE, bool NA>
LevelFn pick_ap(int ap, int model, int scheme) {
  return ap == AICDF_PWL ? pick_ms<NE, NA, AICDF_PWL>(model, scheme) : pick_ms<NE, NA, AICDF_PWC>(model, scheme);
}

static LevelFn select_level_kernel(int kind, int ap, int model, int scheme) {
  const bool ne = kind_needs_exact(kind), na = kind_needs_approx(kind);
  if (ne && na) return pick_ap<true, true>(ap, model, scheme);
  if (ne) return pick_ap<true, false>(ap, model, scheme);
  return pick_ap<false, true>(ap, model, scheme);
}

aicdf_status prepare_level_args(const aicdf_sde_params *prm, aicdf_table approx, int level,
                                int kind, uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                                uint32_t tag, LevelArgs *a) {
  if (!prm || !table_ok(approx)) return AICDF_ERR_ARG;
  if (level < 0 || level > 20) return AICDF_ERR_ARG;
  if (kind < AICDF_KIND_APPROX2 || kind > AICDF_KIND_PLAIN_APPROX) return AICDF_ERR_ARG;
  if (prm->model != AICDF_MODEL_GBM && prm->model != AICDF_MODEL_CIR) return AICDF_ERR_ARG;
  if (prm->scheme != AICDF_SCHEME_EM && prm->scheme != AICDF_SCHEME_MILSTEIN) return AICDF_ERR_ARG;
  if (prm->payoff != AICDF_PAYOFF_X && prm->payoff != AICDF_PAYOFF_CALL) return AICDF_ERR_ARG;
  if (n_paths == 0) return AICDF_ERR_ARG;
  if (path_offset + n_paths < path_offset) return AICDF_ERR_ARG;  // wraps
  const double vals[] = {prm->X0, prm->T, prm->K, prm->mu, prm->sigma, prm->kappa, prm->theta,
                         prm->discount};
  for (double v : vals)
    if (!std::isfinite(v)) return AICDF_ERR_DOMAIN;
  if (!(prm->T > 0.0) || prm->sigma < 0.0) return AICDF_ERR_DOMAIN;
  if (prm->model == AICDF_MODEL_CIR && (prm->kappa < 0.0 || prm->theta < 0.0)) return AICDF_ERR_DOMAIN;
  std::memset(a, 0, sizeof(*a));
  a->keys = make_keys(seed);
  a->n_paths = n_paths;
  a->path_offset = path_offset;
  a->tag = tag;
  a->level = level;
  a->kind = kind;
  a->model = prm->model;
  a->scheme = prm->scheme;
  a->payoff = prm->payoff;
  a->approx = approx->method;
  a->X0 = (float)prm->X0;
  a->K = (float)prm->K;
  a->discount = (float)prm->discount;
  a->mu = (float)prm->mu;
  a->sigma = (float)prm->sigma;
  a->kappa = (float)prm->kappa;
  a->theta = (float)prm->theta;
  a->dt = (float)(prm->T / std::ldexp(1.0, level));
  if (approx->method == AICDF_PWL) {
    if (approx->n > 15) return AICDF_ERR_UNSUPPORTED;
    for (int i = 0; i < 16; ++i) {
      const int r = std::min(i, approx->n);
      a->tab[i] = approx->f0[r];
      a->tab[16 + i] = approx->f1[r];
    }
  } else {
    if (approx->n > 1024) return AICDF_ERR_UNSUPPORTED;
    for (int i = 0; i < approx->n; ++i) a->tab[i] = approx->f0[i];
    a->nf = (float)approx->n;
  }
  a->ntab = approx->n;
  return AICDF_OK;
}

int level_grid(uint64_t n_paths) {
  const uint64_t want = (n_paths + kLevelThreads - 1) / kLevelThreads;
  const uint64_t cap = (uint64_t)sm_count() * (2048 / kLevelThreads);
  uint64_t g = std::min<uint64_t>(want, std::min<uint64_t>(cap, kMaxLevelBlocks));
  return (int)std::max<uint64_t>(g, 1);
}

aicdf_status launch_level(const LevelArgs &a, int kind, double *sums_dev, void *ws,
                          cudaStream_t st) {
  LevelFn k = select_level_kernel(kind, a.approx, a.model, a.scheme);
  const int grid = level_grid(a.n_paths);
  double2 *parts = reinterpret_cast<double2 *>(ws);
  k<<<grid, kLevelThreads, 0, st>>>(a, parts);
  k_reduce_partials<<<1, 256, 0, st>>>(parts, grid, (double)a.n_paths, sums_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error((int)e);
    return AICDF_ERR_CUDA;
  }
  return AICDF_OK;
}

}  // namespace aicdf

using namespace aicdf;

extern "C" size_t aicdf_mlmc_level_workspace_bytes(void) {
  return sizeof(double2) * (size_t)kMaxLevelBlocks;
}

extern "C" aicdf_status aicdf_mlmc_level(const aicdf_sde_params *params, aicdf_table approx,
                                         int level, int kind, uint64_t n_paths,
                                         uint64_t path_offset, uint64_t seed, uint32_t tag,
                                         double *sums_dev, void *workspace_dev,
                                         size_t workspace_bytes, aicdf_stream_t stream) {
  static thread_local LevelArgs a;
  aicdf_status s = prepare_level_args(params, approx, level, kind, n_paths, path_offset, seed,
                                      tag, &a);
  if (s != AICDF_OK) return s;
  if (!sums_dev || ((uintptr_t)sums_dev % 8)) return AICDF_ERR_ARG;
  if (!workspace_dev || ((uintptr_t)workspace_dev % 16)) return AICDF_ERR_ARG;
  if (workspace_bytes < aicdf_mlmc_level_workspace_bytes()) return AICDF_ERR_ARG;
  return launch_level(a, kind, sums_dev, workspace_dev, (cudaStream_t)stream);
}
