// Host MLMC driver (Section 4.1): pilot runs, Lagrange-optimal path counts
// from measured variances and per-path device costs, and levels added until
// the bias estimate is below eps / sqrt(2).  Every path launch goes through
// aicdf_mlmc_level; sums come back to the host once per launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "aicdf_internal.h"

namespace {

struct Term {
  int level = 0, kind = 0, slot = 0;
  uint32_t tag = 0;
  uint64_t n = 0;
  double s1 = 0.0, s2 = 0.0;
  double ns_per_path = 0.0;   // from the largest launch so far
  uint64_t cost_launch = 0;   // size of that launch
  double mean() const { return n ? s1 / (double)n : 0.0; }
  double var() const {
    if (n < 2) return 0.0;
    const double m = s1 / (double)n;
    return std::max(s2 / (double)n - m * m, 0.0) * (double)n / (double)(n - 1);
  }
};

struct Ctx {
  const aicdf_sde_params *prm;
  aicdf_table tab;
  uint64_t seed;
  double *sums_dev;
  void *ws;
  size_t ws_bytes;
  cudaStream_t st;
  cudaEvent_t e0, e1;
  double gpu_ms = 0.0;
  int launches = 0;
};

constexpr uint64_t kMaxPathsPerLaunch = 1ull << 32;

aicdf_status extend(Ctx &c, Term &t, uint64_t add) {
  while (add > 0) {
    const uint64_t m = std::min(add, kMaxPathsPerLaunch);
    if (cudaEventRecord(c.e0, c.st) != cudaSuccess) return AICDF_ERR_CUDA;
    aicdf_status s = aicdf_mlmc_level(c.prm, c.tab, t.level, t.kind, m, t.n, c.seed, t.tag,
                                      c.sums_dev, c.ws, c.ws_bytes, (aicdf_stream_t)c.st);
    if (s != AICDF_OK) return s;
    double h[3];
    if (cudaEventRecord(c.e1, c.st) != cudaSuccess ||
        cudaMemcpyAsync(h, c.sums_dev, sizeof(h), cudaMemcpyDeviceToHost, c.st) != cudaSuccess ||
        cudaStreamSynchronize(c.st) != cudaSuccess) {
      aicdf::set_cuda_error((int)cudaGetLastError());
      return AICDF_ERR_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c.e0, c.e1);
    c.gpu_ms += ms;
    c.launches += 1;
    t.s1 += h[0];
    t.s2 += h[1];
    t.n += m;
    if (m >= t.cost_launch) {
      t.cost_launch = m;
      t.ns_per_path = std::max((double)ms * 1e6 / (double)m, 1e-6);
    }
    add -= m;
  }
  return AICDF_OK;
}

}  // namespace

extern "C" size_t aicdf_mlmc_run_workspace_bytes(void) {
  return aicdf_mlmc_level_workspace_bytes() + 256;
}

extern "C" aicdf_status aicdf_mlmc_run(const aicdf_sde_params *params, aicdf_table approx,
                                       const aicdf_mlmc_opts *o, aicdf_mlmc_result *r,
                                       void *workspace_dev, size_t workspace_bytes,
                                       aicdf_stream_t stream) {
  if (!params || !o || !r || !workspace_dev) return AICDF_ERR_ARG;
  if (!aicdf::table_ok(approx)) return AICDF_ERR_ARG;
  if (!(o->eps > 0.0) || o->L_min < 0 || o->L_max < o->L_min || o->L_max >= AICDF_MAX_LEVELS ||
      o->L_max > 20 || o->fixed_L >= AICDF_MAX_LEVELS || o->fixed_L > 20)
    return AICDF_ERR_ARG;
  if (o->estimator < AICDF_EST_NESTED || o->estimator > AICDF_EST_PLAIN) return AICDF_ERR_ARG;
  if (o->estimator == AICDF_EST_PLAIN && o->fixed_L < 0) return AICDF_ERR_ARG;
  if (workspace_bytes < aicdf_mlmc_run_workspace_bytes() || ((uintptr_t)workspace_dev % 256))
    return AICDF_ERR_ARG;
  const auto wall0 = std::chrono::steady_clock::now();
  std::memset(r, 0, sizeof(*r));
  Ctx c;
  c.prm = params;
  c.tab = approx;
  c.seed = o->seed;
  c.ws = workspace_dev;
  c.ws_bytes = aicdf_mlmc_level_workspace_bytes();
  c.sums_dev = reinterpret_cast<double *>((char *)workspace_dev + c.ws_bytes);
  c.st = (cudaStream_t)stream;
  if (cudaEventCreate(&c.e0) != cudaSuccess || cudaEventCreate(&c.e1) != cudaSuccess) {
    aicdf::set_cuda_error((int)cudaGetLastError());
    return AICDF_ERR_CUDA;
  }
  const uint64_t pilot = o->n_pilot ? o->n_pilot : 10000;
  const double alpha = o->weak_order > 0.0 ? o->weak_order : 1.0;
  const int est = o->estimator;
  std::vector<Term> terms;
  auto add_level = [&](int l) -> aicdf_status {
    std::vector<int> kinds;
    if (est == AICDF_EST_NESTED) kinds = {AICDF_KIND_APPROX2, AICDF_KIND_CORR4};
    else if (est == AICDF_EST_REGULAR) kinds = {AICDF_KIND_EXACT2};
    else kinds = {AICDF_KIND_PLAIN};
    for (size_t i = 0; i < kinds.size(); ++i) {
      Term t;
      t.level = l;
      t.kind = kinds[i];
      t.slot = (int)i;
      t.tag = 1u + 64u * (uint32_t)est + 2u * (uint32_t)l + (uint32_t)i;
      terms.push_back(t);
      aicdf_status s = extend(c, terms.back(), pilot);
      if (s != AICDF_OK) return s;
    }
    return AICDF_OK;
  };
  aicdf_status s = AICDF_OK;
  int L;
  if (est == AICDF_EST_PLAIN) {
    L = o->fixed_L;
    s = add_level(L);
  } else {
    L = o->fixed_L >= 0 ? o->fixed_L : o->L_min;
    for (int l = 0; l <= L && s == AICDF_OK; ++l) s = add_level(l);
  }
  bool converged = false;
  const double eps = o->eps;
  while (s == AICDF_OK) {
    // optimal counts for the current set of terms (Section 4.1)
    std::vector<double> v, cst, m(terms.size());
    for (auto &t : terms) {
      v.push_back(t.var());
      cst.push_back(t.ns_per_path);
    }
    double total = 0.0;
    s = aicdf_mlmc_allocate((int)terms.size(), v.data(), cst.data(), eps, m.data(), &total);
    if (s != AICDF_OK) break;
    for (size_t i = 0; i < terms.size() && s == AICDF_OK; ++i) {
      const double want = std::ceil(m[i]);
      if (!(want < 1e15)) {
        s = AICDF_ERR_NOCONVERGE;
        break;
      }
      if ((uint64_t)want > terms[i].n) s = extend(c, terms[i], (uint64_t)want - terms[i].n);
    }
    if (s != AICDF_OK) break;
    if (est == AICDF_EST_PLAIN || o->fixed_L >= 0) {
      converged = true;
      break;
    }
    // bias estimate from the two finest levels' total corrections
    auto level_mean = [&](int l) {
      double mm = 0.0;
      for (auto &t : terms)
        if (t.level == l) mm += t.mean();
      return mm;
    };
    const double a2 = std::pow(2.0, alpha);
    double bias = std::fabs(level_mean(L)) / (a2 - 1.0);
    if (L > 0) bias = std::max(bias, std::fabs(level_mean(L - 1)) / a2 / (a2 - 1.0));
    r->bias = bias;
    if (bias <= eps / std::sqrt(2.0)) {
      converged = true;
      break;
    }
    if (L >= o->L_max) break;
    ++L;
    s = add_level(L);
  }
  cudaEventDestroy(c.e0);
  cudaEventDestroy(c.e1);
  if (s != AICDF_OK) return s;
  double estv = 0.0, var = 0.0;
  for (auto &t : terms) {
    estv += t.mean();
    var += t.n ? t.var() / (double)t.n : 0.0;
    r->paths[t.level][t.slot] = t.n;
    r->mean[t.level][t.slot] = t.mean();
    r->var[t.level][t.slot] = t.var();
    r->cost_ns[t.level][t.slot] = t.ns_per_path;
  }
  r->estimate = estv;
  r->variance = var;
  r->L = L;
  r->converged = converged ? 1 : 0;
  r->n_terms = est == AICDF_EST_NESTED ? 2 : 1;
  r->gpu_ms = c.gpu_ms;
  r->launches = c.launches;
  r->wall_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
  return AICDF_OK;
}
