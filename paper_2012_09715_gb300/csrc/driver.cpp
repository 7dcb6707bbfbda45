// Host MLMC driver (Section 4.1): pilot runs, Lagrange-optimal path counts
// from measured variances and per-path device costs, and levels added until
// the bias estimate is below eps / sqrt(2).
//
// Each round is one batched persistent launch: the pilot paths of every new
// level in one, the extra paths of every term in the next.  Per-path costs
// for the allocation come from a per-step cost of each estimator kind,
// calibrated once per process, device and model by timing one large level
// launch of that kind, times (2^l + 1) steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "aicdf_internal.h"

namespace {

struct Term {
  int level = 0, kind = 0, slot = 0;
  bool active = true;  // false: a nested pair the adaptive estimator replaced by an exact term
  uint32_t tag = 0;
  uint64_t n = 0;
  double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
  double mean() const { return n ? s1 / (double)n : 0.0; }
  double var() const {
    if (n < 2) return 0.0;
    const double m = s1 / (double)n;
    return std::max(s2 / (double)n - m * m, 0.0) * (double)n / (double)(n - 1);
  }
  // Kurtosis E[(Y - EY)^4] / Var(Y)^2 from the four power sums (3 for a
  // Gaussian Y; 0 when it cannot be formed).
  double kurt() const {
    if (n < 4) return 0.0;
    const double N = (double)n, m = s1 / N, e2 = s2 / N, e3 = s3 / N, e4 = s4 / N;
    const double v = e2 - m * m;
    if (!(v > 0.0)) return 0.0;
    const double c4 = e4 - 4.0 * m * e3 + 6.0 * m * m * e2 - 3.0 * m * m * m * m;
    return std::max(c4, 0.0) / (v * v);
  }
  void add_sums(const double *h, uint64_t paths) {
    s1 += h[0];
    s2 += h[1];
    s3 += h[2];
    s4 += h[3];
    n += paths;
  }
};

// The sample variance of n paths of a term with kurtosis k has relative
// standard error about sqrt((k - 1) / n).  The optimal allocation (Section
// 4.1) trusts each term's variance; what matters is the error that a term's
// variance estimate puts into the estimator's variance sum_i V_i / n_i, in
// which the term has the share f = (V / n) / sum.  So a term keeps at least
// the paths that make f sqrt((k - 1) / n) <= 1/4, n >= (k - 1) (4 f)^2: a
// heavy-tailed term (the four-way corrections, whose Y is the rare large
// difference between exact and approximate paths) with a real share of the
// variance gets enough paths to be measured, and one whose share is tiny
// costs nothing extra.
constexpr double kVarRelErr = 0.25;
uint64_t kurtosis_floor(const Term &t, double share) {
  const double k = t.kurt();
  if (!(k > 1.0) || !(share > 0.0)) return 0;
  const double f = share / kVarRelErr;
  return (uint64_t)std::min(1e12, std::ceil((k - 1.0) * f * f));
}

// Shares (V_i / m_i) / sum_j (V_j / m_j) of the terms in the estimator's
// variance at the allocated counts m.
std::vector<double> variance_shares(const std::vector<double> &v, const std::vector<double> &m) {
  std::vector<double> f(v.size(), 0.0);
  double tot = 0.0;
  for (size_t i = 0; i < v.size(); ++i)
    if (m[i] > 0.0) tot += v[i] / m[i];
  if (tot > 0.0)
    for (size_t i = 0; i < v.size(); ++i)
      if (m[i] > 0.0) f[i] = v[i] / m[i] / tot;
  return f;
}

// The adaptive estimator (Section 4.1's cost model applied per level): the
// nested pair of level l -- the approximate two-way term (variance V2, cost
// c2 per path) and the four-way correction (V4, c4) -- needs total work
// (sqrt(V2 c2) + sqrt(V4 c4))^2 / eps'^2 for a given variance share, the exact
// two-way term about V2 ce / eps'^2 (its variance is the approximate one's up
// to the approximation error).  The pair stays where it is cheaper.
bool nested_pays(const Term &t2, const Term &t4, double c2, double c4, double ce) {
  const double v2 = t2.var(), v4 = t4.var();
  const double nested = std::sqrt(v2 * c2) + std::sqrt(v4 * c4);
  return nested * nested <= v2 * ce;
}

// Philox stream of the exact term that replaces level l's nested pair (tags
// 1 + 64 est + 2 l + t are the pairs'; these follow them, below 256).
uint32_t exact_level_tag(int est, int l) { return 1u + 64u * (uint32_t)est + 42u + (uint32_t)l; }

// Pilot paths of a new multilevel term at level l: n at levels <= L_min,
// halved for each level above (at least 128).  The optimal counts of level
// corrections fall like 2^-l for the usual variance decay and cost growth
// (Section 4.1), so a full pilot at a fine level would be most of that
// level's cost.  Plain Monte Carlo (one term at its level) keeps n.
uint64_t level_pilot(uint64_t n, int l, int L_min, int estimator) {
  if (estimator == AICDF_EST_PLAIN) return n;
  const int d = std::max(0, l - L_min);
  return std::max<uint64_t>(std::min<uint64_t>(n, 128), d >= 63 ? 0 : n >> d);
}

// Pilot paths of a new four-way correction term of the nested estimator.
// Its variance is that of the approximation error -- 2^-11 .. 2^-14 of the
// two-way terms' for the piecewise-linear table (Section 4) -- so its optimal
// path count is one to two orders of magnitude below theirs, and a full-size
// pilot would be most of its cost at the fine levels.  n_pilot / 16 (at
// least 128) still estimates the variance to ~10%.
uint64_t corr_pilot(uint64_t pilot) { return std::min(pilot, std::max<uint64_t>(128, pilot / 16)); }

constexpr size_t kSumsBytes = 256 + 8192;
// Calibration launch: level 5 with 2^21 paths (33 fine steps each) fills
// every SM for several waves, so the measured time is the throughput cost
// per path-step rather than launch latency and the tail of a partial wave.
constexpr int kCalLevel = 5;
constexpr uint64_t kCalPaths = 1u << 21;

std::mutex g_cal_mu;
std::map<std::tuple<int, int, int, int, int>, double> g_step_ns;  // (dev, model, scheme, approx, kind)

// Device ns per fine step of one path of `kind` (calibrated once).
aicdf_status step_cost_ns(const aicdf_sde_params *prm, aicdf_table tab, int kind, void *ws, size_t wsb,
                          double *sums_dev, cudaStream_t st, double *out) {
  int dev = 0, method = 0, n = 0;
  cudaGetDevice(&dev);
  aicdf_table_info(tab, &method, &n);
  const auto key = std::make_tuple(dev, prm->model, prm->scheme, method, kind);
  {
    std::lock_guard<std::mutex> lock(g_cal_mu);
    auto it = g_step_ns.find(key);
    if (it != g_step_ns.end()) {
      *out = it->second;
      return AICDF_OK;
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  aicdf_status s = aicdf_mlmc_level(prm, tab, kCalLevel, kind, kCalPaths, 0, 1234, 0xCA1u, sums_dev, ws, wsb,
                                    (aicdf_stream_t)st);  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 2 && s == AICDF_OK; ++rep) {
    cudaEventRecord(e0, st);
    s = aicdf_mlmc_level(prm, tab, kCalLevel, kind, kCalPaths, 0, 1234, 0xCA1u, sums_dev, ws, wsb,
                         (aicdf_stream_t)st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != AICDF_OK) return s;
  const double ns = (double)best * 1e6 / ((double)kCalPaths * (double)((1 << kCalLevel) + 1));
  std::lock_guard<std::mutex> lock(g_cal_mu);
  g_step_ns[key] = ns;
  *out = ns;
  return AICDF_OK;
}

}  // namespace

extern "C" size_t aicdf_mlmc_run_workspace_bytes(void) {
  // level-kernel partials | calibration sums (256 B) | per-round term sums
  // (8 KiB: 2 x 21 terms x 5 doubles) | batch tile list and partials
  return aicdf_mlmc_level_workspace_bytes() + kSumsBytes + (8u << 20);
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
  if (o->estimator < AICDF_EST_NESTED || o->estimator > AICDF_EST_ADAPTIVE) return AICDF_ERR_ARG;
  if (o->estimator == AICDF_EST_PLAIN && o->fixed_L < 0) return AICDF_ERR_ARG;
  if (workspace_bytes < aicdf_mlmc_run_workspace_bytes() || ((uintptr_t)workspace_dev % 256))
    return AICDF_ERR_ARG;
  const auto wall0 = std::chrono::steady_clock::now();
  std::memset(r, 0, sizeof(*r));
  cudaStream_t st = (cudaStream_t)stream;
  char *w = (char *)workspace_dev;
  const size_t lvl_ws = aicdf_mlmc_level_workspace_bytes();
  double *cal_sums = reinterpret_cast<double *>(w + lvl_ws);
  double *term_sums = reinterpret_cast<double *>(w + lvl_ws + 256);  // <= 2 x 21 terms x 5 doubles
  void *batch_ws = w + lvl_ws + kSumsBytes;
  const size_t batch_wsb = workspace_bytes - lvl_ws - kSumsBytes;

  const int est = o->estimator;
  std::vector<int> kinds;
  if (est == AICDF_EST_NESTED || est == AICDF_EST_ADAPTIVE) kinds = {AICDF_KIND_APPROX2, AICDF_KIND_CORR4};
  else if (est == AICDF_EST_REGULAR) kinds = {AICDF_KIND_EXACT2};
  else kinds = {AICDF_KIND_PLAIN};
  std::vector<int> cal = kinds;
  if (est == AICDF_EST_ADAPTIVE) cal.push_back(AICDF_KIND_EXACT2);
  double kind_ns[5] = {0, 0, 0, 0, 0};
  for (int k : cal) {
    aicdf_status s = step_cost_ns(params, approx, k, w, lvl_ws, cal_sums, st, &kind_ns[k]);
    if (s != AICDF_OK) return s;
  }
  auto cost = [&](const Term &t) { return kind_ns[t.kind] * (double)((1u << t.level) + 1); };

  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double gpu_ms = 0.0;
  int launches = 0;
  std::vector<Term> terms;
  // one batched launch adding add[i] paths to terms[i] (add[i] = 0: skipped)
  auto run_round = [&](const std::vector<uint64_t> &add) -> aicdf_status {
    std::vector<aicdf_batch_term> bt;
    std::vector<int> idx;
    for (size_t i = 0; i < terms.size(); ++i)
      if (add[i] > 0) {
        aicdf_batch_term x;
        x.set = 0;
        x.level = terms[i].level;
        x.kind = terms[i].kind;
        x.tag = terms[i].tag;
        x.n_paths = add[i];
        x.path_offset = terms[i].n;
        bt.push_back(x);
        idx.push_back((int)i);
      }
    if (bt.empty()) return AICDF_OK;
    cudaEventRecord(e0, st);
    aicdf_status s = aicdf::batch_run_once(params, 1, bt.data(), (int)bt.size(), approx, o->seed, term_sums,
                                           batch_ws, batch_wsb, st);
    if (s != AICDF_OK) return s;
    cudaEventRecord(e1, st);
    std::vector<double> h(aicdf::kSumsPerTerm * bt.size());
    if (cudaMemcpyAsync(h.data(), term_sums, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      aicdf::set_cuda_error((int)cudaGetLastError());
      return AICDF_ERR_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    gpu_ms += ms;
    launches += 1;
    for (size_t j = 0; j < idx.size(); ++j)
      terms[idx[j]].add_sums(&h[aicdf::kSumsPerTerm * j], bt[j].n_paths);
    return AICDF_OK;
  };
  const uint64_t pilot = o->n_pilot ? o->n_pilot : 10000;
  const uint64_t pilot4 = corr_pilot(pilot);
  auto add_levels = [&](int l0, int l1) -> aicdf_status {  // pilot for levels l0..l1
    const size_t first = terms.size();
    for (int l = l0; l <= l1; ++l)
      for (size_t i = 0; i < kinds.size(); ++i) {
        Term t;
        t.level = l;
        t.kind = kinds[i];
        t.slot = (int)i;
        t.tag = 1u + 64u * (uint32_t)est + 2u * (uint32_t)l + (uint32_t)i;
        terms.push_back(t);
      }
    std::vector<uint64_t> add(terms.size(), 0);
    for (size_t i = first; i < terms.size(); ++i)
      add[i] = level_pilot(terms[i].kind == AICDF_KIND_CORR4 ? pilot4 : pilot, terms[i].level, o->L_min, est);
    aicdf_status rs = run_round(add);
    if (rs != AICDF_OK || est != AICDF_EST_ADAPTIVE) return rs;
    // adaptive: the new levels whose nested pair does not pay get an exact term
    const size_t last = terms.size();
    for (size_t i = first; i + 1 < last; i += 2) {
      Term &t2 = terms[i], &t4 = terms[i + 1];
      if (nested_pays(t2, t4, cost(t2), cost(t4), kind_ns[AICDF_KIND_EXACT2] * (double)((1u << t2.level) + 1)))
        continue;
      t2.active = t4.active = false;
      Term t;
      t.level = t2.level;
      t.kind = AICDF_KIND_EXACT2;
      t.slot = 0;
      t.tag = exact_level_tag(est, t2.level);
      terms.push_back(t);
    }
    if (terms.size() == last) return AICDF_OK;
    std::vector<uint64_t> add2(terms.size(), 0);
    for (size_t i = last; i < terms.size(); ++i) add2[i] = level_pilot(pilot, terms[i].level, o->L_min, est);
    return run_round(add2);
  };

  aicdf_status s = AICDF_OK;
  int L;
  if (est == AICDF_EST_PLAIN) {
    L = o->fixed_L;
    s = add_levels(L, L);
  } else {
    L = o->fixed_L >= 0 ? o->fixed_L : o->L_min;
    s = add_levels(0, L);
  }
  bool converged = false;
  const double eps = o->eps;
  const double alpha = o->weak_order > 0.0 ? o->weak_order : 1.0;
  while (s == AICDF_OK) {
    // optimal counts for the current terms (Section 4.1)
    std::vector<double> v, c, m(terms.size());
    for (auto &t : terms) {
      v.push_back(t.active ? t.var() : 0.0);  // a replaced pair gets no more paths
      c.push_back(cost(t));
    }
    double total = 0.0;
    s = aicdf_mlmc_allocate((int)terms.size(), v.data(), c.data(), eps, m.data(), &total);
    if (s != AICDF_OK) break;
    std::vector<uint64_t> add(terms.size(), 0);
    const std::vector<double> share = variance_shares(v, m);
    for (size_t i = 0; i < terms.size(); ++i) {
      const double want = std::max(std::ceil(m[i]), (double)kurtosis_floor(terms[i], share[i]));
      if (!(want < 1e15)) {
        s = AICDF_ERR_NOCONVERGE;
        break;
      }
      if ((uint64_t)want > terms[i].n) add[i] = (uint64_t)want - terms[i].n;
    }
    if (s != AICDF_OK) break;
    s = run_round(add);
    if (s != AICDF_OK) break;
    if (est == AICDF_EST_PLAIN || o->fixed_L >= 0) {
      converged = true;
      break;
    }
    // bias estimate from the two finest levels' total corrections
    auto level_mean = [&](int l) {
      double mm = 0.0;
      for (auto &t : terms)
        if (t.level == l && t.active) mm += t.mean();
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
    // the weak error decays like 2^(-alpha l): add at once the levels that
    // bring the estimated bias under eps / sqrt(2) (at least one), so that
    // the counts are re-allocated once per jump rather than once per level
    const double gap = std::log2(bias / (eps / std::sqrt(2.0))) / alpha;
    const int jump = std::max(1, (int)std::ceil(gap));
    const int L_new = std::min(o->L_max, L + jump);
    s = add_levels(L + 1, L_new);
    L = L_new;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != AICDF_OK) return s;
  double estv = 0.0, var = 0.0;
  for (auto &t : terms) {
    if (!t.active) continue;
    estv += t.mean();
    var += t.n ? t.var() / (double)t.n : 0.0;
    r->paths[t.level][t.slot] = t.n;
    r->mean[t.level][t.slot] = t.mean();
    r->var[t.level][t.slot] = t.var();
    r->kurt[t.level][t.slot] = t.kurt();
    r->cost_ns[t.level][t.slot] = cost(t);
    if (t.kind == AICDF_KIND_EXACT2 && est == AICDF_EST_ADAPTIVE) r->exact_level[t.level] = 1;
  }
  r->estimate = estv;
  r->variance = var;
  r->L = L;
  r->converged = converged ? 1 : 0;
  r->n_terms = (est == AICDF_EST_NESTED || est == AICDF_EST_ADAPTIVE) ? 2 : 1;
  r->gpu_ms = gpu_ms;
  r->launches = launches;
  r->wall_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
  return AICDF_OK;
}

// ---------------------------------------------------------------------------
// Many independent parameter sets at once (Section 4.1 per set): every round
// is one batched launch holding the new paths of all sets' terms, so a small
// set costs no launch of its own.  Per set: pilot paths on levels 0..L_min,
// the optimal allocation from its own variances and the calibrated per-step
// costs of its model, the bias test, and the predicted level jump.
namespace {
constexpr size_t kSetSumsBytes = 256 * 8;  // per set: 5 sums x 2 kinds x 24 levels (1920 B), 256-B multiple
constexpr size_t kSetBatchBytes = 2 * AICDF_MAX_LEVELS * 128;                // per set: tiles, specs, slots
constexpr size_t kBatchSlack = 16u << 20;                                    // load-balancing tiles
}  // namespace

extern "C" size_t aicdf_mlmc_run_sets_workspace_bytes(int n_sets) {
  if (n_sets <= 0) return 0;
  return aicdf_mlmc_level_workspace_bytes() + 256 + (size_t)n_sets * (kSetSumsBytes + kSetBatchBytes) +
         kBatchSlack;
}

extern "C" aicdf_status aicdf_mlmc_run_sets(const aicdf_sde_params *sets, int n_sets, aicdf_table approx,
                                            const aicdf_mlmc_opts *o, aicdf_mlmc_result *results,
                                            void *workspace_dev, size_t workspace_bytes,
                                            aicdf_stream_t stream) {
  if (!sets || n_sets <= 0 || n_sets > (1 << 20) || !o || !results || !workspace_dev) return AICDF_ERR_ARG;
  if (!aicdf::table_ok(approx)) return AICDF_ERR_ARG;
  if (!(o->eps > 0.0) || o->L_min < 0 || o->L_max < o->L_min || o->L_max >= AICDF_MAX_LEVELS ||
      o->L_max > 20 || o->fixed_L >= AICDF_MAX_LEVELS || o->fixed_L > 20)
    return AICDF_ERR_ARG;
  if (o->estimator < AICDF_EST_NESTED || o->estimator > AICDF_EST_ADAPTIVE) return AICDF_ERR_ARG;
  if (o->estimator == AICDF_EST_PLAIN && o->fixed_L < 0) return AICDF_ERR_ARG;
  if (workspace_bytes < aicdf_mlmc_run_sets_workspace_bytes(n_sets) || ((uintptr_t)workspace_dev % 256))
    return AICDF_ERR_ARG;
  const auto wall0 = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)stream;
  char *w = (char *)workspace_dev;
  const size_t lvl_ws = aicdf_mlmc_level_workspace_bytes();
  double *cal_sums = reinterpret_cast<double *>(w + lvl_ws);
  double *term_sums = reinterpret_cast<double *>(w + lvl_ws + 256);
  char *batch_ws = w + lvl_ws + 256 + (size_t)n_sets * kSetSumsBytes;
  const size_t batch_wsb = workspace_bytes - (size_t)(batch_ws - w);

  const int est = o->estimator;
  std::vector<int> kinds;
  if (est == AICDF_EST_NESTED || est == AICDF_EST_ADAPTIVE) kinds = {AICDF_KIND_APPROX2, AICDF_KIND_CORR4};
  else if (est == AICDF_EST_REGULAR) kinds = {AICDF_KIND_EXACT2};
  else kinds = {AICDF_KIND_PLAIN};
  std::vector<int> cal = kinds;
  if (est == AICDF_EST_ADAPTIVE) cal.push_back(AICDF_KIND_EXACT2);
  // calibrated per-step costs, per (model, scheme) of the sets (cached per process)
  std::map<std::pair<int, int>, std::vector<double>> kind_ns;
  for (int s = 0; s < n_sets; ++s) {
    const auto key = std::make_pair(sets[s].model, sets[s].scheme);
    if (kind_ns.count(key)) continue;
    std::vector<double> ns(5, 0.0);
    for (int k : cal) {
      aicdf_status rc = step_cost_ns(&sets[s], approx, k, w, lvl_ws, cal_sums, st, &ns[k]);
      if (rc != AICDF_OK) return rc;
    }
    kind_ns[key] = ns;
  }
  struct SetState {
    std::vector<Term> terms;
    int L = 0;
    bool active = true, converged = false;
    double bias = 0.0;
  };
  std::vector<SetState> S(n_sets);
  auto cost = [&](int s, const Term &t) {
    return kind_ns[std::make_pair(sets[s].model, sets[s].scheme)][t.kind] * (double)((1u << t.level) + 1);
  };
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double gpu_ms = 0.0;
  int launches = 0;
  // one batched launch adding add[s][i] paths to S[s].terms[i]
  auto run_round = [&](const std::vector<std::vector<uint64_t>> &add) -> aicdf_status {
    std::vector<aicdf_batch_term> bt;
    std::vector<std::pair<int, int>> idx;
    for (int s = 0; s < n_sets; ++s)
      for (size_t i = 0; i < add[s].size(); ++i)
        if (add[s][i] > 0) {
          const Term &t = S[s].terms[i];
          aicdf_batch_term x;
          x.set = (uint32_t)s;
          x.level = t.level;
          x.kind = t.kind;
          x.tag = t.tag;
          x.n_paths = add[s][i];
          x.path_offset = t.n;
          bt.push_back(x);
          idx.emplace_back(s, (int)i);
        }
    if (bt.empty()) return AICDF_OK;
    cudaEventRecord(e0, st);
    // one launch; a round whose tile plan does not fit the workspace is split
    // in halves (each half one launch), recursively
    std::function<aicdf_status(size_t, size_t)> launch = [&](size_t lo, size_t hi) -> aicdf_status {
      aicdf_status q = aicdf::batch_run_once(sets, n_sets, bt.data() + lo, (int)(hi - lo), approx, o->seed,
                                             term_sums + aicdf::kSumsPerTerm * lo, batch_ws, batch_wsb, st);
      if (q == AICDF_OK) ++launches;
      if (q == AICDF_ERR_NOMEM && hi - lo > 1) {
        const size_t mid = lo + (hi - lo) / 2;
        q = launch(lo, mid);
        if (q == AICDF_OK) q = launch(mid, hi);
      }
      return q;
    };
    aicdf_status rc = launch(0, bt.size());
    if (rc != AICDF_OK) return rc;
    cudaEventRecord(e1, st);
    std::vector<double> h(aicdf::kSumsPerTerm * bt.size());
    if (cudaMemcpyAsync(h.data(), term_sums, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      aicdf::set_cuda_error((int)cudaGetLastError());
      return AICDF_ERR_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    gpu_ms += ms;
    for (size_t j = 0; j < idx.size(); ++j)
      S[idx[j].first].terms[idx[j].second].add_sums(&h[aicdf::kSumsPerTerm * j], bt[j].n_paths);
    return AICDF_OK;
  };
  const uint64_t pilot = o->n_pilot ? o->n_pilot : 10000;
  const uint64_t pilot4 = corr_pilot(pilot);
  // new terms for levels l0..l1 of set s, with their pilot counts in add
  auto new_levels = [&](int s, int l0, int l1, std::vector<std::vector<uint64_t>> &add) {
    for (int l = l0; l <= l1; ++l)
      for (size_t i = 0; i < kinds.size(); ++i) {
        Term t;
        t.level = l;
        t.kind = kinds[i];
        t.slot = (int)i;
        // distinct streams per set, estimator, level and kind
        t.tag = ((uint32_t)s << 8) + 1u + 64u * (uint32_t)est + 2u * (uint32_t)l + (uint32_t)i;
        S[s].terms.push_back(t);
        add[s].push_back(level_pilot(t.kind == AICDF_KIND_CORR4 ? pilot4 : pilot, l, o->L_min, est));
      }
  };
  // adaptive: after a pilot round, each set's new levels whose nested pair
  // does not pay (nested_pays) get an exact term instead, piloted in one more
  // launch; first[s] = the set's first term of that round
  auto adapt = [&](const std::vector<size_t> &first) -> aicdf_status {
    if (est != AICDF_EST_ADAPTIVE) return AICDF_OK;
    std::vector<std::vector<uint64_t>> add2(n_sets);
    bool any = false;
    for (int s = 0; s < n_sets; ++s) {
      std::vector<Term> &T = S[s].terms;
      const size_t last = T.size();
      const double ce_step = kind_ns[std::make_pair(sets[s].model, sets[s].scheme)][AICDF_KIND_EXACT2];
      for (size_t i = first[s]; i + 1 < last; i += 2) {
        if (!nested_pays(T[i], T[i + 1], cost(s, T[i]), cost(s, T[i + 1]),
                         ce_step * (double)((1u << T[i].level) + 1)))
          {
            T[i].active = T[i + 1].active = false;
            Term t;
            t.level = T[i].level;
            t.kind = AICDF_KIND_EXACT2;
            t.slot = 0;
            t.tag = ((uint32_t)s << 8) + exact_level_tag(est, t.level);
            T.push_back(t);
          }
      }
      add2[s].assign(T.size(), 0);
      for (size_t i = last; i < T.size(); ++i) {
        add2[s][i] = level_pilot(pilot, T[i].level, o->L_min, est);
        any = true;
      }
    }
    return any ? run_round(add2) : AICDF_OK;
  };
  std::vector<std::vector<uint64_t>> add(n_sets);
  for (int s = 0; s < n_sets; ++s) {
    if (est == AICDF_EST_PLAIN) {
      S[s].L = o->fixed_L;
      new_levels(s, S[s].L, S[s].L, add);
    } else {
      S[s].L = o->fixed_L >= 0 ? o->fixed_L : o->L_min;
      new_levels(s, 0, S[s].L, add);
    }
  }
  aicdf_status rc = run_round(add);
  if (rc == AICDF_OK) rc = adapt(std::vector<size_t>(n_sets, 0));
  const double eps = o->eps;
  const double alpha = o->weak_order > 0.0 ? o->weak_order : 1.0;
  const double a2 = std::pow(2.0, alpha);
  while (rc == AICDF_OK) {
    // allocation round over the active sets
    bool any = false;
    for (int s = 0; s < n_sets; ++s) {
      add[s].assign(S[s].terms.size(), 0);
      if (!S[s].active) continue;
      any = true;
      std::vector<double> v, c, m(S[s].terms.size());
      for (auto &t : S[s].terms) {
        v.push_back(t.active ? t.var() : 0.0);  // a replaced pair gets no more paths
        c.push_back(cost(s, t));
      }
      double total = 0.0;
      rc = aicdf_mlmc_allocate((int)S[s].terms.size(), v.data(), c.data(), eps, m.data(), &total);
      if (rc != AICDF_OK) break;
      const std::vector<double> share = variance_shares(v, m);
      for (size_t i = 0; i < S[s].terms.size(); ++i) {
        const double want = std::max(std::ceil(m[i]), (double)kurtosis_floor(S[s].terms[i], share[i]));
        if (!(want < 1e15)) {
          rc = AICDF_ERR_NOCONVERGE;
          break;
        }
        if ((uint64_t)want > S[s].terms[i].n) add[s][i] = (uint64_t)want - S[s].terms[i].n;
      }
      if (rc != AICDF_OK) break;
    }
    if (rc != AICDF_OK || !any) break;
    rc = run_round(add);
    if (rc != AICDF_OK) break;
    // bias test per set; sets that need more levels get them, piloted in one launch
    bool grow = false;
    std::vector<size_t> first(n_sets);
    for (int s = 0; s < n_sets; ++s) {
      first[s] = S[s].terms.size();
      add[s].assign(S[s].terms.size(), 0);
      SetState &q = S[s];
      if (!q.active) continue;
      if (est == AICDF_EST_PLAIN || o->fixed_L >= 0) {
        q.active = false;
        q.converged = true;
        continue;
      }
      auto level_mean = [&](int l) {
        double mm = 0.0;
        for (auto &t : q.terms)
          if (t.level == l && t.active) mm += t.mean();
        return mm;
      };
      double bias = std::fabs(level_mean(q.L)) / (a2 - 1.0);
      if (q.L > 0) bias = std::max(bias, std::fabs(level_mean(q.L - 1)) / a2 / (a2 - 1.0));
      q.bias = bias;
      if (bias <= eps / std::sqrt(2.0)) {
        q.active = false;
        q.converged = true;
        continue;
      }
      if (q.L >= o->L_max) {
        q.active = false;
        continue;
      }
      const int jump = std::max(1, (int)std::ceil(std::log2(bias / (eps / std::sqrt(2.0))) / alpha));
      const int L_new = std::min(o->L_max, q.L + jump);
      new_levels(s, q.L + 1, L_new, add);
      q.L = L_new;
      grow = true;
    }
    if (grow) rc = run_round(add);
    if (grow && rc == AICDF_OK) rc = adapt(first);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != AICDF_OK) return rc;
  const double wall_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
  for (int s = 0; s < n_sets; ++s) {
    aicdf_mlmc_result *r = &results[s];
    std::memset(r, 0, sizeof(*r));
    double estv = 0.0, var = 0.0;
    for (auto &t : S[s].terms) {
      if (!t.active) continue;
      estv += t.mean();
      var += t.n ? t.var() / (double)t.n : 0.0;
      r->paths[t.level][t.slot] = t.n;
      r->mean[t.level][t.slot] = t.mean();
      r->var[t.level][t.slot] = t.var();
      r->kurt[t.level][t.slot] = t.kurt();
      r->cost_ns[t.level][t.slot] = cost(s, t);
      if (t.kind == AICDF_KIND_EXACT2 && est == AICDF_EST_ADAPTIVE) r->exact_level[t.level] = 1;
    }
    r->estimate = estv;
    r->variance = var;
    r->bias = S[s].bias;
    r->L = S[s].L;
    r->converged = S[s].converged ? 1 : 0;
    r->n_terms = (est == AICDF_EST_NESTED || est == AICDF_EST_ADAPTIVE) ? 2 : 1;
    r->gpu_ms = gpu_ms;
    r->wall_ms = wall_ms;
    r->launches = launches;
  }
  return AICDF_OK;
}
