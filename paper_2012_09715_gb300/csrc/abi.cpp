// ABI utilities: status strings, version, CUDA error record, SM count cache,
// and the host-side MLMC allocation formula (Section 4.1).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "aicdf_internal.h"

namespace aicdf {

static std::atomic<int> g_last_cuda_error{0};

void set_cuda_error(int e) { g_last_cuda_error.store(e); }

bool table_ok(const aicdf_table_s *t) { return t && t->magic == AICDF_TABLE_MAGIC; }

int sm_count() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  std::lock_guard<std::mutex> lock(mu);
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 152;
    cache[dev] = n;
  }
  return cache[dev];
}

int resident_blocks(const void *kernel, int threads) {
  static std::mutex mu;
  static std::map<std::tuple<const void *, int, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_tuple(kernel, threads, dev);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  cache[key] = n;
  return n;
}

}  // namespace aicdf

extern "C" const char *aicdf_status_str(aicdf_status s) {
  switch (s) {
    case AICDF_OK: return "ok";
    case AICDF_ERR_ARG: return "invalid argument";
    case AICDF_ERR_CUDA: return "CUDA error";
    case AICDF_ERR_NOCONVERGE: return "iteration did not converge";
    case AICDF_ERR_DOMAIN: return "parameter outside the model domain";
    case AICDF_ERR_STATE: return "handle in the wrong state";
    case AICDF_ERR_NOMEM: return "out of host memory";
    case AICDF_ERR_UNSUPPORTED: return "unsupported by this build";
  }
  return "unknown status";
}

extern "C" int aicdf_last_cuda_error(void) { return aicdf::g_last_cuda_error.load(); }

extern "C" int aicdf_version(void) { return 100; }

extern "C" aicdf_status aicdf_mlmc_allocate(int nterms, const double *v, const double *c,
                                            double eps, double *m, double *total) {
  if (nterms <= 0 || !v || !c || !m || !(eps > 0.0)) return AICDF_ERR_ARG;
  double s = 0.0;
  for (int i = 0; i < nterms; ++i) {
    if (!(v[i] >= 0.0) || !(c[i] > 0.0) || !std::isfinite(v[i]) || !std::isfinite(c[i]))
      return AICDF_ERR_DOMAIN;
    s += std::sqrt(v[i] * c[i]);
  }
  const double T = 2.0 / (eps * eps) * s * s;  // total time at the optimum
  for (int i = 0; i < nterms; ++i) m[i] = std::sqrt(2.0 * T * v[i] / c[i]) / eps;
  if (total) *total = T;
  return AICDF_OK;
}
