// aicdf_mlmc_level for callers that cannot allocate device memory (the paper
// has no counterpart).  The level kernel's only scratch -- one partial of the
// four FP64 power sums of Y per thread block -- lives in a fixed array inside
// the library instead of a caller workspace.
#include <cuda_runtime.h>

#include <mutex>

#include "aicdf_internal.h"
#include "mlmc_path.cuh"

namespace aicdf {
namespace {

// Every GPU that loads the library holds this array (64 KiB) until the
// process exits.  All calls share it.
constexpr int kNoAllocSlots = 2048;
static __device__ __align__(256) Moments g_noalloc_partials[kNoAllocSlots];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {nullptr};

// Device address of the array for the current device, looked up on the first
// call made on that device.  In host code the array's name only stands in for
// the symbol; it is not an address a kernel may use.
aicdf_status noalloc_scratch(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    set_cuda_error((int)(e != cudaSuccess ? e : cudaErrorInvalidDevice));
    return AICDF_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) {
      set_cuda_error((int)(e != cudaSuccess ? e : cudaErrorInvalidSymbol));
      return AICDF_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return AICDF_OK;
}

}  // namespace
}  // namespace aicdf

using namespace aicdf;

extern "C" aicdf_status aicdf_mlmc_level_noalloc(const aicdf_sde_params *params, aicdf_table approx,
                                                 int level, int kind, uint64_t n_paths,
                                                 uint64_t path_offset, uint64_t seed, uint32_t tag,
                                                 double *sums_dev, aicdf_stream_t stream) {
  static thread_local LevelArgs a;
  aicdf_status s = prepare_level_args(params, approx, level, kind, n_paths, path_offset, seed,
                                      tag, &a);
  if (s != AICDF_OK) return s;
  if (!sums_dev || ((uintptr_t)sums_dev % 8)) return AICDF_ERR_ARG;
  // the launch needs one slot per thread block; refuse what the array cannot hold
  if (level_launch_grid(a) > kNoAllocSlots) return AICDF_ERR_UNSUPPORTED;
  void *scratch = nullptr;
  s = noalloc_scratch(&scratch);
  if (s != AICDF_OK) return s;
  // every slot the reduction reads is written by the same launch first, so the
  // array needs no clearing between calls
  return launch_level(a, sums_dev, scratch, (cudaStream_t)stream);
}
