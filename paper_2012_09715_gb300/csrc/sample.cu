// Standalone sampling kernels: u -> approximate (or exact) Gaussian variate.
//
// One kernel template covers the four methods (piecewise constant, piecewise
// linear, exact FP32, CUDA's normcdfinvf), two output types (FP32, FP16) and
// two uniform sources (in-register Philox, or a caller buffer).  The work is
// pure streaming: a warp owns 32 consecutive 16-byte output vectors per
// iteration (4 FP32 or 8 FP16 samples per thread), written with one 128-bit
// store each, and walks the output with a grid stride that is a multiple of
// the SM count.  No shared state besides the PWC table in shared memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "aicdf_internal.h"
#include "device_common.cuh"
#include "sample_kernels.cuh"

namespace aicdf {

using KernelFn = void (*)(SampleArgs);

template <int METHOD, int OUT, int SRC>
KernelFn pick(bool vec) {
  return vec ? (KernelFn)k_sample_vec<METHOD, OUT, SRC> : (KernelFn)k_sample_scalar<METHOD, OUT, SRC>;
}

template <int METHOD>
KernelFn pick2(int out, int src, bool vec) {
  if (out == AICDF_F32)
    return src == SRC_PHILOX ? pick<METHOD, AICDF_F32, SRC_PHILOX>(vec) : pick<METHOD, AICDF_F32, SRC_INPUT>(vec);
  return src == SRC_PHILOX ? pick<METHOD, AICDF_F16, SRC_PHILOX>(vec) : pick<METHOD, AICDF_F16, SRC_INPUT>(vec);
}

static KernelFn select_kernel(int method, int out, int src, bool vec) {
  switch (method) {
    case AICDF_PWC: return pick2<AICDF_PWC>(out, src, vec);
    case AICDF_PWL: return pick2<AICDF_PWL>(out, src, vec);
    case AICDF_PWP: return pick2<AICDF_PWP>(out, src, vec);
    case AICDF_EXACT: return pick2<AICDF_EXACT>(out, src, vec);
    default: return pick2<AICDF_EXACT_LIB>(out, src, vec);
  }
}

// Fill the kernel argument block; validates the method/table pairing.
aicdf_status prepare_sample_args(aicdf_table table, int method, SampleArgs *a) {
  std::memset(a, 0, sizeof(*a));
  if (method == AICDF_PWC || method == AICDF_PWL || method == AICDF_PWP) {
    if (!table_ok(table) || table->method != method) return AICDF_ERR_ARG;
    if (method == AICDF_PWP) {
      if (table->n > 15) return AICDF_ERR_UNSUPPORTED;
      for (int j = 0; j < 4; ++j)
        for (int r = 0; r < 16; ++r) a->tab[16 * j + r] = table->fv[4 * std::min(r, table->n) + j];
      a->ntab = table->n;
    } else if (method == AICDF_PWC) {
      if (table->n > 1024) return AICDF_ERR_UNSUPPORTED;
      for (int i = 0; i < table->n; ++i) a->tab[i] = table->f0[i];
      a->ntab = table->n;
      a->nf = (float)table->n;
      int q = 0;
      while ((1 << q) < table->n) ++q;
      a->pwc_shift = (uint32_t)(23 - q);
    } else {
      if (table->n > 15) return AICDF_ERR_UNSUPPORTED;  // 16 rows fit one half-warp
      for (int i = 0; i < 16; ++i) {
        const int r = std::min(i, table->n);  // rows past K repeat row K (never indexed)
        a->tab[i] = table->f0[r];
        a->tab[16 + i] = table->f1[r];
      }
      a->ntab = table->n;
    }
  } else if (method == AICDF_EXACT || method == AICDF_EXACT_LIB) {
    if (table) return AICDF_ERR_ARG;
  } else {
    return AICDF_ERR_ARG;
  }
  return AICDF_OK;
}

template <int OUT>
static KernelFn select_philox32(int method) {
  switch (method) {
    case AICDF_PWC: return k_sample_philox32<AICDF_PWC, OUT>;
    case AICDF_PWL: return k_sample_philox32<AICDF_PWL, OUT>;
    case AICDF_PWP: return k_sample_philox32<AICDF_PWP, OUT>;
    case AICDF_EXACT: return k_sample_philox32<AICDF_EXACT, OUT>;
    default: return k_sample_philox32<AICDF_EXACT_LIB, OUT>;
  }
}

aicdf_status launch_sample(const SampleArgs &a, int method, int out_dtype, int src, bool vec,
                           cudaStream_t stream) {
  KernelFn k = select_kernel(method, out_dtype, src, vec);
  const int E = vec ? (out_dtype == AICDF_F32 ? 4 : 8) : 1;
  int waves = 1;
  uint64_t per_thread = 1;  // output units a thread takes per grid-stride step
  if (src == SRC_PHILOX && vec) {
    // 32-bit index variant when counters and element indices stay below 2^32
    // (a warp chunk spans at most 128 vectors)
    const uint64_t nvec = (a.n + E - 1) / E;
    const uint64_t lim = 1ull << 32;
    if ((nvec + 128) * (uint64_t)E < lim && (a.offset >> 2) + (nvec + 128) * (uint64_t)(E / 4) < lim) {
      k = out_dtype == AICDF_F32 ? select_philox32<AICDF_F32>(method) : select_philox32<AICDF_F16>(method);
      waves = 4;  // several resident-block waves even out the end of the grid-stride loop
      per_thread = out_dtype == AICDF_F32 ? 4 : 2;  // vectors of a lane's warp chunk
    }
  }
  const uint64_t units = (a.n + E - 1) / E;
  const int threads = 256;
  // SMs x resident blocks of this kernel x waves (grid-stride inside); small
  // launches get one chunk per warp, so no block starts with nothing to do
  const uint64_t cap = (uint64_t)sm_count() * resident_blocks((const void *)k, threads) * waves;
  uint64_t blocks = (units + threads * per_thread - 1) / (threads * per_thread);
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k<<<(unsigned)blocks, threads, 0, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error((int)e);
    return AICDF_ERR_CUDA;
  }
  return AICDF_OK;
}

template <int OUT, int B>
static KernelFn pick_bits(int method, bool vec) {
  switch (method) {
    case AICDF_PWC: return vec ? k_sample_bits<AICDF_PWC, OUT, B> : k_sample_bits_scalar<AICDF_PWC, OUT, B>;
    case AICDF_PWL: return vec ? k_sample_bits<AICDF_PWL, OUT, B> : k_sample_bits_scalar<AICDF_PWL, OUT, B>;
    case AICDF_PWP: return vec ? k_sample_bits<AICDF_PWP, OUT, B> : k_sample_bits_scalar<AICDF_PWP, OUT, B>;
    case AICDF_EXACT:
      return vec ? k_sample_bits<AICDF_EXACT, OUT, B> : k_sample_bits_scalar<AICDF_EXACT, OUT, B>;
    default:
      return vec ? k_sample_bits<AICDF_EXACT_LIB, OUT, B> : k_sample_bits_scalar<AICDF_EXACT_LIB, OUT, B>;
  }
}

aicdf_status launch_sample_bits(const SampleArgs &a, int method, int bits, int out_dtype, bool vec,
                                cudaStream_t stream) {
  KernelFn k;
  if (bits == 8) k = out_dtype == AICDF_F32 ? pick_bits<AICDF_F32, 8>(method, vec) : pick_bits<AICDF_F16, 8>(method, vec);
  else k = out_dtype == AICDF_F32 ? pick_bits<AICDF_F32, 16>(method, vec) : pick_bits<AICDF_F16, 16>(method, vec);
  const uint64_t S = 4 * (32 / bits);
  const uint64_t units = vec ? (a.n + S - 1) / S : a.n;  // calls (vector) or samples per thread
  const int threads = 256;
  const uint64_t cap = (uint64_t)sm_count() * resident_blocks((const void *)k, threads) * 4;
  uint64_t blocks = (units + threads - 1) / threads;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k<<<(unsigned)blocks, threads, 0, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error((int)e);
    return AICDF_ERR_CUDA;
  }
  return AICDF_OK;
}

}  // namespace aicdf

using namespace aicdf;

extern "C" aicdf_status aicdf_sample(aicdf_table table, int method, const float *u_dev,
                                     uint64_t seed, uint64_t offset, size_t n, void *out_dev,
                                     int out_dtype, aicdf_stream_t stream) {
  if (out_dtype != AICDF_F32 && out_dtype != AICDF_F16) return AICDF_ERR_ARG;
  static thread_local SampleArgs a;  // 4 KiB: keep it off the stack
  aicdf_status s = prepare_sample_args(table, method, &a);
  if (s != AICDF_OK) return s;
  if (n == 0) return AICDF_OK;
  if (!out_dev) return AICDF_ERR_ARG;
  const size_t esz = out_dtype == AICDF_F32 ? 4 : 2;
  if ((uintptr_t)out_dev % esz) return AICDF_ERR_ARG;
  if (u_dev && ((uintptr_t)u_dev % 4)) return AICDF_ERR_ARG;
  a.u = u_dev;
  a.out = out_dev;
  a.n = n;
  a.offset = offset;
  a.keys = make_keys(seed);
  const int src = u_dev ? SRC_INPUT : SRC_PHILOX;
  bool vec = ((uintptr_t)out_dev % 16) == 0;
  if (src == SRC_PHILOX) vec = vec && (offset % 4 == 0);
  else vec = vec && ((uintptr_t)u_dev % 16) == 0;
  return launch_sample(a, method, out_dtype, src, vec, (cudaStream_t)stream);
}

extern "C" aicdf_status aicdf_sample_to_host(aicdf_table table, int method, uint64_t seed,
                                             uint64_t offset, size_t n, void *host_out,
                                             int out_dtype, void *staging_dev,
                                             size_t staging_bytes, aicdf_stream_t stream) {
  if (out_dtype != AICDF_F32 && out_dtype != AICDF_F16) return AICDF_ERR_ARG;
  if (n == 0) return AICDF_OK;
  if (!host_out || !staging_dev || staging_bytes < (2u << 20)) return AICDF_ERR_ARG;
  if ((uintptr_t)staging_dev % 256) return AICDF_ERR_ARG;
  static thread_local SampleArgs a;
  aicdf_status s = prepare_sample_args(table, method, &a);
  if (s != AICDF_OK) return s;
  a.u = nullptr;
  a.keys = make_keys(seed);
  const size_t esz = out_dtype == AICDF_F32 ? 4 : 2;
  cudaStream_t st = (cudaStream_t)stream;
  // Page-locked host memory that the device can address: the kernel stores
  // straight into it over the host link (no staging, no copy engine).
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, host_out) == cudaSuccess && at.type == cudaMemoryTypeHost &&
      at.devicePointer && ((uintptr_t)at.devicePointer % esz) == 0) {
    a.out = at.devicePointer;
    a.n = n;
    a.offset = offset;
    const bool vec = ((uintptr_t)at.devicePointer % 16) == 0 && (offset % 4) == 0;
    s = launch_sample(a, method, out_dtype, SRC_PHILOX, vec, st);
    if (s != AICDF_OK) return s;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_cuda_error((int)e);
      return AICDF_ERR_CUDA;
    }
    return AICDF_OK;
  }
  cudaGetLastError();  // clear a pointer-query error for pageable memory
  // NB staging buffers (4 when the staging holds >= 4 x 1 MiB, else 2), each
  // a multiple of 256 bytes; chunk i is generated into buffer i % NB on the
  // caller's stream and copied out on copy stream i % 2, so two copies can be
  // in flight on separate copy engines while the next chunk is generated.
  const int NB = staging_bytes >= (4u << 20) ? 4 : 2;
  const size_t part = (staging_bytes / NB) & ~(size_t)255;
  const size_t chunk = part / esz;
  cudaEvent_t done[4] = {}, copied[4] = {};
  cudaStream_t copy_st[2] = {};
  bool ok = true;
  for (int i = 0; i < NB; ++i)
    ok = ok && cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < 2; ++i) ok = ok && cudaStreamCreateWithFlags(&copy_st[i], cudaStreamNonBlocking) == cudaSuccess;
  aicdf_status rc = ok ? AICDF_OK : AICDF_ERR_CUDA;
  if (!ok) set_cuda_error((int)cudaGetLastError());
  size_t pos = 0;
  uint64_t k = 0;
  bool used[4] = {false, false, false, false};
  while (rc == AICDF_OK && pos < n) {
    const size_t cnt = std::min(chunk, n - pos);
    const int buf = (int)(k % NB);
    cudaStream_t cs = copy_st[k % 2];
    char *dst = (char *)staging_dev + (size_t)buf * part;
    // the generator may not overwrite a buffer whose copy is still in flight
    if (used[buf]) cudaStreamWaitEvent(st, copied[buf], 0);
    a.out = dst;
    a.n = cnt;
    a.offset = offset + pos;
    const bool vec = ((offset + pos) % 4) == 0;
    rc = launch_sample(a, method, out_dtype, SRC_PHILOX, vec, st);
    if (rc != AICDF_OK) break;
    cudaEventRecord(done[buf], st);
    cudaStreamWaitEvent(cs, done[buf], 0);
    if (cudaMemcpyAsync((char *)host_out + pos * esz, dst, cnt * esz, cudaMemcpyDeviceToHost, cs) !=
        cudaSuccess) {
      set_cuda_error((int)cudaGetLastError());
      rc = AICDF_ERR_CUDA;
      break;
    }
    cudaEventRecord(copied[buf], cs);
    used[buf] = true;
    pos += cnt;
    ++k;
  }
  for (int i = 0; i < 2; ++i)
    if (copy_st[i]) {
      cudaError_t e = cudaStreamSynchronize(copy_st[i]);
      if (e != cudaSuccess && rc == AICDF_OK) {
        set_cuda_error((int)e);
        rc = AICDF_ERR_CUDA;
      }
      cudaStreamDestroy(copy_st[i]);
    }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess && rc == AICDF_OK) {
    set_cuda_error((int)e);
    rc = AICDF_ERR_CUDA;
  }
  for (int i = 0; i < NB; ++i) {
    if (done[i]) cudaEventDestroy(done[i]);
    if (copied[i]) cudaEventDestroy(copied[i]);
  }
  return rc;
}

extern "C" aicdf_status aicdf_sample_bits(aicdf_table table, int method, int bits, uint64_t seed,
                                          uint64_t offset, size_t n, void *out_dev, int out_dtype,
                                          aicdf_stream_t stream) {
  if (out_dtype != AICDF_F32 && out_dtype != AICDF_F16) return AICDF_ERR_ARG;
  if (bits < 1 || bits > 23) return AICDF_ERR_ARG;
  if (bits != 8 && bits != 16) return AICDF_ERR_UNSUPPORTED;
  static thread_local SampleArgs a;
  aicdf_status s = prepare_sample_args(table, method, &a);
  if (s != AICDF_OK) return s;
  if (n == 0) return AICDF_OK;
  if (!out_dev) return AICDF_ERR_ARG;
  const size_t esz = out_dtype == AICDF_F32 ? 4 : 2;
  if ((uintptr_t)out_dev % esz) return AICDF_ERR_ARG;
  a.u = nullptr;
  a.out = out_dev;
  a.n = n;
  a.offset = offset;
  a.keys = make_keys(seed);
  const uint64_t S = 4 * (32 / bits);
  const uintptr_t align = (out_dtype == AICDF_F16 && S == 8) ? 16 : 32;
  const bool vec = ((uintptr_t)out_dev % align) == 0 && (offset % S) == 0;
  return launch_sample_bits(a, method, bits, out_dtype, vec, (cudaStream_t)stream);
}
