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
#include <cstring>

#include "aicdf_internal.h"
#include "device_common.cuh"

namespace aicdf {

enum Source { SRC_PHILOX = 0, SRC_INPUT = 1 };

struct SampleArgs {
  const float *u;      // SRC_INPUT: caller uniforms
  void *out;
  uint64_t n;          // samples
  uint64_t offset;     // SRC_PHILOX: index of the first sample in the stream
  PhiloxKeys keys;
  int ntab;            // PWC: intervals; PWL: K (rows 0..K)
  float nf;            // PWC: (float)ntab
  uint32_t pwc_shift;  // PWC: 23 - log2(ntab)
  float tab[1024];     // PWC constants | PWL alpha[0..15], beta[16..31]
};

// Per-thread evaluator for one method.  Construction stages the table.
// word(x): the sample for the library's uniform from Philox word x (on the
// 2^-24 grid); operator()(u): the sample for any FP32 u (caller uniforms).
template <int METHOD, int SRC>
struct Approx;

template <int SRC>
struct Approx<AICDF_PWC, SRC> {
  const float *s;
  float nf;
  int nmax;
  uint32_t shift;
  __device__ Approx(const SampleArgs &a, float *smem) {
    for (int i = threadIdx.x; i < a.ntab; i += blockDim.x) smem[i] = a.tab[i];
    __syncthreads();
    s = smem;
    nf = a.nf;
    nmax = a.ntab - 1;
    shift = a.pwc_shift;
  }
  __device__ __forceinline__ float word(uint32_t x) const { return s[pwc_index_from_word(x, shift)]; }
  __device__ __forceinline__ float operator()(float u) const { return pwc_eval(u, s, nf, nmax); }
};

template <int SRC>
struct Approx<AICDF_PWL, SRC> {
  PwlLane c;     // general inputs: capped index, sign folded into the row
  PwlRows rows;  // grid inputs: 32 rows, sign by xor
  unsigned kmax;
  __device__ Approx(const SampleArgs &a, float *) {
    if (SRC == SRC_PHILOX) rows = pwl_lane_rows(a.tab, a.tab + 16, a.ntab);
    else c = pwl_lane_coefs(a.tab, a.tab + 16);
    kmax = (unsigned)a.ntab;
  }
  __device__ __forceinline__ float word(uint32_t x) const { return pwl_eval_grid(u01(x), rows); }
  __device__ __forceinline__ float operator()(float u) const { return pwl_eval(u, c, kmax); }
};

template <int SRC>
struct Approx<AICDF_EXACT, SRC> {
  __device__ Approx(const SampleArgs &, float *) {}
  __device__ __forceinline__ float word(uint32_t x) const { return phiinv_f32(u01(x)); }
  __device__ __forceinline__ float operator()(float u) const { return phiinv_f32(u); }
};

template <int SRC>
struct Approx<AICDF_EXACT_LIB, SRC> {
  __device__ Approx(const SampleArgs &, float *) {}
  __device__ __forceinline__ float word(uint32_t x) const { return normcdfinvf(u01(x)); }
  __device__ __forceinline__ float operator()(float u) const { return normcdfinvf(u); }
};

template <int OUT>
struct OutVec;
template <>
struct OutVec<AICDF_F32> {
  static constexpr int kElems = 4;
};
template <>
struct OutVec<AICDF_F16> {
  static constexpr int kElems = 8;
};

__device__ __forceinline__ void store_vec(float *out, uint64_t e, const float (&z)[4]) {
  *reinterpret_cast<float4 *>(out + e) = make_float4(z[0], z[1], z[2], z[3]);
}
__device__ __forceinline__ void store_vec(__half *out, uint64_t e, const float (&z)[8]) {
  uint4 w;
  __half2 h0 = __floats2half2_rn(z[0], z[1]), h1 = __floats2half2_rn(z[2], z[3]);
  __half2 h2 = __floats2half2_rn(z[4], z[5]), h3 = __floats2half2_rn(z[6], z[7]);
  w.x = *reinterpret_cast<uint32_t *>(&h0);
  w.y = *reinterpret_cast<uint32_t *>(&h1);
  w.z = *reinterpret_cast<uint32_t *>(&h2);
  w.w = *reinterpret_cast<uint32_t *>(&h3);
  *reinterpret_cast<uint4 *>(out + e) = w;
}
__device__ __forceinline__ void store_one(float *out, uint64_t e, float z) { out[e] = z; }
__device__ __forceinline__ void store_one(__half *out, uint64_t e, float z) {
  out[e] = __float2half_rn(z);
}

// Vectorised kernel.  Requires: out 16-byte aligned; SRC_PHILOX: offset % 4 == 0;
// SRC_INPUT: u 16-byte aligned.
template <int METHOD, int OUT, int SRC>
__global__ void __launch_bounds__(256) k_sample_vec(const __grid_constant__ SampleArgs a) {
  __shared__ float smem[METHOD == AICDF_PWC ? 1024 : 1];
  const Approx<METHOD, SRC> f(a, smem);
  using T = typename std::conditional<OUT == AICDF_F32, float, __half>::type;
  T *out = reinterpret_cast<T *>(a.out);
  constexpr int E = OutVec<OUT>::kElems;
  // Each warp takes chunks of 2 x 32 consecutive 16-byte vectors; lane L
  // computes vectors L and L + 32 of the chunk, so its two independent
  // Philox chains overlap and both stores stay fully coalesced.
  constexpr int VECS = 2;
  const uint64_t nvec = (a.n + E - 1) / E;
  const uint64_t nchunk = (nvec + 32 * VECS - 1) / (32 * VECS);
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  // warp-uniform loop: every lane runs every iteration (shuffles need all 32)
  for (uint64_t chunk = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; chunk < nchunk;
       chunk += warps) {
    float z[VECS][E];
#pragma unroll
    for (int hv = 0; hv < VECS; ++hv) {
      const uint64_t v = chunk * (32 * VECS) + 32 * hv + lane;
      const uint64_t e0 = v * E;
      if constexpr (SRC == SRC_PHILOX) {
#pragma unroll
        for (int h = 0; h < E / 4; ++h) {
          const uint64_t j = (a.offset >> 2) + v * (E / 4) + h;
          const uint4 r = philox(make_uint4((uint32_t)j, (uint32_t)(j >> 32), 0u, 0u), a.keys);
          z[hv][4 * h + 0] = f.word(r.x);
          z[hv][4 * h + 1] = f.word(r.y);
          z[hv][4 * h + 2] = f.word(r.z);
          z[hv][4 * h + 3] = f.word(r.w);
        }
      } else {
#pragma unroll
        for (int h = 0; h < E / 4; ++h) {
          float4 uu = make_float4(0.5f, 0.5f, 0.5f, 0.5f);
          if (e0 + 4 * h + 3 < a.n) {
            uu = __ldcs(reinterpret_cast<const float4 *>(a.u + e0 + 4 * h));
          } else {
            if (e0 + 4 * h + 0 < a.n) uu.x = a.u[e0 + 4 * h + 0];
            if (e0 + 4 * h + 1 < a.n) uu.y = a.u[e0 + 4 * h + 1];
            if (e0 + 4 * h + 2 < a.n) uu.z = a.u[e0 + 4 * h + 2];
          }
          const float us[4] = {uu.x, uu.y, uu.z, uu.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            float y = f(us[t]);
            z[hv][4 * h + t] = in_unit(us[t]) ? y : __int_as_float(0x7fc00000);
          }
        }
      }
    }
#pragma unroll
    for (int hv = 0; hv < VECS; ++hv) {
      const uint64_t e0 = (chunk * (32 * VECS) + 32 * hv + lane) * E;
      if (e0 + E <= a.n) {
        store_vec(out, e0, z[hv]);
      } else if (e0 < a.n) {
#pragma unroll
        for (int t = 0; t < E; ++t)
          if (e0 + t < a.n) store_one(out, e0 + t, z[hv][t]);
      }
    }
  }
}

// Scalar kernel for unaligned pointers or an offset not divisible by 4.
template <int METHOD, int OUT, int SRC>
__global__ void __launch_bounds__(256) k_sample_scalar(const __grid_constant__ SampleArgs a) {
  __shared__ float smem[METHOD == AICDF_PWC ? 1024 : 1];
  const Approx<METHOD, SRC> f(a, smem);
  using T = typename std::conditional<OUT == AICDF_F32, float, __half>::type;
  T *out = reinterpret_cast<T *>(a.out);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < a.n;
       base += stride) {
    const uint64_t e = base + lane;
    float y;
    if constexpr (SRC == SRC_PHILOX) {
      const uint64_t s = a.offset + e;
      const uint64_t j = s >> 2;
      const uint4 r = philox(make_uint4((uint32_t)j, (uint32_t)(j >> 32), 0u, 0u), a.keys);
      const uint32_t w = (s & 3) == 0 ? r.x : (s & 3) == 1 ? r.y : (s & 3) == 2 ? r.z : r.w;
      y = f.word(w);
    } else {
      const float u = (e < a.n) ? a.u[e] : 0.5f;
      y = f(u);
      if (!in_unit(u)) y = __int_as_float(0x7fc00000);
    }
    if (e < a.n) store_one(out, e, y);
  }
}

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
    case AICDF_EXACT: return pick2<AICDF_EXACT>(out, src, vec);
    default: return pick2<AICDF_EXACT_LIB>(out, src, vec);
  }
}

// Fill the kernel argument block; validates the method/table pairing.
aicdf_status prepare_sample_args(aicdf_table table, int method, SampleArgs *a) {
  std::memset(a, 0, sizeof(*a));
  if (method == AICDF_PWC || method == AICDF_PWL) {
    if (!table_ok(table) || table->method != method) return AICDF_ERR_ARG;
    if (method == AICDF_PWC) {
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

aicdf_status launch_sample(const SampleArgs &a, int method, int out_dtype, int src, bool vec,
                           cudaStream_t stream) {
  KernelFn k = select_kernel(method, out_dtype, src, vec);
  const int E = vec ? (out_dtype == AICDF_F32 ? 4 : 8) : 1;
  const uint64_t units = (a.n + E - 1) / E;
  const int threads = 256;
  // one full wave: SMs x resident blocks of this kernel (grid-stride inside)
  const uint64_t cap = (uint64_t)sm_count() * resident_blocks((const void *)k, threads);
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
  // two halves, each a multiple of 16 bytes and of 8 samples
  size_t half = (staging_bytes / 2) & ~(size_t)255;
  const size_t chunk = half / esz;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t done[2];
  if (cudaEventCreateWithFlags(&done[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&done[1], cudaEventDisableTiming) != cudaSuccess) {
    set_cuda_error((int)cudaGetLastError());
    return AICDF_ERR_CUDA;
  }
  cudaStream_t copy_st;
  if (cudaStreamCreateWithFlags(&copy_st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaEventDestroy(done[0]);
    cudaEventDestroy(done[1]);
    set_cuda_error((int)cudaGetLastError());
    return AICDF_ERR_CUDA;
  }
  cudaEvent_t copied[2];
  cudaEventCreateWithFlags(&copied[0], cudaEventDisableTiming);
  cudaEventCreateWithFlags(&copied[1], cudaEventDisableTiming);
  aicdf_status rc = AICDF_OK;
  size_t pos = 0;
  int buf = 0;
  bool used[2] = {false, false};
  while (pos < n) {
    const size_t cnt = std::min(chunk, n - pos);
    char *dst = (char *)staging_dev + (size_t)buf * half;
    // the generator may not overwrite a half whose copy is still in flight
    if (used[buf]) cudaStreamWaitEvent(st, copied[buf], 0);
    a.out = dst;
    a.n = cnt;
    a.offset = offset + pos;
    const bool vec = ((offset + pos) % 4) == 0;
    rc = launch_sample(a, method, out_dtype, SRC_PHILOX, vec, st);
    if (rc != AICDF_OK) break;
    cudaEventRecord(done[buf], st);
    cudaStreamWaitEvent(copy_st, done[buf], 0);
    if (cudaMemcpyAsync((char *)host_out + pos * esz, dst, cnt * esz, cudaMemcpyDeviceToHost,
                        copy_st) != cudaSuccess) {
      set_cuda_error((int)cudaGetLastError());
      rc = AICDF_ERR_CUDA;
      break;
    }
    cudaEventRecord(copied[buf], copy_st);
    used[buf] = true;
    pos += cnt;
    buf ^= 1;
  }
  cudaError_t e = cudaStreamSynchronize(copy_st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess && rc == AICDF_OK) {
    set_cuda_error((int)e);
    rc = AICDF_ERR_CUDA;
  }
  cudaStreamDestroy(copy_st);
  for (int i = 0; i < 2; ++i) {
    cudaEventDestroy(done[i]);
    cudaEventDestroy(copied[i]);
  }
  return rc;
}
