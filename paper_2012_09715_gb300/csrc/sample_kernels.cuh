// Sampling kernels (device side of sample.cu): u -> approximate or exact
// Gaussian variate for the four methods, two output types and two uniform
// sources.  Kept apart from the host code so that the kernel source can be
// fingerprinted on its own.
#pragma once

#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

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
  const float *s, *w;  // the table in row order; its word-order copy (Philox source)
  float nf;
  int nmax;
  PwcWord pw;
  int q;  // n_table = 2^q
  __device__ Approx(const SampleArgs &a, float *smem) {  // smem: 2 n floats
    const int n = a.ntab;
    for (int i = threadIdx.x; i < n; i += blockDim.x) smem[i] = a.tab[i];
    __syncthreads();
    if (SRC == SRC_PHILOX) {  // the word-order copy from shared memory, not the parameter space
      for (int i = threadIdx.x; i < n; i += blockDim.x) smem[n + i] = smem[pwc_word_row(i, n)];
      __syncthreads();
    }
    s = smem;
    w = smem + n;
    nf = a.nf;
    nmax = n - 1;
    q = 23 - (int)a.pwc_shift;
    pw = pwc_word((uint32_t)q);
  }
  __device__ __forceinline__ float word(uint32_t x) const { return w[pwc_slot_from_word(x, pw)]; }
  __device__ __forceinline__ float operator()(float u) const { return pwc_eval(u, s, nf, nmax); }
  // cell m of a B-bit uniform: floor(2^q (m + 1/2) 2^-B)
  template <int B>
  __device__ __forceinline__ float cell(uint32_t m) const {
    return s[q <= B ? (m >> (B - q)) : ((2u * m + 1u) << (q - B - 1))];
  }
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
  __device__ __forceinline__ float word(uint32_t x) const { return pwl_eval_word(x, rows); }
  __device__ __forceinline__ float operator()(float u) const { return pwl_eval(u, c, kmax); }
  template <int B>
  __device__ __forceinline__ float cell(uint32_t m) const { return pwl_eval_t(tbits<B>(m), rows); }
};

template <int SRC>
struct Approx<AICDF_PWP, SRC> {
  const float4 *rows;  // kPwpStagedRows rows in shared memory
  __device__ Approx(const SampleArgs &a, float *smem) {
    float4 *r = reinterpret_cast<float4 *>(smem);
    pwp_stage_rows(a.tab, a.ntab, r);
    rows = r;
  }
  __device__ __forceinline__ float word(uint32_t x) const { return pwp_staged_word(x, rows); }
  __device__ __forceinline__ float operator()(float u) const { return pwp_staged(u, rows); }
  template <int B>
  __device__ __forceinline__ float cell(uint32_t m) const {
    return pwp_staged_t(tbits<B>(m), rows);
  }
};

template <int SRC>
struct Approx<AICDF_EXACT, SRC> {
  __device__ Approx(const SampleArgs &, float *) {}
  __device__ __forceinline__ float word(uint32_t x) const { return phiinv_f32_word(x); }
  __device__ __forceinline__ float operator()(float u) const { return phiinv_f32(u); }
  template <int B>
  __device__ __forceinline__ float cell(uint32_t m) const { return phiinv_f32_grid(ubits<B>(m)); }
};

template <int SRC>
struct Approx<AICDF_EXACT_LIB, SRC> {
  __device__ Approx(const SampleArgs &, float *) {}
  __device__ __forceinline__ float word(uint32_t x) const { return normcdfinvf(u01(x)); }
  __device__ __forceinline__ float operator()(float u) const { return normcdfinvf(u); }
  template <int B>
  __device__ __forceinline__ float cell(uint32_t m) const { return normcdfinvf(ubits<B>(m)); }
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

// The bits of one 16-byte output vector: 4 FP32 or 8 FP16 (round to nearest even).
__device__ __forceinline__ uint4 pack_vec(const float (&z)[4]) {
  return make_uint4(__float_as_uint(z[0]), __float_as_uint(z[1]), __float_as_uint(z[2]), __float_as_uint(z[3]));
}
__device__ __forceinline__ uint4 pack_vec(const float (&z)[8]) {
  uint4 w;
  __half2 h0 = __floats2half2_rn(z[0], z[1]), h1 = __floats2half2_rn(z[2], z[3]);
  __half2 h2 = __floats2half2_rn(z[4], z[5]), h3 = __floats2half2_rn(z[6], z[7]);
  w.x = *reinterpret_cast<uint32_t *>(&h0);
  w.y = *reinterpret_cast<uint32_t *>(&h1);
  w.z = *reinterpret_cast<uint32_t *>(&h2);
  w.w = *reinterpret_cast<uint32_t *>(&h3);
  return w;
}
__device__ __forceinline__ void store_vec(float *out, uint64_t e, const float (&z)[4]) {
  *reinterpret_cast<uint4 *>(out + e) = pack_vec(z);
}
__device__ __forceinline__ void store_vec(__half *out, uint64_t e, const float (&z)[8]) {
  *reinterpret_cast<uint4 *>(out + e) = pack_vec(z);
}
__device__ __forceinline__ void store_one(float *out, uint64_t e, float z) { out[e] = z; }
__device__ __forceinline__ void store_one(__half *out, uint64_t e, float z) {
  out[e] = __float2half_rn(z);
}

// Vectorised kernel.  Requires: out 16-byte aligned; SRC_PHILOX: offset % 4 == 0;
// SRC_INPUT: u 16-byte aligned.
template <int METHOD, int OUT, int SRC>
__global__ void __launch_bounds__(256) k_sample_vec(const __grid_constant__ SampleArgs a) {
  __shared__ __align__(16) float smem[METHOD == AICDF_PWC ? 2048 : METHOD == AICDF_PWP ? 4 * kPwpStagedRows : 1];
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

// The vectorised Philox kernel when every index fits in 32 bits (the host
// checks j0 + (nvec + 128) E/4 < 2^32 and (nvec + 128) E < 2^32): 32-bit index
// arithmetic, the counter's high words are the constant 0 (so the compiler
// folds part of the first round), and chunks that lie wholly inside the
// output are stored without per-vector bounds checks.  Each lane runs the
// Philox calls of its four 16-byte vectors interleaved round by round.  The
// counter of the lane's first call and the address of its first vector are
// carried from chunk to chunk (one add each per grid stride), so no vector
// address is formed by a 64-bit multiply: the kernel is bound by its integer
// multiply and logic pipes, and those products were ~6% of its multiply work.
template <int METHOD, int OUT>
__global__ void __launch_bounds__(256, 3) k_sample_philox32(const __grid_constant__ SampleArgs a) {
  __shared__ __align__(16) float smem[METHOD == AICDF_PWC ? 2048 : METHOD == AICDF_PWP ? 4 * kPwpStagedRows : 1];
  const Approx<METHOD, SRC_PHILOX> f(a, smem);
  using T = typename std::conditional<OUT == AICDF_F32, float, __half>::type;
  T *out = reinterpret_cast<T *>(a.out);
  constexpr int E = OutVec<OUT>::kElems;
  constexpr int VECS = OUT == AICDF_F32 ? 4 : 2;  // 16-byte vectors per lane per chunk
  constexpr int CPV = E / 4;                      // Philox calls per vector
  constexpr int NC = VECS * CPV;                  // Philox calls per lane per chunk (4)
  constexpr uint32_t CH = 32 * VECS;              // vectors per warp chunk
  const uint32_t n = (uint32_t)a.n;
  const uint32_t nvec = (n + E - 1) / E;
  const uint32_t nchunk = (nvec + CH - 1) / CH;
  const uint32_t nfull = (n / E) / CH;  // chunks with every vector complete
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  uint32_t chunk = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint32_t ctr = (uint32_t)(a.offset >> 2) + (chunk * CH + lane) * CPV;  // call of vector 0, word 0
  const uint32_t ctr_step = warps * CH * CPV;
  uint4 *pv = reinterpret_cast<uint4 *>(a.out) + (size_t)chunk * CH + lane;  // vector 0 of the lane
  const size_t pv_step = (size_t)warps * CH;
  for (; chunk < nchunk; chunk += warps, ctr += ctr_step, pv += pv_step) {
    uint4 c[NC];
#pragma unroll
    for (int hv = 0; hv < VECS; ++hv)
#pragma unroll
      for (int h = 0; h < CPV; ++h) c[hv * CPV + h] = make_uint4(ctr + 32 * CPV * hv + h, 0u, 0u, 0u);
    philox_n<NC>(c, a.keys);
    float z[VECS][E];
#pragma unroll
    for (int hv = 0; hv < VECS; ++hv)
#pragma unroll
      for (int h = 0; h < CPV; ++h) {
        const uint4 r = c[hv * CPV + h];
        z[hv][4 * h + 0] = f.word(r.x);
        z[hv][4 * h + 1] = f.word(r.y);
        z[hv][4 * h + 2] = f.word(r.z);
        z[hv][4 * h + 3] = f.word(r.w);
      }
    if (chunk < nfull) {  // warp-uniform
#pragma unroll
      for (int hv = 0; hv < VECS; ++hv) pv[32 * hv] = pack_vec(z[hv]);
    } else {
#pragma unroll
      for (int hv = 0; hv < VECS; ++hv) {
        const uint32_t e0 = (chunk * CH + 32 * hv + lane) * E;
        if (e0 + E <= n) {
          store_vec(out, e0, z[hv]);
        } else if (e0 < n) {
#pragma unroll
          for (int t = 0; t < E; ++t)
            if (e0 + t < n) store_one(out, e0 + t, z[hv][t]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Truncated-bit sampling: one Philox call gives S = 4F samples (F = 32/B
// B-bit fields per word); sample 4h + t of call j is field h of word t.  A
// thread owns one call and writes its S consecutive outputs as 32-byte
// (or, for 8 halves, 16-byte) vectors, so each warp store covers one
// contiguous 1 KiB / 512 B span.
__device__ __forceinline__ void st_v8(void *p, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                      uint32_t a4, uint32_t a5, uint32_t a6, uint32_t a7) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(a0), "r"(a1),
               "r"(a2), "r"(a3), "r"(a4), "r"(a5), "r"(a6), "r"(a7)
               : "memory");
}

__device__ __forceinline__ uint32_t pack_h2(float x, float y) {
  __half2 h = __floats2half2_rn(x, y);
  return *reinterpret_cast<uint32_t *>(&h);
}

// S consecutive samples at p (p aligned to 32 bytes, or 16 for 8 halves).
template <int S>
__device__ __forceinline__ void store_call(float *p, const float (&z)[S]) {
#pragma unroll
  for (int q = 0; q < S; q += 8)
    st_v8(p + q, __float_as_uint(z[q]), __float_as_uint(z[q + 1]), __float_as_uint(z[q + 2]),
          __float_as_uint(z[q + 3]), __float_as_uint(z[q + 4]), __float_as_uint(z[q + 5]),
          __float_as_uint(z[q + 6]), __float_as_uint(z[q + 7]));
}
template <int S>
__device__ __forceinline__ void store_call(__half *p, const float (&z)[S]) {
  if constexpr (S == 8) {
    *reinterpret_cast<uint4 *>(p) =
        make_uint4(pack_h2(z[0], z[1]), pack_h2(z[2], z[3]), pack_h2(z[4], z[5]), pack_h2(z[6], z[7]));
  } else {
#pragma unroll
    for (int q = 0; q < S; q += 16)
      st_v8(p + q, pack_h2(z[q], z[q + 1]), pack_h2(z[q + 2], z[q + 3]), pack_h2(z[q + 4], z[q + 5]),
            pack_h2(z[q + 6], z[q + 7]), pack_h2(z[q + 8], z[q + 9]), pack_h2(z[q + 10], z[q + 11]),
            pack_h2(z[q + 12], z[q + 13]), pack_h2(z[q + 14], z[q + 15]));
  }
}

template <int METHOD, int B>
__device__ __forceinline__ void call_samples(const Approx<METHOD, SRC_PHILOX> &f, const uint4 &r,
                                             float (&z)[4 * (32 / B)]) {
  constexpr int F = 32 / B;
  constexpr uint32_t M = (1u << B) - 1u;
  const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int h = 0; h < F; ++h)
#pragma unroll
    for (int t = 0; t < 4; ++t) z[4 * h + t] = f.template cell<B>((w[t] >> (h * B)) & M);
}

// Vector form.  Requires offset % S == 0 and out aligned to 32 bytes (16 for
// FP16 with S = 8).  A warp chunk is NC x 32 calls; lane L runs calls
// q x 32 + L (q < NC) interleaved, and each q writes one contiguous span.
template <int METHOD, int OUT, int B>
__global__ void __launch_bounds__(256) k_sample_bits(const __grid_constant__ SampleArgs a) {
  __shared__ __align__(16) float smem[METHOD == AICDF_PWC ? 2048 : METHOD == AICDF_PWP ? 4 * kPwpStagedRows : 1];
  const Approx<METHOD, SRC_PHILOX> f(a, smem);
  using T = typename std::conditional<OUT == AICDF_F32, float, __half>::type;
  T *out = reinterpret_cast<T *>(a.out);
  constexpr int S = 4 * (32 / B);
  constexpr int NC = B == 16 ? 4 : 2;
  const uint64_t ncall = (a.n + S - 1) / S;
  const uint64_t nchunk = (ncall + 32 * NC - 1) / (32 * NC);
  const uint64_t j0 = a.offset / S;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  // warp-uniform loop: every lane runs every iteration (shuffles need all 32)
  for (uint64_t chunk = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; chunk < nchunk;
       chunk += warps) {
    uint4 r[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const uint64_t j = j0 + chunk * (32 * NC) + 32 * q + lane;
      r[q] = make_uint4((uint32_t)j, (uint32_t)(j >> 32), 0u, 0u);
    }
    philox_n<NC>(r, a.keys);
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const uint64_t c = chunk * (32 * NC) + 32 * q + lane;  // call index relative to j0
      float z[S];
      call_samples<METHOD, B>(f, r[q], z);
      const uint64_t e0 = c * S;
      if (e0 + S <= a.n) {
        store_call<S>(out + e0, z);
      } else if (e0 < a.n) {
#pragma unroll
        for (int t = 0; t < S; ++t)
          if (e0 + t < a.n) store_one(out, e0 + t, z[t]);
      }
    }
  }
}

// Any offset / alignment: one output element per lane (the lane recomputes
// its call; only for ragged or unaligned requests).
template <int METHOD, int OUT, int B>
__global__ void __launch_bounds__(256) k_sample_bits_scalar(const __grid_constant__ SampleArgs a) {
  __shared__ __align__(16) float smem[METHOD == AICDF_PWC ? 2048 : METHOD == AICDF_PWP ? 4 * kPwpStagedRows : 1];
  const Approx<METHOD, SRC_PHILOX> f(a, smem);
  using T = typename std::conditional<OUT == AICDF_F32, float, __half>::type;
  T *out = reinterpret_cast<T *>(a.out);
  constexpr int F = 32 / B;
  constexpr int S = 4 * F;
  constexpr uint32_t M = (1u << B) - 1u;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < a.n;
       base += stride) {
    const uint64_t e = base + lane;
    const uint64_t s = a.offset + e;
    const uint64_t j = s / S;
    const uint32_t r = (uint32_t)(s % S), h = r >> 2, t = r & 3;
    const uint4 q = philox(make_uint4((uint32_t)j, (uint32_t)(j >> 32), 0u, 0u), a.keys);
    const uint32_t w = t == 0 ? q.x : t == 1 ? q.y : t == 2 ? q.z : q.w;
    const float y = f.template cell<B>((w >> (h * B)) & M);
    if (e < a.n) store_one(out, e, y);
  }
}

// Scalar kernel for unaligned pointers or an offset not divisible by 4.
template <int METHOD, int OUT, int SRC>
__global__ void __launch_bounds__(256) k_sample_scalar(const __grid_constant__ SampleArgs a) {
  __shared__ __align__(16) float smem[METHOD == AICDF_PWC ? 2048 : METHOD == AICDF_PWP ? 4 * kPwpStagedRows : 1];
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


}  // namespace aicdf
