// The surrogate network on tcgen05: pieces shared by the batched evaluation,
// the training step and the CIR path kernel.  A CTA of 128 threads holds a
// tile of 128 samples (thread = sample = row): layer 1 (FP32, tanh) writes the
// row's H1 in BF16 into a shared tile in the canonical K-major layout, one
// thread issues the 128 x 64 x 64 product H1 W2^T as four depth-16 MMAs into a
// 64-column TMEM accumulator, and each thread reads its row of Z2 back for
// tanh(Z2 + b2) . w3 + b3.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

#include "mlp_device.cuh"
#include "tc_device.cuh"

namespace aicdf {

constexpr int kTcRows = 128;  // samples per tile (the MMA's M)

// The surrogate handle keeps W2 in BF16 in the canonical layout twice --
// W2 [n][k] (kW2cBytes) then W2^T [k][n] -- so that a CTA loads it with one
// bulk copy.
constexpr uint32_t kW2cBytes = kH * kH * sizeof(__nv_bfloat16);

// The network's FP32 vectors, staged per CTA.
struct MlpVecs {
  float w1[2 * kH], b1[kH], b2[kH], w3[kH], b3;
};

__device__ __forceinline__ void mlp_stage_vecs(const float *__restrict__ p, MlpVecs &v) {
  for (int i = threadIdx.x; i < 2 * kH; i += blockDim.x) v.w1[i] = p[kOffW1 + i];
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    v.b1[i] = p[kOffB1 + i];
    v.b2[i] = p[kOffB2 + i];
    v.w3[i] = p[kOffW3 + i];
  }
  if (threadIdx.x == 0) v.b3 = p[kOffB3];
}

// Layer 1 of sample (x0, x1) into row `row` of a 128 x 64 BF16 canonical tile.
__device__ __forceinline__ void mlp_tc_layer1(const MlpVecs &s, __nv_bfloat16 *tile, int row, float x0, float x1) {
  unsigned char *base = reinterpret_cast<unsigned char *>(tile);
#pragma unroll
  for (int j = 0; j < kH / 8; ++j) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 8 * j + 2 * q;
      const float h0 = tanh_fast(fmaf(s.w1[2 * k], x0, fmaf(s.w1[2 * k + 1], x1, s.b1[k])));
      const float h1 = tanh_fast(fmaf(s.w1[2 * k + 2], x0, fmaf(s.w1[2 * k + 3], x1, s.b1[k + 1])));
      w[q] = pack_bf16(h0, h1);
    }
    *reinterpret_cast<uint4 *>(base + tc_canon_off64(row, 8 * j)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Z2 = H1 W2^T into the accumulator at d_tmem (one thread), completion on mbar.
__device__ __forceinline__ void mlp_tc_issue(uint32_t d_tmem, uint32_t a_base, uint32_t b_base, uint32_t mbar) {
  constexpr uint32_t idesc = tc_idesc_bf16(kTcRows, kH);
#pragma unroll
  for (int kk = 0; kk < kH / 16; ++kk)
    tc_mma_bf16(d_tmem, tc_desc(a_base + 256 * kk, 128, 1024), tc_desc(b_base + 256 * kk, 128, 1024), idesc,
                kk > 0);
  tc_commit(mbar);
}

// tanh(Z2 + b2) . w3 + b3 for this thread's row: `row_tmem` addresses the
// accumulator's first column in this warp's lane quarter.  Warp-collective.
__device__ __forceinline__ float mlp_tc_output(const MlpVecs &s, uint32_t row_tmem) {
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < kH; c += 16) {
    float v[16];
    tc_ld16(row_tmem + (uint32_t)c, v);
#pragma unroll
    for (int q = 0; q < 16; ++q) acc = fmaf(s.w3[c + q], tanh_fast(v[q] + s.b2[c + q]), acc);
  }
  return acc + s.b3;
}

}  // namespace aicdf
