// The surrogate network on tcgen05: pieces shared by the batched evaluation
// and the training step.  A CTA holds a tile of 128 samples (one per row) with
// two threads per sample, each owning half of the 64 hidden units: layer 1
// (FP32, tanh) writes the thread's half of the row's H1 in BF16 into a shared
// tile in the canonical K-major layout, one thread issues the 128 x 64 x 64
// product H1 W2^T as four depth-16 MMAs into a 64-column TMEM accumulator, and
// each thread reads its half of the row of Z2 back for its half of
// tanh(Z2 + b2) . w3; the two halves are added in a fixed order.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

#include "mlp_device.cuh"
#include "tc_device.cuh"

namespace aicdf {

constexpr int kTcRows = 128;  // samples per tile (the MMA's M)
constexpr int kHalf = kH / 2;  // hidden units per thread

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

// Layer 1, hidden units c0 .. c0 + kHalf - 1, of two samples into row `row`
// of two 128 x 64 BF16 canonical tiles: sample (xa0, xa1) into tile_a and
// (xb0, xb1) into tile_b, each weight read once for both.
__device__ __forceinline__ void mlp_tc_layer1_pair(const MlpVecs &s, __nv_bfloat16 *tile_a, __nv_bfloat16 *tile_b,
                                                   int row, int c0, float xa0, float xa1, float xb0, float xb1) {
  unsigned char *ba = reinterpret_cast<unsigned char *>(tile_a), *bb = reinterpret_cast<unsigned char *>(tile_b);
#pragma unroll
  for (int j = 0; j < kHalf / 8; ++j) {
    uint32_t wa[4], wb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = c0 + 8 * j + 2 * q;
      const float p0 = s.w1[2 * k], p1 = s.w1[2 * k + 1], p2 = s.w1[2 * k + 2], p3 = s.w1[2 * k + 3];
      const float q0 = s.b1[k], q1 = s.b1[k + 1];
      wa[q] = pack_bf16(tanh_fast(fmaf(p0, xa0, fmaf(p1, xa1, q0))), tanh_fast(fmaf(p2, xa0, fmaf(p3, xa1, q1))));
      wb[q] = pack_bf16(tanh_fast(fmaf(p0, xb0, fmaf(p1, xb1, q0))), tanh_fast(fmaf(p2, xb0, fmaf(p3, xb1, q1))));
    }
    const uint32_t off = tc_canon_off64(row, c0 + 8 * j);
    *reinterpret_cast<uint4 *>(ba + off) = make_uint4(wa[0], wa[1], wa[2], wa[3]);
    *reinterpret_cast<uint4 *>(bb + off) = make_uint4(wb[0], wb[1], wb[2], wb[3]);
  }
}

// Z2 = H1 W2^T into the accumulator at d_tmem (one thread).
__device__ __forceinline__ void mlp_tc_issue(uint32_t d_tmem, uint32_t a_base, uint32_t b_base) {
  constexpr uint32_t idesc = tc_idesc_bf16(kTcRows, kH);
#pragma unroll
  for (int kk = 0; kk < kH / 16; ++kk)
    tc_mma_bf16(d_tmem, tc_desc(a_base + 256 * kk, 128, 1024), tc_desc(b_base + 256 * kk, 128, 1024), idesc,
                kk > 0);
}

// The halves of tanh(Z2 + b2) . w3 over columns c0 .. c0 + kHalf - 1 of this
// thread's row in two accumulators (at row_tmem and row_tmem + kH), each added
// in column order; `row_tmem` addresses the first accumulator's first column in
// this warp's lane quarter.  Warp-collective.
__device__ __forceinline__ void mlp_tc_output_half_pair(const MlpVecs &s, uint32_t row_tmem, int c0, float &ya,
                                                        float &yb) {
  ya = 0.f;
  yb = 0.f;
#pragma unroll
  for (int c = 0; c < kHalf; c += 16) {
    float va[16], vb[16];
    tc_ld16(row_tmem + (uint32_t)(c0 + c), va);
    tc_ld16(row_tmem + (uint32_t)(kH + c0 + c), vb);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float w = s.w3[c0 + c + q], b = s.b2[c0 + c + q];
      ya = fmaf(w, tanh_fast(va[q] + b), ya);
      yb = fmaf(w, tanh_fast(vb[q] + b), yb);
    }
  }
}

}  // namespace aicdf
