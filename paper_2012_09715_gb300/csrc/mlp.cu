// Learned surrogate for the non-central chi-squared inverse CDF (Section 5.1):
// P~(U; lambda) = Phi^{-1}(U) + sqrt(y) N(s(U)/3, 2 sqrt(y) - 1) ~ P_nu(U; y),
// y = nu / (lambda + nu), so that C~^{-1}_nu(U; lambda) = lambda + nu +
// 2 sqrt(lambda + nu) P~ (mlp_device.cuh explains the form).
//
// Kernels: batched evaluation and a fused forward + backward training step,
// both with their 64-wide products (layer 2, dH1 = dZ2 W2, dW2 = dZ2^T H1) as
// tcgen05 MMAs in BF16 into TMEM FP32 accumulators; a fixed-order reduction
// of the per-block gradients with an Adam update of FP32 master weights; and
// the generation of exact training targets with the FP64 root finder.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "aicdf_internal.h"
#include "device_common.cuh"
#include "mlp_device.cuh"
#include "ncx2.cuh"
#include "mlp_tc.cuh"
#include "tc_device.cuh"

namespace aicdf {

constexpr int kGradSlots = kMlpParams;         // per-block partial: params + loss at kLossSlot
constexpr int kLossSlot = kOffB3 + 1;          // 4417

// ------------------------------------------------------------------ evaluation
// Batched evaluation on tcgen05 (the pieces in mlp_tc.cuh): a CTA of 256
// threads takes tiles of 128 samples two at a time (thread t: sample t mod 128
// of both tiles, hidden units 32 (t / 128) .. +31; both halves of a warp group
// read the same TMEM lane quarter), so that each FP32 weight read from shared
// memory serves two samples.  The pair's two MMAs go to two 64-column
// accumulators under one commit; other CTAs on the SM fill the wait.  Inputs
// are loaded one pair ahead.  The network's output is b3 + (lower half + upper
// half), the training step's forward value, and the sample is
// Phi^{-1}(u) + sqrt(y) times it.  Should the MMAs' completion not arrive
// within the bounded wait, the pair's outputs are NaN and the CTA stops.
constexpr int kEvalThreads = 2 * kTcRows;
constexpr uint32_t kTcCols = 128;  // TMEM columns per CTA: two 64-column accumulators

struct MlpTcSmem {
  __nv_bfloat16 a[2][kTcRows * kH];  // H1 tiles (2 x 16 KiB)
  __nv_bfloat16 b[kH * kH];          // W2 [out][in] (8 KiB)
  MlpVecs v;
  float ypart[2][kTcRows];           // upper halves of the pair's outputs
  unsigned long long mbar, wbar;
  uint32_t tmem;
};
// Dynamic shared memory per CTA, padded so that at most 4 CTAs fit an SM and
// their TMEM (4 x 128 columns) never exceeds the SM's 512 columns.
constexpr size_t kTcSmemBytes = 52 * 1024;
static_assert(sizeof(MlpTcSmem) + 1024 <= kTcSmemBytes, "tile layout exceeds the padded allocation");

__global__ void __launch_bounds__(kEvalThreads, 4)
    k_mlp_eval(const float *__restrict__ params, const __nv_bfloat16 *__restrict__ w2c,
               const float *__restrict__ u, const float *__restrict__ lam, float *__restrict__ out, uint64_t n,
               float nu) {
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  MlpTcSmem &s = *reinterpret_cast<MlpTcSmem *>(tc_raw + ((1024 - (tc_smem(tc_raw) & 1023)) & 1023));
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m = tid & (kTcRows - 1), hf = tid >> 7, c0 = kHalf * hf;  // sample, half, first unit
  if (tid == 0) {  // W2 (BF16, canonical) by one bulk copy
    tc_mbar_init(tc_smem(&s.wbar), 1);
    tc_bulk_g2s(tc_smem(s.b), w2c, kW2cBytes, tc_smem(&s.wbar));
  }
  mlp_stage_vecs(params, s.v);
  if (tid == 0) tc_mbar_init(tc_smem(&s.mbar), 1);
  if (warp == 0) tc_alloc(tc_smem(&s.tmem), kTcCols);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = s.tmem, b_base = tc_smem(s.b);
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;  // this warp's TMEM lane quarter
  // the MMA issuer needs W2 in place; a copy that never lands leaves NaN outputs
  const bool w2_ok = tid == 0 ? tc_mbar_wait(tc_smem(&s.wbar), 0) : true;
  const uint64_t ntiles = (n + kTcRows - 1) / kTcRows, step = 2 * (uint64_t)gridDim.x;
  auto load = [&](uint64_t tile, float &ru, float &rl) {  // raw inputs of one row of a tile
    const uint64_t i = tile * kTcRows + m;
    ru = tile < ntiles && i < n ? u[i] : 0.5f;
    rl = tile < ntiles && i < n ? lam[i] : 1.0f;
  };
  uint64_t t0 = 2 * (uint64_t)blockIdx.x;  // first tile of this CTA's pair
  float pua, pla, pub, plb;                  // inputs of the pair at t0
  load(t0, pua, pla);
  load(t0 + 1, pub, plb);
  for (uint32_t j = 0; t0 < ntiles; t0 += step, ++j) {
    const float sya = mlp_sqrt_y(pla, nu), syb = mlp_sqrt_y(plb, nu);
    const float xa0 = mlp_feature_u(pua), xa1 = mlp_feature_y(sya);
    const float xb0 = mlp_feature_u(pub), xb1 = mlp_feature_y(syb);
    const float za = phiinv_f32(pua), zb = phiinv_f32(pub);
    load(t0 + step, pua, pla);  // the next pair's inputs, in flight during this pair
    load(t0 + step + 1, pub, plb);
    mlp_tc_layer1_pair(s.v, s.a[0], s.a[1], m, c0, xa0, xa1, xb0, xb1);
    tc_fence_smem_to_async();
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    if (tid == 0 && w2_ok) {
      mlp_tc_issue(tmem, tc_smem(s.a[0]), b_base);
      mlp_tc_issue(tmem + kH, tc_smem(s.a[1]), b_base);
      tc_commit(tc_smem(&s.mbar));
    }
    // warp-uniform, as the TMEM loads below are warp-collective
    const bool done = __all_sync(0xffffffffu, tc_mbar_wait(tc_smem(&s.mbar), j & 1));
    tc_fence_after_sync();
    float ya = __int_as_float(0x7fc00000), yb = ya;
    if (done) mlp_tc_output_half_pair(s.v, tmem + lane_base, c0, ya, yb);
    if (hf) {
      s.ypart[0][m] = ya;
      s.ypart[1][m] = yb;
    }
    tc_fence_before_sync();
    __syncthreads();  // ypart written; H1 tiles and accumulators free for the next pair
    tc_fence_after_sync();
    if (!hf) {
      const uint64_t ia = t0 * kTcRows + m, ib = ia + kTcRows;
      if (ia < n) out[ia] = fmaf(sya, s.v.b3 + (ya + s.ypart[0][m]), za);
      if (ib < n) out[ib] = fmaf(syb, s.v.b3 + (yb + s.ypart[1][m]), zb);
    }
    if (!__syncthreads_and(done)) break;  // also: ypart read before the next pair writes it
  }
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, kTcCols);
}

// ------------------------------------------------------------------ training
// One CTA = 128 consecutive samples of the batch, two threads per sample
// (thread t: sample m = t mod 128, hidden units 32 (t / 128) .. +31), the
// three 64-wide products on tcgen05 with TMEM accumulators:
//   Z2  = H1 W2^T      (M 128 samples, N 64, K 64)   TMEM columns   0..63
//   dH1 = dZ2 W2       (M 128 samples, N 64, K 64)   TMEM columns  64..127
//   dW2 = dZ2^T H1     (M 64 outputs padded to 128 with zero rows, N 64,
//                       K 128 samples)               TMEM columns 128..191
// BF16 operands in the canonical K-major shared layout (H1^T and dZ2^T are
// written column by column; W2 and W2^T arrive by one bulk copy); everything
// else in FP32.  The column sums over the CTA's samples (gradients of w3, b2,
// b1, W1) go through a transposing shared buffer and are added in a fixed
// order, so the partials are deterministic.  The network is fitted to
// g_i = (t_i - Phi^{-1}(u_i)) / sqrt(y_i) for the target t_i of P (the form
// of mlp_device.cuh).  Writes the CTA's gradient of sum_i (N_i - g_i)^2 * scale
// and its sum of (N_i - g_i)^2 to partial[blockIdx].
constexpr int kTrainThreads = 2 * kTcRows;
constexpr uint32_t kTrainCols = 256;  // TMEM columns (three 64-column accumulators)

struct MlpTrainSmem {
  __nv_bfloat16 w2k[kH * kH];           // W2 [n][k]: B of Z2
  __nv_bfloat16 w2t[kH * kH];           // W2^T [k][n]: B of dH1
  __nv_bfloat16 h1[kTcRows * kH];       // H1 [m][k]: A of Z2
  __nv_bfloat16 dz2[kTcRows * kH];      // dZ2 [m][n]: A of dH1
  __nv_bfloat16 dz2t[kTcRows * kTcRows];  // dZ2^T [n][m], rows 64..127 zero: A of dW2
  __nv_bfloat16 h1t[kH * kTcRows];      // H1^T [k][m]: B of dW2
  float red[kTcRows][3 * kH + 1];       // column sums, up to three 64-wide quantities a pass (pitch 193)
  float psum[2][2 * kH];                // the two row halves of a pass's column sums
  float ypart[2][kTcRows];              // the two halves of each sample's output
  float w1[2 * kH], b1[kH], b2[kH], w3[kH], b3;
  float wsum[kTcRows / 32][2];          // per-warp sums of dy and err^2
  unsigned long long mbar, wbar;
  uint32_t tmem;
};
static_assert(offsetof(MlpTrainSmem, w2t) == offsetof(MlpTrainSmem, w2k) + kW2cBytes, "W2 tiles not adjacent");
constexpr size_t kTrainSmem = sizeof(MlpTrainSmem) + 1024;
static_assert(kTrainSmem <= 227u * 1024u, "training CTA exceeds the 227 KB of shared memory a CTA may opt in to");

// byte offset of (r, k) in a canonical K-major tile with K = 128
__device__ __forceinline__ uint32_t canon_off128(int r, int k) {
  return (uint32_t)((r >> 3) * 2048 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Column sums of red[0..127][c], c < ncols (<= 128), in a fixed order: thread
// t sums column t mod 128 over rows 64 (t / 128) .. +63 as eight interleaved
// partial sums, and the two row halves are then added.  The caller has filled
// red and passed a barrier; two barriers inside, so red may be refilled after.
__device__ __forceinline__ float train_colsum(MlpTrainSmem &s, int ncols) {
  const int tid = threadIdx.x, c = tid & (kTcRows - 1), rh = tid >> 7;
  if (c < ncols) {
    float p[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int r = 0; r < kTcRows / 16; ++r)
#pragma unroll
      for (int q = 0; q < 8; ++q) p[q] += s.red[64 * rh + 8 * r + q][c];
    s.psum[rh][c] = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
  }
  __syncthreads();
  const float a = (rh == 0 && c < ncols) ? s.psum[0][c] + s.psum[1][c] : 0.f;
  __syncthreads();
  return a;
}

// Column sums of red[0..127][c] for all c < 3 kH in a fixed order: thread c
// sums its column over the 128 rows as eight interleaved partial sums.  The
// caller has filled red and passed a barrier; one barrier inside, so red may be
// refilled after.
__device__ __forceinline__ float train_colsum_wide(MlpTrainSmem &s) {
  const int c = threadIdx.x;
  float a = 0.f;
  if (c < 3 * kH) {
    float p[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int r = 0; r < kTcRows / 8; ++r)
#pragma unroll
      for (int q = 0; q < 8; ++q) p[q] += s.red[8 * r + q][c];
    a = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
  }
  __syncthreads();
  return a;
}

// Programmatic dependent launch, used between the training graph's gradient
// and Adam launches: a kernel launched with the programmatic-serialization
// attribute may start while its predecessor is still running.  pdl_wait()
// returns once the predecessor grid has completed and its writes are visible
// (at once for a kernel launched without the attribute); after
// pdl_launch_dependents() in every CTA the successor may start its prologue.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// A training sample's network inputs and target: (x0, x1, g) of (u, lambda,
// target) -- the features of mlp_device.cuh and g = (target - Phi^{-1}(u)) /
// sqrt(y).  The training loop computes them once per call into a float4 per
// sample (w unused) instead of once per epoch inside the gradient kernel.
__device__ __forceinline__ float3 train_features(float ui, float li, float ti, float nu) {
  const float sy = mlp_sqrt_y(li, nu);
  return make_float3(mlp_feature_u(ui), mlp_feature_y(sy), (ti - phiinv_f32(ui)) / sy);
}

__global__ void k_mlp_features(const float *__restrict__ u, const float *__restrict__ lam,
                               const float *__restrict__ target, uint64_t n, float nu, float4 *__restrict__ feat) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const float3 f = train_features(u[i], lam[i], target[i], nu);
    feat[i] = make_float4(f.x, f.y, f.z, 0.f);
  }
}

// FEAT: the samples' (x0, x1, g) come from feat (k_mlp_features); otherwise
// from u, lam and target here.
template <bool FEAT>
__global__ void __launch_bounds__(kTrainThreads)
    k_mlp_train(const float *__restrict__ params, const __nv_bfloat16 *__restrict__ w2c,
                const float *__restrict__ u, const float *__restrict__ lam, const float *__restrict__ target,
                const float4 *__restrict__ feat, uint64_t begin, uint64_t count, float scale,
                float *__restrict__ partial, float nu, long long *__restrict__ step_count) {
  extern __shared__ __align__(1024) unsigned char tr_raw[];
  MlpTrainSmem &s = *reinterpret_cast<MlpTrainSmem *>(tr_raw + ((1024 - (tc_smem(tr_raw) & 1023)) & 1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = tid & (kTcRows - 1), hf = tid >> 7, c0 = kHalf * hf;  // sample, half, first unit
  unsigned char *w2k = reinterpret_cast<unsigned char *>(s.w2k), *w2t = reinterpret_cast<unsigned char *>(s.w2t);
  unsigned char *h1 = reinterpret_cast<unsigned char *>(s.h1), *dz2 = reinterpret_cast<unsigned char *>(s.dz2);
  unsigned char *dz2t = reinterpret_cast<unsigned char *>(s.dz2t), *h1t = reinterpret_cast<unsigned char *>(s.h1t);
  if (warp == 0) tc_alloc(tc_smem(&s.tmem), kTrainCols);
  // ---- this thread's sample (inputs no launch writes), before the wait for
  // the previous Adam step
  const uint64_t m_idx = (uint64_t)blockIdx.x * kTcRows + m;
  const bool ok = m_idx < count;
  const uint64_t i = begin + m_idx;
  float3 f = make_float3(0.f, 0.f, 0.f);  // (x0, x1, g); g is the network's own target
  if (ok) {
    if constexpr (FEAT) {
      const float4 q = feat[i];
      f = make_float3(q.x, q.y, q.z);
    } else {
      f = train_features(u[i], lam[i], target[i], nu);
    }
  }
  const float x0 = f.x, x1 = f.y, tg = f.z;
  for (int c = tid; c < (kTcRows - kH) * kTcRows / 8; c += blockDim.x)  // rows 64..127 of dZ2^T
    *reinterpret_cast<uint4 *>(dz2t + (size_t)(kH / 8) * 2048 + 16 * (size_t)c) = make_uint4(0u, 0u, 0u, 0u);
  // the Adam step after this one may start (it waits for these partials); the
  // parameters, W2 and the step counter below come from the Adam step before
  pdl_launch_dependents();
  pdl_wait();
  // ---- W2 and W2^T (BF16, canonical, adjacent) by one bulk copy; the FP32
  // vectors by the threads
  if (tid == 0) {
    tc_mbar_init(tc_smem(&s.wbar), 1);
    tc_bulk_g2s(tc_smem(w2k), w2c, 2 * kW2cBytes, tc_smem(&s.wbar));
  }
  for (int c = tid; c < 2 * kH; c += blockDim.x) s.w1[c] = params[kOffW1 + c];
  for (int c = tid; c < kH; c += blockDim.x) {
    s.b1[c] = params[kOffB1 + c];
    s.b2[c] = params[kOffB2 + c];
    s.w3[c] = params[kOffW3 + c];
  }
  if (tid == 0) {
    s.b3 = params[kOffB3];
    tc_mbar_init(tc_smem(&s.mbar), 1);
  }
  if (step_count && blockIdx.x == 0 && tid == 0) *step_count += 1;  // the Adam kernel after this reads it
  __syncthreads();  // vectors staged
  // ---- layer 1: this thread's 32 units of H1 (BF16), by rows and by columns
#pragma unroll
  for (int j = 0; j < kHalf / 8; ++j) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = c0 + 8 * j + 2 * q;
      const float a = tanh_fast(fmaf(s.w1[2 * k], x0, fmaf(s.w1[2 * k + 1], x1, s.b1[k])));
      const float b = tanh_fast(fmaf(s.w1[2 * k + 2], x0, fmaf(s.w1[2 * k + 3], x1, s.b1[k + 1])));
      const __nv_bfloat162 hb = __floats2bfloat162_rn(a, b);
      w[q] = pack_bf16(a, b);
      *reinterpret_cast<__nv_bfloat16 *>(h1t + canon_off128(k, m)) = hb.x;
      *reinterpret_cast<__nv_bfloat16 *>(h1t + canon_off128(k + 1, m)) = hb.y;
    }
    *reinterpret_cast<uint4 *>(h1 + tc_canon_off64(m, c0 + 8 * j)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  tc_fence_smem_to_async();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = s.tmem;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;  // this warp's TMEM lane quarter
  constexpr uint32_t idesc = tc_idesc_bf16(kTcRows, kH);
  // the MMA issuer needs W2 in place; a copy that never lands leaves NaN gradients
  const bool w2_ok = tid == 0 ? tc_mbar_wait(tc_smem(&s.wbar), 0) : true;
  if (tid == 0 && w2_ok) {
#pragma unroll
    for (int kk = 0; kk < kH / 16; ++kk)
      tc_mma_bf16(tmem, tc_desc(tc_smem(h1) + 256 * kk, 128, 1024), tc_desc(tc_smem(w2k) + 256 * kk, 128, 1024),
                  idesc, kk > 0);
    tc_commit(tc_smem(&s.mbar));
  }
  bool done = __all_sync(0xffffffffu, tc_mbar_wait(tc_smem(&s.mbar), 0));
  tc_fence_after_sync();
  // ---- layer 2 activation on this thread's 32 units; the output from both halves
  float h2[kHalf], v[kHalf];
#pragma unroll
  for (int c = 0; c < kHalf; c += 16) {
    float z[16];
    if (done) tc_ld16(tmem + lane_base + (uint32_t)(c0 + c), z);
#pragma unroll
    for (int q = 0; q < 16; ++q) h2[c + q] = done ? tanh_fast(z[q] + s.b2[c0 + c + q]) : 0.f;
  }
  float yp = 0.f;
#pragma unroll
  for (int c = 0; c < kHalf; ++c) yp = fmaf(s.w3[c0 + c], h2[c], yp);
  s.ypart[hf][m] = yp;
  __syncthreads();
  const float y = s.b3 + (s.ypart[0][m] + s.ypart[1][m]);  // the same in both threads of a sample
  const float err = ok ? y - tg : 0.f;
  const float dy = 2.0f * err * scale;
  // ---- dZ2 on this thread's 32 units, by rows and by columns
#pragma unroll
  for (int j = 0; j < kHalf / 8; ++j) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 8 * j + 2 * q, n = c0 + c;
      const float d0 = dy * s.w3[n] * (1.f - h2[c] * h2[c]);
      const float d1 = dy * s.w3[n + 1] * (1.f - h2[c + 1] * h2[c + 1]);
      v[c] = d0;
      v[c + 1] = d1;
      const __nv_bfloat162 db = __floats2bfloat162_rn(d0, d1);
      w[q] = pack_bf16(d0, d1);
      *reinterpret_cast<__nv_bfloat16 *>(dz2t + canon_off128(n, m)) = db.x;
      *reinterpret_cast<__nv_bfloat16 *>(dz2t + canon_off128(n + 1, m)) = db.y;
    }
    *reinterpret_cast<uint4 *>(dz2 + tc_canon_off64(m, c0 + 8 * j)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  // FP32 rows for the column sums: dZ2 (gradient of b2) and dy h2 (of w3)
#pragma unroll
  for (int c = 0; c < kHalf; ++c) {
    s.red[m][c0 + c] = v[c];
    s.red[m][kH + c0 + c] = dy * h2[c];
  }
  tc_fence_smem_to_async();
  tc_fence_before_sync();
  __syncthreads();  // dZ2 tiles and red rows complete
  tc_fence_after_sync();
  if (tid == 0 && w2_ok) {  // dH1 = dZ2 W2 and dW2 = dZ2^T H1, in flight during the sums below
#pragma unroll
    for (int kk = 0; kk < kH / 16; ++kk)
      tc_mma_bf16(tmem + 64, tc_desc(tc_smem(dz2) + 256 * kk, 128, 1024),
                  tc_desc(tc_smem(w2t) + 256 * kk, 128, 1024), idesc, kk > 0);
#pragma unroll
    for (int kk = 0; kk < kTcRows / 16; ++kk)
      tc_mma_bf16(tmem + 128, tc_desc(tc_smem(dz2t) + 256 * kk, 128, 2048),
                  tc_desc(tc_smem(h1t) + 256 * kk, 128, 2048), idesc, kk > 0);
    tc_commit(tc_smem(&s.mbar));
  }
  float *out = partial + (size_t)blockIdx.x * kGradSlots;
  {
    const float a = train_colsum(s, 2 * kH);
    if (tid < kTcRows) out[(tid < kH ? kOffB2 : kOffW3 - kH) + tid] = a;
  }
  done = __all_sync(0xffffffffu, tc_mbar_wait(tc_smem(&s.mbar), 1)) && done;
  tc_fence_after_sync();
  // ---- dZ1 = dH1 (1 - h1^2) on this thread's 32 units, h1 as stored (BF16)
  float dz1[kHalf];
#pragma unroll
  for (int c = 0; c < kHalf; c += 16) {
    float d[16];
    if (done) tc_ld16(tmem + 64 + lane_base + (uint32_t)(c0 + c), d);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float hv = __bfloat162float(
          *reinterpret_cast<const __nv_bfloat16 *>(h1 + tc_canon_off64(m, c0 + c + q)));
      dz1[c + q] = done ? d[q] * (1.f - hv * hv) : 0.f;
    }
  }
#pragma unroll
  for (int c = 0; c < kHalf; ++c) {
    s.red[m][c0 + c] = dz1[c];
    s.red[m][kH + c0 + c] = dz1[c] * x0;
    s.red[m][2 * kH + c0 + c] = dz1[c] * x1;
  }
  __syncthreads();
  {
    const float a = train_colsum_wide(s);  // gradients of b1, W1[., 0] and W1[., 1] in one pass
    if (tid < 3 * kH)
      out[tid < kH ? kOffB1 + tid : tid < 2 * kH ? kOffW1 + 2 * (tid - kH) : kOffW1 + 2 * (tid - 2 * kH) + 1] = a;
  }
  // ---- dW2 rows n = TMEM lanes 0..63 (warps 0, 1 and 4, 5 for the two
  // column halves; every warp runs the warp-collective loads), staged in
  // `red` (free again after the last column sum) so that the 64 x 64 block
  // goes out in coalesced rows: a lane's own row is 256 bytes from its
  // neighbour's, and stored directly every warp store touched 32 sectors
#pragma unroll
  for (int c = 0; c < kHalf; c += 16) {
    float d[16];
    if (done) tc_ld16(tmem + 128 + lane_base + (uint32_t)(c0 + c), d);
    if (m < kH) {
#pragma unroll
      for (int q = 0; q < 16; ++q) s.red[m][c0 + c + q] = done ? d[q] : __int_as_float(0x7fc00000);
    }
  }
  __syncthreads();
  for (int i = tid; i < kH * kH; i += kTrainThreads) out[kOffW2 + i] = s.red[i / kH][i % kH];
  // ---- sums of dy (gradient of b3) and err^2 over the samples (first half
  // of the threads), in a fixed order
  if (hf == 0) {
    float sdy = dy, loss = err * err;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sdy += __shfl_xor_sync(0xffffffffu, sdy, o);
      loss += __shfl_xor_sync(0xffffffffu, loss, o);
    }
    if (lane == 0) {
      s.wsum[warp][0] = sdy;
      s.wsum[warp][1] = loss;
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  if (tid == 0) {
    float a = 0.f, l = 0.f;
    for (int w = 0; w < kTcRows / 32; ++w) {
      a += s.wsum[w][0];
      l += s.wsum[w][1];
    }
    out[kOffB3] = done ? a : __int_as_float(0x7fc00000);
    out[kLossSlot] = l;
  }
  if (warp == 0) tc_dealloc(tmem, kTrainCols);
}

// Sum of partial[b * kGradSlots + p] over the blocks b in a fixed order: eight
// interleaved chains (b mod 8) combined pairwise, so that the loads overlap.
__device__ __forceinline__ float sum_partials(const float *__restrict__ partial, int nblocks, int p) {
  float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int b = 0;
  for (; b + 8 <= nblocks; b += 8)
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] += partial[(size_t)(b + q) * kGradSlots + p];
  for (int q = 0; b + q < nblocks; ++q) a[q] += partial[(size_t)(b + q) * kGradSlots + p];
  return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

// The same sum with the eight chains on eight lanes (lane q sums blocks q,
// q + 8, ...), combined by xor shuffles in the pairing above, so the result is
// the same bits while each lane waits for one round of loads instead of eight.
// All lanes of the warp call it; every lane of an aligned 8-lane group gets
// the sum (lanes with valid = false add nothing but take part).
__device__ __forceinline__ float sum_partials_lanes(const float *__restrict__ partial, int nblocks, int p, int q,
                                                    bool valid) {
  float a = 0.f;
  if (valid) {
#pragma unroll 8
    for (int b = q; b < nblocks; b += 8) a += partial[(size_t)b * kGradSlots + p];
  }
  a += __shfl_xor_sync(0xffffffffu, a, 1);
  a += __shfl_xor_sync(0xffffffffu, a, 2);
  a += __shfl_xor_sync(0xffffffffu, a, 4);
  return a;
}

// Sum per-block gradients in a fixed order and take one Adam step: eight
// lanes per parameter (and per the loss slot), in small blocks so that the
// summing spreads over many SMs.
constexpr int kAdamThreads = 64;
constexpr int kAdamBlocks = ((kLossSlot + 1) * 8 + kAdamThreads - 1) / kAdamThreads;

// The step size and bias corrections of a scheduled Adam step come from the
// device step counter (advanced by the gradient kernel before it): step st
// (1-based) has lr = lr0 2^(log2_ratio (st - 1 - base)) -- the geometric decay
// from lr0 to lr_final over the steps after `base` -- and corrections
// 1 - b^st.  With on = 0 the kernel's explicit lr, bc1, bc2 are used.
struct AdamSched {
  int on;
  float lr0, log2_ratio;
  long long base;
  float log2_b1, log2_b2;
};

__global__ void __launch_bounds__(kAdamThreads)
    k_mlp_adam(float *__restrict__ params, float *__restrict__ m1, float *__restrict__ m2,
               __nv_bfloat16 *__restrict__ w2c, const float *__restrict__ partial, int nblocks, float lr,
               float b1, float b2, float eps, float bc1, float bc2, float *__restrict__ loss_out,
               float loss_scale, const long long *__restrict__ step_count, AdamSched sch) {
  pdl_launch_dependents();  // the next gradient launch may set up; it waits for these parameters
  pdl_wait();               // the partials of the gradient launch before
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 3, q = threadIdx.x & 7;
  const float gsum = sum_partials_lanes(partial, nblocks, p, q, p <= kLossSlot);
  if (q != 0 || p > kLossSlot) return;
  if (p == kLossSlot) {
    if (loss_out) *loss_out = gsum * loss_scale;
    return;
  }
  if (sch.on) {
    const float st = (float)*step_count;
    lr = sch.lr0 * exp2f(sch.log2_ratio * (st - 1.0f - (float)sch.base));
    bc1 = 1.0f - exp2f(st * sch.log2_b1);
    bc2 = 1.0f - exp2f(st * sch.log2_b2);
  }
  const float m = b1 * m1[p] + (1.f - b1) * gsum;
  const float v = b2 * m2[p] + (1.f - b2) * gsum * gsum;
  m1[p] = m;
  m2[p] = v;
  const float w = params[p] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
  params[p] = w;
  if (p >= kOffW2 && p < kOffW2 + kH * kH) {  // the BF16 canonical copies of W2 and W2^T
    const int nn = (p - kOffW2) / kH, k = (p - kOffW2) % kH;
    const __nv_bfloat16 wb = __float2bfloat16_rn(w);
    w2c[tc_canon_off64(nn, k) / 2] = wb;
    w2c[kH * kH + tc_canon_off64(k, nn) / 2] = wb;
  }
}

// Just the gradient (summed over blocks), for the gradient check.
__global__ void k_mlp_grad_sum(const float *__restrict__ partial, int nblocks, float *__restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kLossSlot) return;
  grad[p] = sum_partials(partial, nblocks, p);
}

// ------------------------------------------------------------------ exact targets
// Sample i: u from word 0 and ln(lambda) ~ U(lo, hi) from word 1 of Philox
// block i (counter (i mod 2^32, i >> 32, 0, tag)); target
// P = (C^{-1}_nu(u; lambda) - lambda - nu) / (2 sqrt(lambda + nu)).
__global__ void k_ncx2_targets(PhiloxKeys keys, uint32_t tag, double nu, float loglam_lo,
                               float loglam_hi, uint64_t n, float *__restrict__ u_out,
                               float *__restrict__ lam_out, float *__restrict__ p_out,
                               int *__restrict__ status) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  int st = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 r = philox(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0u, tag), keys);
    const float u = u01(r.x);
    const float ll = loglam_lo + (loglam_hi - loglam_lo) * u01(r.y);
    const float lam = __expf(ll);
    const double q = ncx2_ppf((double)u, nu, (double)lam, &st);
    const double h = (double)lam + nu;
    u_out[i] = u;
    lam_out[i] = lam;
    p_out[i] = (float)((q - h) / (2.0 * sqrt(h)));
  }
  if (st) atomicOr(status, st);
}

// Exact quantiles for caller arrays (FP64 arithmetic, FP32 in/out for u).
__global__ void k_ncx2_ppf(const float *__restrict__ u, const double *__restrict__ lam, double nu,
                           uint64_t n, double *__restrict__ out, int *__restrict__ status) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  int st = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = ncx2_ppf((double)u[i], nu, lam[i], &st);
  if (st) atomicOr(status, st);
}

}  // namespace aicdf

using namespace aicdf;

// ------------------------------------------------------------------ handle
struct aicdf_surrogate_s {
  uint32_t magic;
  int device;
  double nu;
  float *params = nullptr;   // FP32 master weights [kMlpParams]
  __nv_bfloat16 *w2c = nullptr;  // W2 in BF16, canonical tcgen05 layout: W2 [n][k] | W2^T [k][n]
  float *m1 = nullptr, *m2 = nullptr;
  float *partial = nullptr;  // per-block gradient partials
  int partial_blocks = 0;
  int *status = nullptr;
  float4 *feat = nullptr;    // training samples' (x0, x1, g), aicdf_surrogate_train
  size_t feat_n = 0;
  long long *d_step = nullptr;  // Adam steps taken, on the device (scheduled training reads it)
  long long step = 0;           // the same on the host
};

constexpr uint32_t kSurrogateMagic = 0x53555247u;

static bool sur_ok(const aicdf_surrogate_s *s) { return s && s->magic == kSurrogateMagic; }

static aicdf_status cuda_fail() {
  set_cuda_error((int)cudaGetLastError());
  return AICDF_ERR_CUDA;
}

// FP32 -> BF16, round to nearest even (NaN kept quiet)
static uint16_t host_bf16(float f) {
  uint32_t b;
  std::memcpy(&b, &f, 4);
  if ((b & 0x7F800000u) == 0x7F800000u && (b & 0x7FFFFFu)) return (uint16_t)((b >> 16) | 0x40u);
  return (uint16_t)((b + 0x7FFFu + ((b >> 16) & 1u)) >> 16);
}

// Upload the BF16 canonical copies of W2 from host FP32 parameters.
static aicdf_status upload_w2c(aicdf_surrogate_s *s, const float *p) {
  std::vector<uint16_t> c(2 * kH * kH);
  for (int n = 0; n < kH; ++n)
    for (int k = 0; k < kH; ++k) {
      const uint16_t b = host_bf16(p[kOffW2 + n * kH + k]);
      const int o1 = (n >> 3) * 1024 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;  // (row n, col k)
      const int o2 = (k >> 3) * 1024 + (n >> 3) * 128 + (k & 7) * 16 + (n & 7) * 2;  // (row k, col n)
      c[o1 / 2] = b;
      c[kH * kH + o2 / 2] = b;
    }
  if (cudaMemcpy(s->w2c, c.data(), c.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess)
    return cuda_fail();
  return AICDF_OK;
}

extern "C" aicdf_status aicdf_surrogate_create(double nu, uint64_t seed, aicdf_surrogate *out) {
  if (!out || !(nu > 0.0) || !std::isfinite(nu)) return AICDF_ERR_ARG;
  *out = nullptr;
  aicdf_surrogate_s *s = new (std::nothrow) aicdf_surrogate_s();
  if (!s) return AICDF_ERR_NOMEM;
  s->magic = kSurrogateMagic;
  s->nu = nu;
  cudaGetDevice(&s->device);
  if (cudaMalloc(&s->params, sizeof(float) * kMlpParams) != cudaSuccess ||
      cudaMalloc(&s->m1, sizeof(float) * kMlpParams) != cudaSuccess ||
      cudaMalloc(&s->m2, sizeof(float) * kMlpParams) != cudaSuccess ||
      cudaMalloc(&s->w2c, 2 * (size_t)kW2cBytes) != cudaSuccess ||
      cudaMalloc(&s->status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&s->d_step, sizeof(long long)) != cudaSuccess) {
    aicdf_surrogate_destroy(s);
    return cuda_fail();
  }
  // Glorot-uniform weights, zero biases (host RNG, seeded)
  std::vector<float> p(kMlpParams, 0.f);
  std::mt19937_64 rng(seed);
  auto uni = [&](double lim) {
    return (float)(lim * (2.0 * std::uniform_real_distribution<double>(0.0, 1.0)(rng) - 1.0));
  };
  for (int i = 0; i < 2 * kH; ++i) p[kOffW1 + i] = uni(std::sqrt(6.0 / (2 + kH)) * 2.0);
  for (int i = 0; i < kH * kH; ++i) p[kOffW2 + i] = uni(std::sqrt(6.0 / (2 * kH)));
  for (int i = 0; i < kH; ++i) p[kOffW3 + i] = uni(std::sqrt(6.0 / (kH + 1)));
  for (int i = 0; i < kH; ++i) p[kOffB1 + i] = uni(1.0);
  if (cudaMemcpy(s->params, p.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->m1, 0, sizeof(float) * kMlpParams) != cudaSuccess ||
      cudaMemset(s->m2, 0, sizeof(float) * kMlpParams) != cudaSuccess ||
      cudaMemset(s->status, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(s->d_step, 0, sizeof(long long)) != cudaSuccess || upload_w2c(s, p.data()) != AICDF_OK) {
    aicdf_surrogate_destroy(s);
    return cuda_fail();
  }
  *out = s;
  return AICDF_OK;
}

extern "C" void aicdf_surrogate_destroy(aicdf_surrogate s) {
  if (!sur_ok(s)) return;
  cudaFree(s->params);
  cudaFree(s->w2c);
  cudaFree(s->m1);
  cudaFree(s->m2);
  cudaFree(s->partial);
  cudaFree(s->feat);
  cudaFree(s->status);
  cudaFree(s->d_step);
  s->magic = 0;
  delete s;
}

extern "C" aicdf_status aicdf_surrogate_get_params(aicdf_surrogate s, float *host, int cap) {
  if (!sur_ok(s) || !host || cap < kMlpParams) return AICDF_ERR_ARG;
  if (cudaMemcpy(host, s->params, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_fail();
  return AICDF_OK;
}

extern "C" aicdf_status aicdf_surrogate_set_params(aicdf_surrogate s, const float *host, int n) {
  if (!sur_ok(s) || !host || n < kOffB3 + 1 || n > kMlpParams) return AICDF_ERR_ARG;
  if (cudaMemcpy(s->params, host, sizeof(float) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->m1, 0, sizeof(float) * kMlpParams) != cudaSuccess ||
      cudaMemset(s->m2, 0, sizeof(float) * kMlpParams) != cudaSuccess ||
      cudaMemset(s->d_step, 0, sizeof(long long)) != cudaSuccess)
    return cuda_fail();
  if (upload_w2c(s, host) != AICDF_OK) return AICDF_ERR_CUDA;
  s->step = 0;
  return AICDF_OK;
}

extern "C" int aicdf_surrogate_param_count(void) { return kOffB3 + 1; }

// File format of a saved surrogate: the 8 bytes "AICDFSG1", nu (FP64), the
// parameter count (int32), then the FP32 parameter blob; little-endian, as
// written by the host.  The optimiser state is not saved.
static const char kSurrogateFileMagic[8] = {'A', 'I', 'C', 'D', 'F', 'S', 'G', '1'};

extern "C" aicdf_status aicdf_surrogate_save(aicdf_surrogate s, const char *path) {
  if (!sur_ok(s) || !path) return AICDF_ERR_ARG;
  std::vector<float> p(kMlpParams);
  aicdf_status rc = aicdf_surrogate_get_params(s, p.data(), kMlpParams);
  if (rc != AICDF_OK) return rc;
  FILE *f = std::fopen(path, "wb");
  if (!f) return AICDF_ERR_ARG;
  const int32_t np = kOffB3 + 1;
  const bool ok = std::fwrite(kSurrogateFileMagic, 1, 8, f) == 8 && std::fwrite(&s->nu, sizeof(double), 1, f) == 1 &&
                  std::fwrite(&np, sizeof(np), 1, f) == 1 && std::fwrite(p.data(), sizeof(float), np, f) == (size_t)np;
  return (std::fclose(f) == 0 && ok) ? AICDF_OK : AICDF_ERR_ARG;
}

extern "C" aicdf_status aicdf_surrogate_load(const char *path, aicdf_surrogate *out) {
  if (!path || !out) return AICDF_ERR_ARG;
  *out = nullptr;
  FILE *f = std::fopen(path, "rb");
  if (!f) return AICDF_ERR_ARG;
  char magic[8];
  double nu = 0.0;
  int32_t np = 0;
  std::vector<float> p(kMlpParams, 0.f);
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kSurrogateFileMagic, 8) == 0 &&
            std::fread(&nu, sizeof(double), 1, f) == 1 && std::fread(&np, sizeof(np), 1, f) == 1 &&
            np == kOffB3 + 1 && std::fread(p.data(), sizeof(float), np, f) == (size_t)np;
  std::fclose(f);
  if (!ok || !(nu > 0.0) || !std::isfinite(nu)) return AICDF_ERR_ARG;
  aicdf_surrogate s = nullptr;
  aicdf_status rc = aicdf_surrogate_create(nu, 0, &s);
  if (rc != AICDF_OK) return rc;
  rc = aicdf_surrogate_set_params(s, p.data(), np);
  if (rc != AICDF_OK) {
    aicdf_surrogate_destroy(s);
    return rc;
  }
  *out = s;
  return AICDF_OK;
}

namespace aicdf {
const float *surrogate_params(aicdf_surrogate s) { return sur_ok(s) ? s->params : nullptr; }
double surrogate_nu(aicdf_surrogate s) { return sur_ok(s) ? s->nu : 0.0; }
bool surrogate_ok(aicdf_surrogate s) { return sur_ok(s); }
}  // namespace aicdf

extern "C" aicdf_status aicdf_surrogate_eval(aicdf_surrogate s, const float *u_dev, const float *lam_dev,
                                             size_t n, float *p_out_dev, aicdf_stream_t stream) {
  if (!sur_ok(s)) return AICDF_ERR_ARG;
  if (n == 0) return AICDF_OK;
  if (!u_dev || !lam_dev || !p_out_dev) return AICDF_ERR_ARG;
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_mlp_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBytes);
  if (attr != cudaSuccess) return cuda_fail();
  // persistent: at most 4 CTAs per SM (the padded shared memory sees to it),
  // each taking tiles two at a time
  const uint64_t pairs = ((n + kTcRows - 1) / kTcRows + 1) / 2;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(pairs, (uint64_t)sm_count() * 4));
  k_mlp_eval<<<grid, kEvalThreads, kTcSmemBytes, (cudaStream_t)stream>>>(s->params, s->w2c, u_dev, lam_dev, p_out_dev,
                                                                     n, (float)s->nu);
  return cudaGetLastError() == cudaSuccess ? AICDF_OK : cuda_fail();
}

static aicdf_status ensure_partials(aicdf_surrogate_s *s, int blocks) {
  if (s->partial_blocks >= blocks) return AICDF_OK;
  cudaFree(s->partial);
  s->partial = nullptr;
  s->partial_blocks = 0;
  if (cudaMalloc(&s->partial, sizeof(float) * (size_t)kGradSlots * blocks) != cudaSuccess) return cuda_fail();
  s->partial_blocks = blocks;
  return AICDF_OK;
}

// Partials for `blocks` CTAs and the kernel's shared-memory opt-in: the
// set-up of a gradient launch, done before any launch (and any capture).
static aicdf_status prepare_train_grad(aicdf_surrogate_s *s, int blocks) {
  aicdf_status rc = ensure_partials(s, blocks);
  if (rc != AICDF_OK) return rc;
  static const cudaError_t attr =  // opt in to > 48 KB of dynamic shared memory once
      cudaFuncSetAttribute(k_mlp_train<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
  static const cudaError_t attr_f =
      cudaFuncSetAttribute(k_mlp_train<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
  return attr == cudaSuccess && attr_f == cudaSuccess ? AICDF_OK : cuda_fail();
}

// The gradient kernel over samples [begin, begin + count); step_count (may be
// NULL) is advanced by one for the Adam step that follows.
static aicdf_status launch_train_grad(aicdf_surrogate_s *s, const float *u, const float *lam,
                                      const float *target, uint64_t begin, uint64_t count,
                                      cudaStream_t st, int *blocks_out, long long *step_count) {
  const int blocks = (int)((count + kTcRows - 1) / kTcRows);
  aicdf_status rc = prepare_train_grad(s, blocks);
  if (rc != AICDF_OK) return rc;
  k_mlp_train<false><<<blocks, kTrainThreads, kTrainSmem, st>>>(s->params, s->w2c, u, lam, target, nullptr,
                                                                begin, count, 1.0f / (float)count, s->partial,
                                                                (float)s->nu, step_count);
  *blocks_out = blocks;
  return cudaGetLastError() == cudaSuccess ? AICDF_OK : cuda_fail();
}

extern "C" aicdf_status aicdf_surrogate_grad(aicdf_surrogate s, const float *u_dev, const float *lam_dev,
                                             const float *target_dev, size_t n, float *grad_dev,
                                             aicdf_stream_t stream) {
  if (!sur_ok(s) || !u_dev || !lam_dev || !target_dev || !grad_dev || n == 0 || n > (1u << 24))
    return AICDF_ERR_ARG;
  int blocks = 0;
  aicdf_status rc =
      launch_train_grad(s, u_dev, lam_dev, target_dev, 0, n, (cudaStream_t)stream, &blocks, nullptr);
  if (rc != AICDF_OK) return rc;
  k_mlp_grad_sum<<<(kLossSlot + 64) / 64, 64, 0, (cudaStream_t)stream>>>(s->partial, blocks, grad_dev);
  return cudaGetLastError() == cudaSuccess ? AICDF_OK : cuda_fail();
}

extern "C" aicdf_status aicdf_surrogate_train_step(aicdf_surrogate s, const float *u_dev,
                                                   const float *lam_dev, const float *target_dev,
                                                   size_t n, float lr, float *loss_dev,
                                                   aicdf_stream_t stream) {
  if (!sur_ok(s) || !u_dev || !lam_dev || !target_dev || n == 0 || n > (1u << 24) || !(lr > 0.f))
    return AICDF_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int blocks = 0;
  aicdf_status rc = launch_train_grad(s, u_dev, lam_dev, target_dev, 0, n, st, &blocks, s->d_step);
  if (rc != AICDF_OK) return rc;
  s->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - (float)std::pow((double)b1, (double)s->step);
  const float bc2 = 1.f - (float)std::pow((double)b2, (double)s->step);
  k_mlp_adam<<<kAdamBlocks, kAdamThreads, 0, st>>>(
      s->params, s->m1, s->m2, s->w2c, s->partial, blocks, lr, b1, b2, 1e-8f, bc1, bc2, loss_dev, 1.0f / (float)n,
      s->d_step, AdamSched{0, 0.f, 0.f, 0, 0.f, 0.f});
  return cudaGetLastError() == cudaSuccess ? AICDF_OK : cuda_fail();
}

// Kernel launch with programmatic stream serialization when `pdl` is set (the
// kernel must call pdl_wait() before it reads what its predecessor writes).
template <class... KArgs, class... Args>
static cudaError_t launch_pdl(void (*k)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, bool pdl,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, (KArgs)args...);
}

extern "C" aicdf_status aicdf_surrogate_train(aicdf_surrogate s, const float *u_dev, const float *lam_dev,
                                              const float *target_dev, size_t n, size_t batch,
                                              int epochs, float lr, float lr_final, float *loss_dev,
                                              aicdf_stream_t stream) {
  if (!sur_ok(s) || !u_dev || !lam_dev || !target_dev || n == 0 || batch == 0 || batch > (1u << 24) ||
      epochs <= 0 || !(lr > 0.f) || !(lr_final > 0.f))
    return AICDF_ERR_ARG;
  const size_t steps_per_epoch = n / batch;
  if (steps_per_epoch == 0) return AICDF_ERR_ARG;
  const size_t total = steps_per_epoch * (size_t)epochs;
  const int blocks = (int)((batch + kTcRows - 1) / kTcRows);
  aicdf_status rc = prepare_train_grad(s, blocks);
  if (rc != AICDF_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // The samples' features, once for all epochs (16 bytes a sample, kept by the
  // surrogate); without room for them each gradient launch forms its own.
  const size_t used = steps_per_epoch * batch;
  if (s->feat_n < used) {
    cudaFree(s->feat);
    s->feat = nullptr;
    s->feat_n = 0;
    if (cudaMalloc(&s->feat, sizeof(float4) * used) == cudaSuccess) s->feat_n = used;
    else (void)cudaGetLastError();  // clear the failed allocation; train without the buffer
  }
  const bool feat = s->feat != nullptr;
  if (feat) {
    const int grid = (int)std::min<uint64_t>((used + 255) / 256, (uint64_t)sm_count() * 8);
    k_mlp_features<<<grid, 256, 0, st>>>(u_dev, lam_dev, target_dev, used, (float)s->nu, s->feat);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail();
  }
  // One epoch -- a gradient launch and an Adam launch per batch -- is captured
  // as a CUDA graph and replayed once per epoch: the launches run back to back
  // with no host in between.  The step size and bias corrections of each step
  // follow from the device step counter (AdamSched), so every epoch replays
  // the same graph.
  const AdamSched sch{1, lr, (float)(std::log2((double)lr_final / (double)lr) / (double)std::max<size_t>(total - 1, 1)),
                      s->step, (float)std::log2(0.9), (float)std::log2(0.999)};
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return cuda_fail();
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  rc = AICDF_OK;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    rc = AICDF_ERR_CUDA;
  } else {
    // each launch after the first may start under the tail of the one before
    // (programmatic dependent launch; the kernels wait where they read it)
    cudaError_t e = cudaSuccess;
    for (size_t b = 0; b < steps_per_epoch && e == cudaSuccess; ++b) {
      e = launch_pdl(feat ? k_mlp_train<true> : k_mlp_train<false>, blocks, kTrainThreads, kTrainSmem, cap, b > 0,
                     (const float *)s->params, (const __nv_bfloat16 *)s->w2c, feat ? nullptr : u_dev,
                     feat ? nullptr : lam_dev, feat ? nullptr : target_dev, (const float4 *)s->feat,
                     (uint64_t)(b * batch), (uint64_t)batch, 1.0f / (float)batch, s->partial, (float)s->nu,
                     s->d_step);
      if (e == cudaSuccess)
        e = launch_pdl(k_mlp_adam, kAdamBlocks, kAdamThreads, 0, cap, true, s->params,
                       s->m1, s->m2, s->w2c, (const float *)s->partial, blocks, lr, 0.9f, 0.999f, 1e-8f, 1.f, 1.f,
                       b + 1 == steps_per_epoch ? loss_dev : (float *)nullptr, 1.0f / (float)batch,
                       (const long long *)s->d_step, sch);
    }
    if (cudaStreamEndCapture(cap, &g) != cudaSuccess || e != cudaSuccess || cudaGetLastError() != cudaSuccess)
      rc = AICDF_ERR_CUDA;
  }
  if (rc == AICDF_OK && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) rc = AICDF_ERR_CUDA;
  for (int e = 0; e < epochs && rc == AICDF_OK; ++e)
    if (cudaGraphLaunch(exec, st) != cudaSuccess) rc = AICDF_ERR_CUDA;
  if (rc != AICDF_OK) set_cuda_error((int)cudaGetLastError());
  // the launches are queued on the caller's stream; the graph may go once they are
  if (exec) cudaGraphExecDestroy(exec);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (rc == AICDF_OK) s->step += (long long)total;
  return rc;
}

extern "C" aicdf_status aicdf_ncx2_targets(double nu, float loglam_lo, float loglam_hi, uint64_t seed,
                                           uint32_t tag, size_t n, float *u_dev, float *lam_dev,
                                           float *p_dev, int *status_dev, aicdf_stream_t stream) {
  if (!(nu > 0.0) || !(loglam_hi >= loglam_lo) || !u_dev || !lam_dev || !p_dev || !status_dev)
    return AICDF_ERR_ARG;
  if (n == 0) return AICDF_OK;
  const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)sm_count() * 8);
  k_ncx2_targets<<<grid, 256, 0, (cudaStream_t)stream>>>(make_keys(seed), tag, nu, loglam_lo, loglam_hi,
                                                          n, u_dev, lam_dev, p_dev, status_dev);
  return cudaGetLastError() == cudaSuccess ? AICDF_OK : cuda_fail();
}

extern "C" aicdf_status aicdf_ncx2_ppf(const float *u_dev, const double *lam_dev, double nu, size_t n,
                                       double *out_dev, int *status_dev, aicdf_stream_t stream) {
  if (!(nu > 0.0) || !u_dev || !lam_dev || !out_dev || !status_dev) return AICDF_ERR_ARG;
  if (n == 0) return AICDF_OK;
  const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)sm_count() * 8);
  k_ncx2_ppf<<<grid, 256, 0, (cudaStream_t)stream>>>(u_dev, lam_dev, nu, n, out_dev, status_dev);
  return cudaGetLastError() == cudaSuccess ? AICDF_OK : cuda_fail();
}
