// One coupled MLMC path (Section 4): Euler-Maruyama or Milstein for GBM or
// CIR, driven by exact and/or approximate variates from the same uniforms;
// plus the argument block and FP64 block reduction used by the level and
// batched kernels.
#pragma once

#include <cstdint>

#include "aicdf_internal.h"
#include "device_common.cuh"

namespace aicdf {

struct LevelArgs {
  PhiloxKeys keys;
  uint64_t n_paths, path_offset;
  uint32_t tag;
  int level, kind, model, scheme, payoff, approx, ntab;
  float nf;
  float X0, K, discount;
  // per-step coefficients (fine step dt, coarse step 2 dt), see make_path_consts
  float mu, sigma, kappa, theta, dt;
  float tab[1024];  // PWC constants | PWL alpha[0..15], beta[16..31]
};

inline bool kind_needs_exact(int kind) {
  return kind == AICDF_KIND_CORR4 || kind == AICDF_KIND_EXACT2 || kind == AICDF_KIND_PLAIN;
}
inline bool kind_needs_approx(int kind) {
  return kind == AICDF_KIND_CORR4 || kind == AICDF_KIND_APPROX2 || kind == AICDF_KIND_PLAIN_APPROX;
}

// Approximation evaluator used inside path loops.
template <int AP>
struct ApproxTable;

template <>
struct ApproxTable<AICDF_PWL> {
  PwlLane c;
  unsigned kmax;
  __device__ ApproxTable(const float *tab, int ntab, float *) {
    c = pwl_lane_coefs(tab, tab + 16);
    kmax = (unsigned)ntab;
  }
  __device__ __forceinline__ float operator()(float u) const { return pwl_eval(u, c, kmax); }
};

template <>
struct ApproxTable<AICDF_PWC> {
  const float *s;
  float nf;
  int nmax;
  __device__ ApproxTable(const float *tab, int ntab, float *smem) {
    for (int i = threadIdx.x; i < ntab; i += blockDim.x) smem[i] = tab[i];
    __syncthreads();
    s = smem;
    nf = (float)ntab;
    nmax = ntab - 1;
  }
  __device__ __forceinline__ float operator()(float u) const { return pwc_eval(u, s, nf, nmax); }
};

// Step multipliers.  GBM, with Z the standard normal of one step of size h:
//   EM:       X <- X (1 + mu h + sigma sqrt(h) Z)
//   Milstein: X <- X (1 + mu h + sigma sqrt(h) Z + sigma^2 h (Z^2 - 1) / 2)
// For the coarse step (h = 2 dt) the increment is sqrt(dt) (Z1 + Z2) = sqrt(dt) S,
// so with S in place of Z the same polynomial holds with sqrt(dt) and 2 dt.
// CIR (truncated):   X <- X + kappa (theta - X) h + sigma sqrt(|X|) dW
//                         [+ sigma^2 (dW^2 - h) / 4  for Milstein]
struct PathConsts {
  // GBM: fine multiplier g0 + g1 Z + g2 Z^2, coarse c0 + c1 S + c2 S^2
  float g0, g1, g2, c0, c1, c2;
  // CIR: fine  X (1 - kappa dt) + kappa theta dt + sig_sdt sqrt|X| Z + m (Z^2 - 1)
  //      coarse X (1 - 2 kappa dt) + 2 kappa theta dt + sig_sdt sqrt|X| S + m (S^2 - 2)
  float a1f, a0f, a1c, a0c, sig_sdt, mq;
};

__device__ __forceinline__ PathConsts make_path_consts(const LevelArgs &a) {
  PathConsts p;
  const float dt = a.dt, sdt = sqrtf(dt);
  const bool mil = a.scheme == AICDF_SCHEME_MILSTEIN;
  const float hs2 = 0.5f * a.sigma * a.sigma * dt;
  p.g0 = 1.0f + a.mu * dt - (mil ? hs2 : 0.f);
  p.g1 = a.sigma * sdt;
  p.g2 = mil ? hs2 : 0.f;
  p.c0 = 1.0f + 2.0f * a.mu * dt - (mil ? 2.0f * hs2 : 0.f);
  p.c1 = a.sigma * sdt;
  p.c2 = mil ? hs2 : 0.f;
  p.a1f = 1.0f - a.kappa * dt;
  p.a0f = a.kappa * a.theta * dt;
  p.a1c = 1.0f - 2.0f * a.kappa * dt;
  p.a0c = 2.0f * a.kappa * a.theta * dt;
  p.sig_sdt = a.sigma * sdt;
  p.mq = mil ? 0.25f * a.sigma * a.sigma * dt : 0.f;
  return p;
}

template <int MODEL>
__device__ __forceinline__ float step_fine(float x, float z, const PathConsts &p) {
  if (MODEL == AICDF_MODEL_GBM) return x * fmaf(fmaf(p.g2, z, p.g1), z, p.g0);
  const float r = sqrtf(fabsf(x));
  return fmaf(p.a1f, x, p.a0f) + fmaf(p.sig_sdt * r, z, p.mq * fmaf(z, z, -1.0f));
}

template <int MODEL>
__device__ __forceinline__ float step_coarse(float x, float s, const PathConsts &p) {
  if (MODEL == AICDF_MODEL_GBM) return x * fmaf(fmaf(p.c2, s, p.c1), s, p.c0);
  const float r = sqrtf(fabsf(x));
  return fmaf(p.a1c, x, p.a0c) + fmaf(p.sig_sdt * r, s, p.mq * fmaf(s, s, -2.0f));
}

__device__ __forceinline__ float payoff(const LevelArgs &a, float x) {
  return a.payoff == AICDF_PAYOFF_CALL ? a.discount * fmaxf(x - a.K, 0.0f) : a.discount * x;
}

// Y of one path.  All 32 lanes of a warp must call it together (the PWL
// approximation shuffles across the warp).
template <bool NE, bool NA, int AP, int MODEL, int SCHEME>
__device__ __forceinline__ float path_y(const LevelArgs &a, const PathConsts &pc,
                                        const ApproxTable<AP> &ap, uint64_t p) {
  const int nfine = 1 << a.level;
  const bool coarse = a.level > 0;
  float xfe = a.X0, xce = a.X0, xfa = a.X0, xca = a.X0;
  float se = 0.f, sa = 0.f;  // pair sums of fine variates
  const uint32_t plo = (uint32_t)p, phi = (uint32_t)(p >> 32);
  for (int s4 = 0; s4 < nfine; s4 += 4) {
    const uint4 r = philox(make_uint4((uint32_t)(s4 >> 2), plo, phi, a.tag), a.keys);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t < nfine) {  // only levels 0 and 1 use part of a Philox block
        const float u = u01(w[t]);
        if (NE) {
          const float ze = phiinv_f32(u);
          xfe = step_fine<MODEL>(xfe, ze, pc);
          se += ze;
        }
        if (NA) {
          const float za = ap(u);
          xfa = step_fine<MODEL>(xfa, za, pc);
          sa += za;
        }
        if ((t & 1) && coarse) {
          if (NE) xce = step_coarse<MODEL>(xce, se, pc);
          if (NA) xca = step_coarse<MODEL>(xca, sa, pc);
          se = 0.f;
          sa = 0.f;
        }
      }
    }
  }
  const float pfe = NE ? payoff(a, xfe) : 0.f, pfa = NA ? payoff(a, xfa) : 0.f;
  const float pce = (NE && coarse) ? payoff(a, xce) : 0.f;
  const float pca = (NA && coarse) ? payoff(a, xca) : 0.f;
  switch (a.kind) {
    case AICDF_KIND_APPROX2: return pfa - pca;
    case AICDF_KIND_CORR4: return (pfe - pfa) - (pce - pca);
    case AICDF_KIND_EXACT2: return pfe - pce;
    case AICDF_KIND_PLAIN: return pfe;
    default: return pfa;
  }
}

// FP64 block reduction of two values; result valid in thread 0.
template <int NW>
__device__ __forceinline__ double2 block_reduce2(double d1, double d2, double2 (&s_red)[NW]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d1 += __shfl_down_sync(FULL_MASK, d1, o);
    d2 += __shfl_down_sync(FULL_MASK, d2, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s_red[warp] = make_double2(d1, d2);
  __syncthreads();
  double2 t = make_double2(0.0, 0.0);
  if (threadIdx.x == 0) {
    for (int w = 0; w < NW; ++w) {
      t.x += s_red[w].x;
      t.y += s_red[w].y;
    }
  }
  return t;
}

// Validate parameters and fill the argument block (host).
aicdf_status prepare_level_args(const aicdf_sde_params *params, aicdf_table approx, int level,
                                int kind, uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                                uint32_t tag, LevelArgs *a);

}  // namespace aicdf
