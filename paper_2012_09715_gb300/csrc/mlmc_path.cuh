// One coupled MLMC path (Section 4): Euler-Maruyama or Milstein for GBM or
// CIR, driven by exact and/or approximate variates from the same uniforms;
// plus the per-term specification and the FP64 block reduction shared by the
// level kernel and the batched persistent kernel.
#pragma once

#include <cstdint>

#include <cuda_fp16.h>

#include "aicdf_internal.h"
#include "device_common.cuh"

namespace aicdf {

// Everything one estimator term needs besides the approximation table.
struct PathSpec {
  uint32_t tag;                       // Philox counter word 3
  int level, kind, model, scheme, payoff;
  float X0, K, discount;
  float mu, sigma, kappa, theta, dt;  // dt = T / 2^level (fine step)
};

struct LevelArgs {
  PhiloxKeys keys;
  uint64_t n_paths, path_offset;
  PathSpec ps;
  int approx, ntab;
  float tab[1024];  // PWC constants | PWL alpha[0..15], beta[16..31]
};

inline bool kind_needs_exact(int kind) {
  return kind == AICDF_KIND_CORR4 || kind == AICDF_KIND_EXACT2 || kind == AICDF_KIND_PLAIN;
}
inline bool kind_needs_approx(int kind) {
  return kind == AICDF_KIND_CORR4 || kind == AICDF_KIND_APPROX2 || kind == AICDF_KIND_PLAIN_APPROX;
}

// Approximation evaluator used inside path loops.  Path uniforms always come
// from the library's Philox words, so it takes the word x and evaluates at
// u01(x) through the word forms (v and the sign bit straight from x).
template <int AP>
struct ApproxTable;

template <>
struct ApproxTable<AICDF_PWL> {
  PwlRows rows;
  __device__ ApproxTable(const float *tab, int ntab, float *) {
    rows = pwl_lane_rows(tab, tab + 16, ntab);
  }
  __device__ __forceinline__ float operator()(uint32_t x) const { return pwl_eval_word(x, rows); }
};

template <>
struct ApproxTable<AICDF_PWP> {
  const float4 *rows;  // kPwpStagedRows rows in shared memory
  __device__ ApproxTable(const float *tab, int ntab, float *smem) {
    float4 *r = reinterpret_cast<float4 *>(smem);
    pwp_stage_rows(tab, ntab, r);
    rows = r;
  }
  __device__ __forceinline__ float operator()(uint32_t x) const { return pwp_staged_word(x, rows); }
};

template <>
struct ApproxTable<AICDF_PWC> {
  const float *w;  // word-order copy of the table
  PwcWord pw;
  __device__ ApproxTable(const float *tab, int ntab, float *smem) {
    for (int i = threadIdx.x; i < ntab; i += blockDim.x) smem[i] = tab[pwc_word_row(i, ntab)];
    __syncthreads();
    w = smem;
    pw = pwc_word(31u - __clz(ntab));  // ntab = 2^q
  }
  __device__ __forceinline__ float operator()(uint32_t x) const { return w[pwc_slot_from_word(x, pw)]; }
};

// Steps are written as X <- X + increment so that FP32 rounding of the
// constant factors never biases every step the same way: rounding 1 + mu dt
// to FP32 once would shift the drift by up to 2^-24 per step, a bias that
// grows like 2^l.  GBM, with Z the standard normal of one step of size h:
//   EM:       X <- X + X (mu h + sigma sqrt(h) Z)
//   Milstein: X <- X + X (mu h + sigma sqrt(h) Z + sigma^2 h (Z^2 - 1) / 2)
// For the coarse step (h = 2 dt) the increment is sqrt(dt) (Z1 + Z2) = sqrt(dt) S,
// so with S in place of Z the same polynomial holds with sqrt(dt) and 2 dt.
// CIR (truncated):   X <- X + kappa (theta - X) h + sigma sqrt(|X|) dW
//                         [+ sigma^2 (dW^2 - h) / 4  for Milstein]
struct PathConsts {
  // GBM: fine increment factor g0 + g1 Z + g2 Z^2, coarse c0 + c1 S + c2 S^2
  float g0, g1, g2, c0, c1, c2;
  // CIR: fine   Z (sig_sdt sqrt|X| + mq Z) + (nkdt X + dc1)
  //      coarse S (sig_sdt sqrt|X| + mq S) + (nkdt2 X + dc2)
  // with nkdt = -kappa h, dc1 = kappa h theta - mq (coarse: twice each): the
  // drift kappa (theta - X) h and the Milstein term's -mq in one FMA, the noise
  // sigma sqrt|X| dW + mq dW^2 / h in two (mq = 0 for Euler-Maruyama).  The
  // constants' rounding is relative to the drift per step, not to X.
  float nkdt, nkdt2, dc1, dc2, sig_sdt, mq;
  // payoff discount * max(X - pk, pfloor): the call has (K, 0); P = X has
  // (0, NaN), since X - 0 is X and fmaxf returns its other operand for a NaN
  // one (a NaN X stays NaN), so both payoffs are one branch-free form
  float pk, pfloor;
};

// (all products and differences rounded separately, _rn intrinsics: the
// constants must not depend on how a kernel's compilation contracts them)
__device__ __forceinline__ PathConsts make_path_consts(const PathSpec &a) {
  PathConsts p;
  const float dt = a.dt, sdt = sqrtf(dt);
  const bool mil = a.scheme == AICDF_SCHEME_MILSTEIN;
  const float s2 = __fmul_rn(a.sigma, a.sigma);
  const float hs2 = __fmul_rn(__fmul_rn(0.5f, s2), dt);
  const float mdt = __fmul_rn(a.mu, dt);
  p.g0 = __fsub_rn(mdt, mil ? hs2 : 0.f);
  p.g1 = __fmul_rn(a.sigma, sdt);
  p.g2 = mil ? hs2 : 0.f;
  p.c0 = __fsub_rn(__fmul_rn(2.0f, mdt), mil ? __fmul_rn(2.0f, hs2) : 0.f);
  p.c1 = p.g1;
  p.c2 = mil ? hs2 : 0.f;
  const float kdt = __fmul_rn(a.kappa, dt), kth = __fmul_rn(kdt, a.theta);
  p.sig_sdt = p.g1;
  p.mq = mil ? __fmul_rn(__fmul_rn(0.25f, s2), dt) : 0.f;
  p.nkdt = -kdt;
  p.nkdt2 = __fmul_rn(-2.0f, kdt);
  p.dc1 = __fsub_rn(kth, p.mq);
  p.dc2 = __fmul_rn(2.0f, p.dc1);
  const bool call = a.payoff == AICDF_PAYOFF_CALL;
  p.pk = call ? a.K : 0.0f;
  p.pfloor = call ? 0.0f : __int_as_float(0x7fffffff);
  return p;
}

// sqrt|X| of the CIR step with the hardware's approximate square root: its
// error of a few ulps of sqrt|X| enters the step scaled by sig_sdt Z, while
// the IEEE-rounded sqrtf is a multi-instruction sequence paid once per fine
// and coarse step.
__device__ __forceinline__ float cir_sqrt_abs(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(fabsf(x)));
  return r;
}

// MIL: Milstein.  The Euler-Maruyama forms leave out the Z^2 terms, whose
// constants are zero there: fmaf(0, z, c) = c for finite z, so both forms give
// the same bits and EM saves one FMA per fine and per coarse step.
template <int MODEL, bool MIL>
__device__ __forceinline__ float step_fine(float x, float z, const PathConsts &p) {
  if (MODEL == AICDF_MODEL_GBM) return fmaf(x, fmaf(MIL ? fmaf(p.g2, z, p.g1) : p.g1, z, p.g0), x);
  const float r = cir_sqrt_abs(x);
  const float inc = fmaf(z, MIL ? fmaf(p.mq, z, p.sig_sdt * r) : p.sig_sdt * r, fmaf(p.nkdt, x, p.dc1));
  return x + inc;
}

template <int MODEL, bool MIL>
__device__ __forceinline__ float step_coarse(float x, float s, const PathConsts &p) {
  if (MODEL == AICDF_MODEL_GBM) return fmaf(x, fmaf(MIL ? fmaf(p.c2, s, p.c1) : p.c1, s, p.c0), x);
  const float r = cir_sqrt_abs(x);
  const float inc = fmaf(s, MIL ? fmaf(p.mq, s, p.sig_sdt * r) : p.sig_sdt * r, fmaf(p.nkdt2, x, p.dc2));
  return x + inc;
}

// The four power sums of Y over one term's paths (Section 4.1 estimators:
// the sample mean and variance, plus the third and fourth moments that show
// how far the variance estimate can be trusted).
struct __align__(16) Moments {
  double s1, s2, s3, s4;  // sum Y, sum Y^2, sum Y^3, sum Y^4
};

// Per-thread power sums of Y: FP32 over chunks of about 16 paths for Y and
// Y^2, each chunk added to FP64 accumulators (FP64 runs at 1/64 of the FP32
// rate on this GPU: a warp's FP64 add holds its sub-partition's FP64 unit for
// ~64 cycles), in a fixed order per thread.  Y^3 and Y^4, which only serve the
// kurtosis of a term, are FP32 running sums over the thread's k paths (two
// registers, no per-chunk work; relative error at most (k-1) 2^-24 and
// typically sqrt(k) 2^-24: ~4e-6 at the few thousand paths per thread of a
// 10^9-path level launch).  add() is FP32 only; flush() is
// called by the loops below once per chunk, outside the per-path body, so
// that the FP64 adds are never if-converted into predicated instructions
// issued for every path (predicated-off FP64 instructions still occupy the
// FP64 unit).  Lanes past the end of their range add zero (valid = false),
// which keeps every lane's chunking and the control flow warp-uniform.
struct PathSums {
  float f1 = 0.f, f2 = 0.f;  // current chunk
  float f3 = 0.f, f4 = 0.f;  // running sums of Y^3, Y^4
  double d1 = 0.0, d2 = 0.0;
  __device__ __forceinline__ void add(float y, bool valid) {
    y = valid ? y : 0.0f;
    f1 = __fadd_rn(f1, y);
    const float y2 = __fmul_rn(y, y);
    f2 = __fadd_rn(f2, y2);
    f3 = fmaf(y2, y, f3);
    f4 = fmaf(y2, y2, f4);
  }
  __device__ __forceinline__ void flush() {
    d1 += (double)f1;
    d2 += (double)f2;
    f1 = f2 = 0.f;
  }
  // the thread's totals (call after the last flush)
  __device__ __forceinline__ Moments total() const { return Moments{d1, d2, (double)f3, (double)f4}; }
};

constexpr int kChunkPaths = 16;       // paths per thread between FP64 flushes
constexpr int kGroupChunkPaths = 32;  // the same at levels 0 and 1 (one or two steps a path)

// for (b = first; b < end; b += stride) body(b), in chunks of `per_chunk`
// iterations with acc.flush() after each chunk.  first, end and stride are
// warp-uniform, so both loops are.
template <class Body>
__device__ __forceinline__ void chunked_loop(uint64_t first, uint64_t end, uint64_t stride, int per_chunk,
                                             PathSums &acc, Body body) {
  const uint64_t span = stride * (uint64_t)per_chunk;
  for (uint64_t b0 = first; b0 < end; b0 += span) {
    const uint64_t lim = end - b0 < span ? end : b0 + span;
    for (uint64_t b = b0; b < lim; b += stride) body(b);
    acc.flush();
  }
}

// Payoffs and the differences of Y use the _rn intrinsics, which the compiler
// never contracts into FMAs, so that Y of a path is the same bits in every
// kernel that inlines this code (the four-way Y is a small difference of
// nearly equal payoffs, where one contraction changes it visibly).
__device__ __forceinline__ float payoff(const PathSpec &a, const PathConsts &pc, float x) {
  return __fmul_rn(a.discount, fmaxf(__fsub_rn(x, pc.pk), pc.pfloor));
}

// Y of a path from its final fine / coarse states (exact e, approximate a).
// Without a coarse path (level 0) every kind of a given (NE, NA) gives the
// same Y (a zero coarse payoff subtracts exactly), so no test of the kind.
template <bool NE, bool NA, bool COARSE>
__device__ __forceinline__ float path_result(const PathSpec &a, const PathConsts &pc, float xfe, float xce,
                                             float xfa, float xca) {
  const float pfe = NE ? payoff(a, pc, xfe) : 0.f, pfa = NA ? payoff(a, pc, xfa) : 0.f;
  if constexpr (!COARSE) return (NE && NA) ? __fsub_rn(pfe, pfa) : NE ? pfe : pfa;
  const float pce = NE ? payoff(a, pc, xce) : 0.f;
  const float pca = NA ? payoff(a, pc, xca) : 0.f;
  switch (a.kind) {
    case AICDF_KIND_APPROX2: return __fsub_rn(pfa, pca);
    case AICDF_KIND_CORR4: return __fsub_rn(__fsub_rn(pfe, pfa), __fsub_rn(pce, pca));
    case AICDF_KIND_EXACT2: return __fsub_rn(pfe, pce);
    case AICDF_KIND_PLAIN: return pfe;
    default: return pfa;
  }
}

// Philox4x32-10 calls (j, plo, phi, tag) of one path.  The first Philox round
// multiplies the path-constant word phi and the call index j; the second
// multiplies the first's x (a path constant) and z (which depends on j and the
// tag only, the same on every lane of a warp).  So the path-constant halves
// of both rounds are taken once per path here, and a call redoes only the
// j-dependent products (warp-uniform) and the remaining eight rounds.  Same
// words as philox().
struct PhiloxPath {
  uint32_t y1;      // first round: lo(M1 phi)
  uint32_t hx, lx;  // second round: hi / lo (M0 x1), x1 = hi(M1 phi) ^ plo ^ k0[0]
};
__device__ __forceinline__ PhiloxPath philox_path(uint32_t plo, uint32_t phi, const PhiloxKeys &k) {
  const uint64_t p1 = (uint64_t)PHILOX_M1 * phi;
  const uint32_t x1 = (uint32_t)(p1 >> 32) ^ plo ^ k.k0[0];
  const uint64_t q0 = (uint64_t)PHILOX_M0 * x1;
  return PhiloxPath{(uint32_t)p1, (uint32_t)(q0 >> 32), (uint32_t)q0};
}
__device__ __forceinline__ uint4 philox_path_call(uint32_t j, uint32_t tag, const PhiloxPath &pp,
                                                  const PhiloxKeys &k) {
  const uint64_t p0 = (uint64_t)PHILOX_M0 * j;
  const uint32_t z1 = (uint32_t)(p0 >> 32) ^ tag ^ k.k1[0], w1 = (uint32_t)p0;
  const uint64_t q1 = (uint64_t)PHILOX_M1 * z1;
  uint4 c = make_uint4((uint32_t)(q1 >> 32) ^ pp.y1 ^ k.k0[1], (uint32_t)q1, pp.hx ^ w1 ^ k.k1[1], pp.lx);
#pragma unroll
  for (int r = 2; r < 10; ++r) c = philox_round(c, k.k0[r], k.k1[r]);
  return c;
}

// Y of one path at level >= 2 (path p owns the Philox calls (s/4, p, tag)).
// All 32 lanes of a warp must call it together (the PWL approximation
// shuffles across the warp).  V16: the approximate variate is rounded to FP16
// before use (FP16 approximate variates); MIL: Milstein steps.
template <bool NE, bool NA, int AP, int MODEL, bool V16, bool MIL>
__device__ __forceinline__ float path_y(const PathSpec &a, const PathConsts &pc,
                                        const ApproxTable<AP> &ap, const PhiloxKeys &keys,
                                        uint64_t p) {
  const int nfine = 1 << a.level;
  float xfe = a.X0, xce = a.X0, xfa = a.X0, xca = a.X0;
  float se = 0.f, sa = 0.f;  // pair sums of fine variates (set at even steps)
  const PhiloxPath pp = philox_path((uint32_t)p, (uint32_t)(p >> 32), keys);
  for (int s4 = 0; s4 < nfine; s4 += 4) {
    const uint4 r = philox_path_call((uint32_t)(s4 >> 2), a.tag, pp, keys);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (NE) {
        const float ze = phiinv_f32_word(w[t]);
        xfe = step_fine<MODEL, MIL>(xfe, ze, pc);
        se = (t & 1) ? se + ze : ze;
      }
      if (NA) {
        float za = ap(w[t]);
        if (V16) za = __half2float(__float2half_rn(za));
        xfa = step_fine<MODEL, MIL>(xfa, za, pc);
        sa = (t & 1) ? sa + za : za;
      }
      if (t & 1) {
        if (NE) xce = step_coarse<MODEL, MIL>(xce, se, pc);
        if (NA) xca = step_coarse<MODEL, MIL>(xca, sa, pc);
      }
    }
  }
  return path_result<NE, NA, true>(a, pc, xfe, xce, xfa, xca);
}

// Levels 0 and 1 have 1 or 2 fine steps per path, so one Philox call serves
// G = 4 >> LEVEL paths: group q (paths q G .. q G + G - 1) uses the call
// (0, q, tag), path q G + g taking words g 2^LEVEL .. g 2^LEVEL + 2^LEVEL - 1.
// y[g] = Y of path q G + g.  All 32 lanes must call it together.
template <bool NE, bool NA, int AP, int MODEL, bool V16, bool MIL, int LEVEL>
__device__ __forceinline__ void group_y(const PathSpec &a, const PathConsts &pc, const ApproxTable<AP> &ap,
                                        const PhiloxKeys &keys, uint64_t q, float (&y)[4]) {
  constexpr int NF = 1 << LEVEL, G = 4 >> LEVEL;
  const uint4 r = philox(make_uint4(0u, (uint32_t)q, (uint32_t)(q >> 32), a.tag), keys);
  const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int g = 0; g < G; ++g) {
    float xfe = a.X0, xce = a.X0, xfa = a.X0, xca = a.X0;
    float se = 0.f, sa = 0.f;
#pragma unroll
    for (int s = 0; s < NF; ++s) {
      const uint32_t x = w[g * NF + s];
      if (NE) {
        const float ze = phiinv_f32_word(x);
        xfe = step_fine<MODEL, MIL>(xfe, ze, pc);
        se = s ? se + ze : ze;
      }
      if (NA) {
        float za = ap(x);
        if (V16) za = __half2float(__float2half_rn(za));
        xfa = step_fine<MODEL, MIL>(xfa, za, pc);
        sa = s ? sa + za : za;
      }
    }
    if (LEVEL == 1) {
      if (NE) xce = step_coarse<MODEL, MIL>(xce, se, pc);
      if (NA) xca = step_coarse<MODEL, MIL>(xca, sa, pc);
    }
    y[g] = path_result<NE, NA, LEVEL == 1>(a, pc, xfe, xce, xfa, xca);
  }
}

// Sums over the paths [p0, p0 + n) of a term at level 0 or 1 by groups of
// G = 4 >> level: group-stride loop over the groups that meet the range,
// starting at group index `first` with stride `stride` (warp-aligned), into
// acc.  GROUP(q, y) fills y.  LV >= 0 fixes the level at compile time
// (the level kernel); LV = -1 takes `level` at run time (the batched kernel).
template <int LV = -1, class GroupFn>
__device__ __forceinline__ void sum_groups(uint64_t p0, uint64_t n, int level, uint64_t first, uint64_t stride,
                                           GroupFn group, PathSums &acc) {
  const int lv = LV >= 0 ? LV : level;
  const int sh = 2 - lv, G = 4 >> lv;
  const bool four = lv == 0;  // G = 4, else G = 2
  const uint64_t q0 = p0 >> sh, ng = ((p0 + n - 1) >> sh) - q0 + 1;
  // Groups wholly inside the range: all but a first group that starts before
  // p0 and a last one that runs past p0 + n.  The warp's groups base ..
  // base + 31 (base a multiple of 32) are all inside iff base + 32 <= qb and
  // not (base = 0 with a partial first group).
  const bool head = (p0 & (uint64_t)(G - 1)) != 0;
  const uint64_t qb = ng - (((p0 + n) & (uint64_t)(G - 1)) ? 1 : 0);
  const int lane = threadIdx.x & 31;
  chunked_loop(first, ng, stride, kGroupChunkPaths / G, acc, [&](uint64_t base) {
    const uint64_t qi = base + lane, q = q0 + qi;
    float y[4];
    group(q, y);
    if (base + 32 <= qb && (base != 0 || !head)) {  // warp-uniform
#pragma unroll
      for (int g = 0; g < 4; ++g)
        if (g < 2 || four) acc.add(y[g], true);
    } else {
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const uint64_t p = (q << sh) + (uint64_t)g;
        if (g < 2 || four) acc.add(y[g], qi < ng && p >= p0 && p < p0 + n);
      }
    }
  });
}

// Sums of Y over the paths [p0, p0 + n) of one term into acc: levels 0 and 1
// by groups of paths sharing a Philox call, finer levels one path per lane;
// `first` (warp-aligned) and `stride` lay the paths over the launch.  All 32
// lanes of a warp must call it together.
template <bool NE, bool NA, int AP, int MODEL, bool V16, bool MIL>
__device__ __forceinline__ void term_sums(const PathSpec &a, const PathConsts &pc, const ApproxTable<AP> &ap,
                                          const PhiloxKeys &keys, uint64_t p0, uint64_t n, uint64_t first,
                                          uint64_t stride, PathSums &acc) {
  if (a.level == 0) {  // warp-uniform
    sum_groups<0>(p0, n, 0, first, stride,
                  [&](uint64_t q, float (&y)[4]) { group_y<NE, NA, AP, MODEL, V16, MIL, 0>(a, pc, ap, keys, q, y); },
                  acc);
  } else if (a.level == 1) {
    sum_groups<1>(p0, n, 1, first, stride,
                  [&](uint64_t q, float (&y)[4]) { group_y<NE, NA, AP, MODEL, V16, MIL, 1>(a, pc, ap, keys, q, y); },
                  acc);
  } else {
    const int lane = threadIdx.x & 31;
    chunked_loop(first, n, stride, kChunkPaths, acc, [&](uint64_t base) {
      const uint64_t i = base + lane;
      acc.add(path_y<NE, NA, AP, MODEL, V16, MIL>(a, pc, ap, keys, p0 + i), i < n);
    });
  }
}

// term_sums with the scheme taken at run time (a uniform branch outside the
// path loops).
template <bool NE, bool NA, int AP, int MODEL, bool V16>
__device__ __forceinline__ void term_sums_scheme(const PathSpec &a, const PathConsts &pc, const ApproxTable<AP> &ap,
                                                 const PhiloxKeys &keys, uint64_t p0, uint64_t n, uint64_t first,
                                                 uint64_t stride, PathSums &acc) {
  if (a.scheme == AICDF_SCHEME_MILSTEIN)
    term_sums<NE, NA, AP, MODEL, V16, true>(a, pc, ap, keys, p0, n, first, stride, acc);
  else
    term_sums<NE, NA, AP, MODEL, V16, false>(a, pc, ap, keys, p0, n, first, stride, acc);
}

// Y of one path (level >= 2) or of one group of paths (levels 0, 1), with the
// kind, model and scheme taken at run time, for kernels that mix terms: the
// branches are uniform across the block, and the path loops stay one loop.
template <bool NE, bool NA, int AP, int MODEL, bool V16>
__device__ __forceinline__ float path_y_scheme(const PathSpec &a, const PathConsts &pc, const ApproxTable<AP> &ap,
                                               const PhiloxKeys &keys, uint64_t p) {
  return a.scheme == AICDF_SCHEME_MILSTEIN ? path_y<NE, NA, AP, MODEL, V16, true>(a, pc, ap, keys, p)
                                           : path_y<NE, NA, AP, MODEL, V16, false>(a, pc, ap, keys, p);
}

template <int AP, bool V16>
__device__ __forceinline__ float path_y_any(const PathSpec &a, const PathConsts &pc, const ApproxTable<AP> &ap,
                                            const PhiloxKeys &keys, uint64_t p) {
  const bool gbm = a.model == AICDF_MODEL_GBM;
  switch (a.kind) {
    case AICDF_KIND_CORR4:
      return gbm ? path_y_scheme<true, true, AP, AICDF_MODEL_GBM, V16>(a, pc, ap, keys, p)
                 : path_y_scheme<true, true, AP, AICDF_MODEL_CIR, V16>(a, pc, ap, keys, p);
    case AICDF_KIND_EXACT2:
    case AICDF_KIND_PLAIN:
      return gbm ? path_y_scheme<true, false, AP, AICDF_MODEL_GBM, V16>(a, pc, ap, keys, p)
                 : path_y_scheme<true, false, AP, AICDF_MODEL_CIR, V16>(a, pc, ap, keys, p);
    default:
      return gbm ? path_y_scheme<false, true, AP, AICDF_MODEL_GBM, V16>(a, pc, ap, keys, p)
                 : path_y_scheme<false, true, AP, AICDF_MODEL_CIR, V16>(a, pc, ap, keys, p);
  }
}

// LEVEL >= 0 fixes the level at compile time; -1 takes it from a.level.
template <bool NE, bool NA, int AP, int MODEL, bool V16, int LEVEL = -1>
__device__ __forceinline__ void group_y_scheme(const PathSpec &a, const PathConsts &pc, const ApproxTable<AP> &ap,
                                               const PhiloxKeys &keys, uint64_t q, float (&y)[4]) {
  const bool mil = a.scheme == AICDF_SCHEME_MILSTEIN;
  if (LEVEL == 0 || (LEVEL < 0 && a.level == 0)) {
    if (mil) group_y<NE, NA, AP, MODEL, V16, true, 0>(a, pc, ap, keys, q, y);
    else group_y<NE, NA, AP, MODEL, V16, false, 0>(a, pc, ap, keys, q, y);
  } else {
    if (mil) group_y<NE, NA, AP, MODEL, V16, true, 1>(a, pc, ap, keys, q, y);
    else group_y<NE, NA, AP, MODEL, V16, false, 1>(a, pc, ap, keys, q, y);
  }
}

// group_y_any with the kind's (NE, NA), and optionally the level, fixed by
// the caller (the model and scheme still taken at run time).
template <bool NE, bool NA, int AP, bool V16, int LEVEL = -1>
__device__ __forceinline__ void group_y_kind(const PathSpec &a, const PathConsts &pc, const ApproxTable<AP> &ap,
                                             const PhiloxKeys &keys, uint64_t q, float (&y)[4]) {
  if (a.model == AICDF_MODEL_GBM) group_y_scheme<NE, NA, AP, AICDF_MODEL_GBM, V16, LEVEL>(a, pc, ap, keys, q, y);
  else group_y_scheme<NE, NA, AP, AICDF_MODEL_CIR, V16, LEVEL>(a, pc, ap, keys, q, y);
}

template <int AP, bool V16>
__device__ __forceinline__ void group_y_any(const PathSpec &a, const PathConsts &pc, const ApproxTable<AP> &ap,
                                            const PhiloxKeys &keys, uint64_t q, float (&y)[4]) {
  const bool gbm = a.model == AICDF_MODEL_GBM;
  switch (a.kind) {
    case AICDF_KIND_CORR4:
      if (gbm) group_y_scheme<true, true, AP, AICDF_MODEL_GBM, V16>(a, pc, ap, keys, q, y);
      else group_y_scheme<true, true, AP, AICDF_MODEL_CIR, V16>(a, pc, ap, keys, q, y);
      break;
    case AICDF_KIND_EXACT2:
    case AICDF_KIND_PLAIN:
      if (gbm) group_y_scheme<true, false, AP, AICDF_MODEL_GBM, V16>(a, pc, ap, keys, q, y);
      else group_y_scheme<true, false, AP, AICDF_MODEL_CIR, V16>(a, pc, ap, keys, q, y);
      break;
    default:
      if (gbm) group_y_scheme<false, true, AP, AICDF_MODEL_GBM, V16>(a, pc, ap, keys, q, y);
      else group_y_scheme<false, true, AP, AICDF_MODEL_CIR, V16>(a, pc, ap, keys, q, y);
  }
}

// FP64 block reduction of the four sums; result valid in thread 0.  Ends with
// a barrier so that s_red may be reused right away.  A warp's FP64 add holds
// its sub-partition's FP64 unit for ~64 cycles whatever the number of active
// lanes, so the warp stage keeps every lane's add useful: the first exchange
// (lanes L, L^16) leaves the lower half with (sum Y, sum Y^2) and the upper
// half with (sum Y^3, sum Y^4) of the two lanes, the second (L, L^8) one sum
// per group of 8 lanes (group k: sum Y^(k+1)) of four lanes, and three xor
// rounds within each group finish it: 6 FP64 adds per warp instead of 20 for
// four separate shuffle trees.  Warp 0 then adds the warps' sums the same way
// (lane 8k + w holds sum k of warp w).  The order of every add is fixed by
// lane and warp indices, so the result is deterministic.
template <int NW>
__device__ __forceinline__ Moments block_reduce_moments(Moments m, Moments (&s_red)[NW]) {
  static_assert(NW <= 8, "at most 8 warps");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool hi = (lane & 16) != 0, mid = (lane & 8) != 0;
  // lanes L, L^16: keep (s1, s2) below 16, (s3, s4) above
  const double r1 = __shfl_xor_sync(FULL_MASK, hi ? m.s1 : m.s3, 16);
  const double r2 = __shfl_xor_sync(FULL_MASK, hi ? m.s2 : m.s4, 16);
  const double a = (hi ? m.s3 : m.s1) + r1, b = (hi ? m.s4 : m.s2) + r2;
  // lanes L, L^8: keep a below 8 (within the half), b above
  double c = (mid ? b : a) + __shfl_xor_sync(FULL_MASK, mid ? a : b, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) c += __shfl_xor_sync(FULL_MASK, c, o);
  double *red = reinterpret_cast<double *>(s_red);  // [warp][4]
  if ((lane & 7) == 0) red[4 * warp + (lane >> 3)] = c;
  __syncthreads();
  Moments t{0.0, 0.0, 0.0, 0.0};
  if (warp == 0) {
    const int nw = (int)(blockDim.x >> 5), w = lane & 7;
    double v = w < nw ? red[4 * w + (lane >> 3)] : 0.0;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    t.s1 = v;
    t.s2 = __shfl_sync(FULL_MASK, v, 8);
    t.s3 = __shfl_sync(FULL_MASK, v, 16);
    t.s4 = __shfl_sync(FULL_MASK, v, 24);
  }
  __syncthreads();
  return t;
}

// Validate SDE parameters and fill a PathSpec (host).
aicdf_status make_path_spec(const aicdf_sde_params *prm, int level, int kind, uint32_t tag,
                            PathSpec *ps);
// Copy an approximation table into the kernel-parameter layout (host).
aicdf_status pack_table(aicdf_table approx, float *tab, int *ntab);
// Validate the arguments of one level call and fill its kernel arguments (host).
aicdf_status prepare_level_args(const aicdf_sde_params *prm, aicdf_table approx, int level,
                                int kind, uint64_t n_paths, uint64_t path_offset, uint64_t seed,
                                uint32_t tag, LevelArgs *a);
// Thread blocks launch_level will use for these arguments (= partial-sum slots).
int level_launch_grid(const LevelArgs &a);
// Launch the level kernel (one Moments partial per block into ws) and the
// fixed-order reduction into sums_dev (host).
aicdf_status launch_level(const LevelArgs &a, double *sums_dev, void *ws, cudaStream_t st);
// Launch the one-block fixed-order sum of per-block partials into
// sums[0..4] = (sum Y, sum Y^2, sum Y^3, sum Y^4, count) (host).
void launch_reduce_partials(const Moments *partials, int nparts, double count, double *sums,
                            cudaStream_t st);

}  // namespace aicdf
