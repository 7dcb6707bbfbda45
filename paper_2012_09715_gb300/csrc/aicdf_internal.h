// Host-side internals of libaicdf (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/aicdf.h"

struct aicdf_table_s {
  uint32_t magic;
  int method;                 // AICDF_PWC, AICDF_PWL or AICDF_PWP
  int n;                      // PWC: number of intervals; PWL, PWP: K
  int construction;           // PWC constant construction; PWP: degree
  std::vector<double> c0, c1; // FP64 coefficients (PWC: constants; PWL: alpha, beta;
                              // PWP: [row][power] in each row's local variable s)
  std::vector<float> f0, f1;  // the same rounded to FP32 (PWC, PWL: what the kernels use)
  std::vector<float> fv;      // PWP: each row of f0 re-expanded in v (what the kernels use)
};

constexpr uint32_t AICDF_TABLE_MAGIC = 0x41494344u;  // "AICD"

namespace aicdf {
// Values per estimator term in every sums_dev array: sum Y, Y^2, Y^3, Y^4, n.
constexpr int kSumsPerTerm = AICDF_SUMS_PER_TERM;
// Set by the launch wrappers; read by aicdf_last_cuda_error().
void set_cuda_error(int e);
bool table_ok(const aicdf_table_s *t);
// SM count of the current device (cached per device).
int sm_count();
// Resident blocks per SM of `kernel` at `threads` per block (occupancy API,
// cached per kernel and device; at least 1).
int resident_blocks(const void *kernel, int threads);
// Host FP64 inverse Gaussian CDF used for the table build.
double host_phiinv(double p);
// One-off batched launch of MLMC terms (no graph); see mlmc.cu.  Returns
// AICDF_ERR_NOMEM when the launch plan does not fit the workspace.
aicdf_status batch_run_once(const aicdf_sde_params *sets, int n_sets, const aicdf_batch_term *terms,
                            int n_terms, aicdf_table approx, uint64_t seed, double *sums_dev, void *ws,
                            size_t ws_bytes, cudaStream_t st);
}  // namespace aicdf
