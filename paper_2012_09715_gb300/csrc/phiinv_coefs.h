/* Generated by fit_phiinv.py -- do not edit.
 * Phi^{-1}(u) = (2u-1) * g(w), w = -ln(4u(1-u)).
 * central: g ~ P_c(w - 3.125) for w < 6.25, max rel err (FP32 Horner) 1.36e-07
 * tail:    g ~ P_t(sqrt(w) - 3.2810096) for 6.25 <= w <= 16.5, max rel err 9.70e-08
 */
#pragma once
#define AICDF_PHIINV_W0 6.25f
#define AICDF_PHIINV_W1 16.5f
#define AICDF_PHIINV_WC 3.125f
#define AICDF_PHIINV_S0 3.28100967f
#define AICDF_PHIINV_DC 10
#define AICDF_PHIINV_DT 10
__device__ __forceinline__ float aicdf_phiinv_poly_central(float t) {
  return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(9.308407378e-10f, t, -6.508231731e-09f), t, -3.488968048e-08f), t, 6.018015029e-07f), t, -1.963471277e-06f), t, -1.963790237e-05f), t, 2.641592582e-04f), t, -1.047509722e-03f), t, -8.532967418e-03f), t, 3.396349549e-01f), t, 2.338620663e+00f);
}
__device__ __forceinline__ float aicdf_phiinv_poly_tail(float t) {
  return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(-5.404909462e-05f, t, 9.954747657e-05f), t, 5.351983782e-05f), t, -5.026651779e-04f), t, 1.241593855e-03f), t, -2.143829595e-03f), t, 3.172026016e-03f), t, -4.890449811e-03f), t, 7.121740375e-03f), t, 1.422107100e+00f), t, 4.405364990e+00f);
}
