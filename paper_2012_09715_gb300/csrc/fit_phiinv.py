"""Generate phiinv_coefs.h: coefficients of the GPU's FP32 exact inverse
Gaussian CDF.

Formulation (Giles, "Approximating the erfinv function", GPU Computing Gems
Jade, 2011): with x = 2u - 1 and w = -ln(1 - x^2) = -ln(4u(1-u)), the ratio
Phi^{-1}(u) / x is a smooth function g(w) of w alone.  We fit
  central  (w <  W0): g(w) ~ P_c(w - W0/2)        polynomial, degree DC
  tail     (W0 <= w <= W1): g(w) ~ P_t(sqrt(w) - S0)  polynomial, degree DT
by weighted least squares on Chebyshev nodes in the relative error, with the
reference values from mpmath at 40 digits.  The coefficients are our own fit;
the script also reports the maximum relative error after rounding the
coefficients to FP32 and evaluating Horner's rule in FP32.

Run:  python fit_phiinv.py > phiinv_coefs.h   (needs numpy, mpmath)
"""
import math
import sys

import mpmath
import numpy as np

mpmath.mp.dps = 40
W0 = 6.25
W1 = 16.5       # u down to ~1.7e-8; below that the FP64 branch takes over
DC = 10
DT = 10


def g_of_w(w):
    """Phi^{-1}(u)/(2u-1) at w = -ln(4u(1-u)), lower half u < 1/2."""
    w = mpmath.mpf(w)
    if w < mpmath.mpf("1e-30"):
        return mpmath.sqrt(2 * mpmath.pi) / 2
    e = mpmath.exp(-w)
    s = mpmath.sqrt(1 - e)          # |x|
    u = e / (2 * (1 + s))           # (1 - s)/2 without cancellation
    z = -mpmath.sqrt(2) * mpmath.erfinv(1 - 2 * u)
    return z / (-s)


def cheb_nodes(a, b, n):
    k = np.arange(n)
    return 0.5 * (a + b) + 0.5 * (b - a) * np.cos(np.pi * (k + 0.5) / n)


def fit(xs, ys, deg):
    # relative least squares: minimise sum ((p(x) - y)/y)^2
    V = np.vander(xs, deg + 1, increasing=True)
    A = V / ys[:, None]
    c, *_ = np.linalg.lstsq(A, np.ones_like(ys), rcond=None)
    return c


def horner_f32(c, t):
    c32 = c.astype(np.float32)
    t = t.astype(np.float32)
    acc = np.full_like(t, c32[-1])
    for k in range(len(c32) - 2, -1, -1):
        acc = (acc.astype(np.float64) * t.astype(np.float64) + np.float64(c32[k])).astype(np.float32)
    return acc


def main():
    # central
    wc = cheb_nodes(0.0, W0, 400)
    gc = np.array([float(g_of_w(w)) for w in wc])
    cc = fit(wc - W0 / 2, gc, DC)
    # tail
    S0 = 0.5 * (math.sqrt(W0) + math.sqrt(W1))
    sc = cheb_nodes(math.sqrt(W0), math.sqrt(W1), 400)
    gt = np.array([float(g_of_w(s * s)) for s in sc])
    ct = fit(sc - S0, gt, DT)
    # verify on a dense grid after FP32 rounding
    wt = np.linspace(0.0, W0, 3001)
    ref = np.array([float(g_of_w(w)) for w in wt])
    errc = np.max(np.abs(horner_f32(cc, wt - W0 / 2) / ref - 1))
    st = np.linspace(math.sqrt(W0), math.sqrt(W1), 3001)
    ref = np.array([float(g_of_w(s * s)) for s in st])
    errt = np.max(np.abs(horner_f32(ct, st - S0) / ref - 1))
    out = sys.stdout
    out.write("/* Generated by fit_phiinv.py -- do not edit.\n")
    out.write(" * Phi^{-1}(u) = (2u-1) * g(w), w = -ln(4u(1-u)).\n")
    out.write(f" * central: g ~ P_c(w - {W0/2}) for w < {W0}, max rel err (FP32 Horner) {errc:.2e}\n")
    out.write(f" * tail:    g ~ P_t(sqrt(w) - {S0:.9g}) for {W0} <= w <= {W1}, max rel err {errt:.2e}\n */\n")
    out.write("#pragma once\n")
    out.write(f"#define AICDF_PHIINV_W0 {W0:.9g}f\n#define AICDF_PHIINV_W1 {W1:.9g}f\n")
    out.write(f"#define AICDF_PHIINV_WC {W0/2:.9g}f\n#define AICDF_PHIINV_S0 {float(np.float32(S0)):.9g}f\n")
    out.write(f"#define AICDF_PHIINV_DC {DC}\n#define AICDF_PHIINV_DT {DT}\n")
    for name, c in (("aicdf_phiinv_poly_central", cc), ("aicdf_phiinv_poly_tail", ct)):
        # Horner's rule as a chain of FMAs with literal coefficients
        expr = f"{float(np.float32(c[-1])):.9e}f"
        for v in c[-2::-1]:
            expr = f"fmaf({expr}, t, {float(np.float32(v)):.9e}f)"
        out.write(f"__device__ __forceinline__ float {name}(float t) {{\n  return {expr};\n}}\n")
    sys.stderr.write(f"central max rel err {errc:.3e}, tail max rel err {errt:.3e}\n")


if __name__ == "__main__":
    main()
