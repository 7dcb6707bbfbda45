"""CPU FP64 oracle for the approximate inverse-CDF method (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``liboracle.so`` (plain C,
``aicdf_oracle.c``) with ctypes and numpy; it shares no code with the GPU
library ``paper_2012_09715_gb300``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aicdf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# model / scheme / payoff / kind codes, mirroring aicdf_oracle.h
KIND_APPROX2, KIND_CORR4, KIND_EXACT2, KIND_PLAIN, KIND_PLAIN_APPROX = 0, 1, 2, 3, 4
MODEL_GBM, MODEL_CIR = 0, 1
SCHEME_EM, SCHEME_MILSTEIN = 0, 1
PAYOFF_X, PAYOFF_CALL = 0, 1
APPROX_PWL, APPROX_PWC, APPROX_PWP = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (strict IEEE: no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "aicdf_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class SdeParams(C.Structure):
    _fields_ = [("model", C.c_int), ("scheme", C.c_int), ("payoff", C.c_int), ("approx", C.c_int),
                ("X0", C.c_double), ("T", C.c_double), ("K", C.c_double),
                ("mu", C.c_double), ("sigma", C.c_double),
                ("kappa", C.c_double), ("theta", C.c_double), ("discount", C.c_double)]


def set_threads(n: int) -> None:
    """Thread count of the oracle's OpenMP loops (samplers, uniforms, MLMC
    paths): one libgomp runtime serves the process, so this sets it for
    every later oracle call."""
    lib()
    C.CDLL("libgomp.so.1").omp_set_num_threads(max(1, int(n)))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            d, i, i64, u32, u64 = C.c_double, C.c_int, C.c_int64, C.c_uint32, C.c_uint64
            P = C.c_void_p
            sig = {
                "or_philox4": (None, [i, i, P, P, P]),
                "or_u01": (d, [u32]),
                "or_uniforms": (None, [u64, u64, i64, P]),
                "or_phi": (d, [d]), "or_Phi": (d, [d]), "or_phiinv": (d, [d]),
                "or_phiinv_n": (None, [P, i64, P]),
                "or_pwc_table": (i, [i, i, P]),
                "or_pwc_l2err2": (d, [i, P]),
                "or_pwl_table": (i, [i, d, P, P]),
                "or_pwl_l2err2": (d, [i, d, P, P]),
                "or_pwl_index": (i, [d, i, d]),
                "or_sample_pwc": (None, [P, i, P, i64, P, P]),
                "or_sample_pwl": (None, [P, P, i, P, i64, P, P]),
                "or_mlmc_level": (None, [P, P, P, i, i, i, u64, u64, u64, u32, P]),
                "or_mlmc_paths": (None, [P, P, P, i, i, i, u64, u64, u64, u32, P]),
                "or_mlmc_alloc": (d, [i, P, P, d, P]),
                "or_gammp": (d, [d, d]),
                "or_ncx2_cdf": (d, [d, d, d]), "or_ncx2_pdf": (d, [d, d, d]),
                "or_ncx2_ppf": (d, [d, d, d]), "or_ncx2_P": (d, [d, d, d]),
                "or_ncx2_sf": (d, [d, d, d]), "or_ncx2_isf": (d, [d, d, d]),
                "or_mlp_forward": (None, [i, P, P, P, P, P, P, P, i64, P]),
                "or_mlp_grad": (d, [i, P, P, P, P, P, P, P, P, i64, P, P, P, P, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- uniforms
def philox4(ctr, key, wbits=32, rounds=10):
    c = np.ascontiguousarray(np.array(ctr, dtype=np.uint64))
    k = np.ascontiguousarray(np.array(key, dtype=np.uint64))
    out = np.zeros(4, dtype=np.uint64)
    lib().or_philox4(wbits, rounds, _p(c), _p(k), _p(out))
    return out


def u01(x: int) -> float:
    return lib().or_u01(int(x) & 0xFFFFFFFF)


def uniforms(seed: int, offset: int, n: int) -> np.ndarray:
    u = np.empty(n, dtype=np.float32)
    lib().or_uniforms(seed, offset, n, _p(u))
    return u


def uniforms_bits(seed: int, offset: int, n: int, bits: int) -> np.ndarray:
    L = lib()
    if not getattr(L, "_ubits_sig", False):
        L.or_uniforms_bits.restype = None
        L.or_uniforms_bits.argtypes = [C.c_uint64, C.c_uint64, C.c_int64, C.c_int, C.c_void_p]
        L._ubits_sig = True
    u = np.empty(n, dtype=np.float32)
    L.or_uniforms_bits(seed, offset, n, bits, _p(u))
    return u


# ---------------------------------------------------------------- Gaussian
def phiinv(u):
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float32))
    z = np.empty(u.shape, dtype=np.float64)
    lib().or_phiinv_n(_p(u), u.size, _p(z))
    return z


def phiinv_f64(u: float) -> float:
    return lib().or_phiinv(float(u))


# ---------------------------------------------------------------- tables
def pwc_table(n: int = 1024, construction: int = 0) -> np.ndarray:
    q = np.empty(n, dtype=np.float64)
    if lib().or_pwc_table(n, construction, _p(q)) != 0:
        raise ValueError("bad piecewise constant table arguments")
    return q


def pwc_l2err2(q: np.ndarray) -> float:
    q = np.ascontiguousarray(q, dtype=np.float64)
    return lib().or_pwc_l2err2(q.size, _p(q))


def pwl_table(K: int = 15, r: float = 0.5):
    a = np.empty(K + 1, dtype=np.float64)
    b = np.empty(K + 1, dtype=np.float64)
    if lib().or_pwl_table(K, r, _p(a), _p(b)) != 0:
        raise ValueError("bad piecewise linear table arguments")
    return a, b


def pwl_l2err2(alpha, beta, r: float = 0.5) -> float:
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    return lib().or_pwl_l2err2(a.size - 1, r, _p(a), _p(b))


def pwl_index(v: float, K: int = 15, r: float = 0.5) -> int:
    return lib().or_pwl_index(float(v), K, r)


# ---------------------------------------------------------------- samplers
def sample_pwc(table_f32, u):
    t = np.ascontiguousarray(table_f32, dtype=np.float32)
    u = np.ascontiguousarray(u, dtype=np.float32)
    out = np.empty(u.size, dtype=np.float64)
    idx = np.empty(u.size, dtype=np.int32)
    lib().or_sample_pwc(_p(t), t.size, _p(u), u.size, _p(out), _p(idx))
    return out, idx


def sample_pwl(alpha_f32, beta_f32, u):
    a = np.ascontiguousarray(alpha_f32, dtype=np.float32)
    b = np.ascontiguousarray(beta_f32, dtype=np.float32)
    u = np.ascontiguousarray(u, dtype=np.float32)
    out = np.empty(u.size, dtype=np.float64)
    idx = np.empty(u.size, dtype=np.int32)
    lib().or_sample_pwl(_p(a), _p(b), a.size - 1, _p(u), u.size, _p(out), _p(idx))
    return out, idx


# ---------------------------------------------------------------- MLMC
def sde_params(model=MODEL_GBM, scheme=SCHEME_EM, payoff=PAYOFF_CALL, approx=APPROX_PWL,
               X0=1.0, T=1.0, K=1.0, mu=0.05, sigma=0.2, kappa=0.0, theta=0.0,
               discount=None) -> SdeParams:
    if discount is None:
        discount = float(np.exp(-mu * T)) if (model == MODEL_GBM and payoff == PAYOFF_CALL) else 1.0
    return SdeParams(model, scheme, payoff, approx, X0, T, K, mu, sigma, kappa, theta, discount)


def _approx_arrays(approx_table):
    if isinstance(approx_table, tuple):
        a = np.ascontiguousarray(approx_table[0], dtype=np.float32)
        b = np.ascontiguousarray(approx_table[1], dtype=np.float32)
        return a, b, a.size - 1
    t = np.ascontiguousarray(approx_table, dtype=np.float32)
    if t.ndim == 2:  # piecewise polynomial rows 0..K x 4 coefficients
        t = t.reshape(-1)
        return t, t, t.size // 4 - 1
    return t, t, t.size


def mlmc_level(prm: SdeParams, approx_table, level: int, kind: int, n_paths: int,
               path_offset: int = 0, seed: int = 0, tag: int = 1) -> np.ndarray:
    a, b, K = _approx_arrays(approx_table)
    sums = np.zeros(5, dtype=np.float64)
    lib().or_mlmc_level(C.byref(prm), _p(a), _p(b), K, level, kind, n_paths, path_offset,
                        seed, tag, _p(sums))
    return sums


def mlmc_paths(prm: SdeParams, approx_table, level: int, kind: int, n_paths: int,
               path_offset: int = 0, seed: int = 0, tag: int = 1) -> np.ndarray:
    a, b, K = _approx_arrays(approx_table)
    y = np.empty(n_paths, dtype=np.float64)
    lib().or_mlmc_paths(C.byref(prm), _p(a), _p(b), K, level, kind, n_paths, path_offset,
                        seed, tag, _p(y))
    return y


def mlmc_alloc(v, c, eps):
    v = np.ascontiguousarray(v, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    m = np.empty(v.size, dtype=np.float64)
    T = lib().or_mlmc_alloc(v.size, _p(v), _p(c), eps, _p(m))
    return T, m


# ---------------------------------------------------------------- NCX2
def gammp(a, x):
    return lib().or_gammp(float(a), float(x))


def ncx2_cdf(x, nu, lam):
    return lib().or_ncx2_cdf(float(x), float(nu), float(lam))


def ncx2_pdf(x, nu, lam):
    return lib().or_ncx2_pdf(float(x), float(nu), float(lam))


def ncx2_ppf(u, nu, lam):
    return lib().or_ncx2_ppf(float(u), float(nu), float(lam))


def ncx2_sf(x, nu, lam):
    return lib().or_ncx2_sf(float(x), float(nu), float(lam))


def ncx2_isf(v, nu, lam):
    return lib().or_ncx2_isf(float(v), float(nu), float(lam))


def ncx2_P(u, x, y):
    return lib().or_ncx2_P(float(u), float(x), float(y))


def _ncx2_poly_sig(L):
    if not getattr(L, "_ncx2_poly_sig", False):
        L.or_ncx2_poly_table.restype = C.c_int
        L.or_ncx2_poly_table.argtypes = [C.c_double, C.c_int, C.c_int, C.c_int, C.c_void_p]
        L.or_ncx2_poly_P.restype = C.c_double
        L.or_ncx2_poly_P.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double]
        L.or_ncx2_poly_ppf.restype = C.c_double
        L.or_ncx2_poly_ppf.argtypes = [C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_double, C.c_double]
        L.or_ncx2_poly_rmse.restype = C.c_double
        L.or_ncx2_poly_rmse.argtypes = [C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_double]
        L._ncx2_poly_sig = True
    return L


def ncx2_poly_table(nu, K=8, n_knots=16, deg=1):
    """Section 5.1 table: array (n_knots, 2 halves, K+1 rows, 4 coefficients)."""
    L = _ncx2_poly_sig(lib())
    c = np.zeros(n_knots * 2 * (K + 1) * 4, dtype=np.float64)
    if L.or_ncx2_poly_table(float(nu), K, n_knots, deg, _p(c)) != 0:
        raise ValueError("bad NCX2 table arguments")
    return c.reshape(n_knots, 2, K + 1, 4)


def _flat(coef):
    return np.ascontiguousarray(coef, dtype=np.float64).reshape(-1)


def ncx2_poly_P(coef, u, y):
    L = _ncx2_poly_sig(lib())
    c = _flat(coef)
    n_knots, _, K1, _ = coef.shape
    return L.or_ncx2_poly_P(_p(c), K1 - 1, n_knots, float(u), float(y))


def ncx2_poly_ppf(coef, nu, u, lam):
    L = _ncx2_poly_sig(lib())
    c = _flat(coef)
    n_knots, _, K1, _ = coef.shape
    return L.or_ncx2_poly_ppf(_p(c), float(nu), K1 - 1, n_knots, float(u), float(lam))


def ncx2_poly_rmse(coef, nu, lam):
    L = _ncx2_poly_sig(lib())
    c = _flat(coef)
    n_knots, _, K1, _ = coef.shape
    return L.or_ncx2_poly_rmse(_p(c), float(nu), K1 - 1, n_knots, float(lam))


# ---------------------------------------------------------------- MLP
def mlp_forward(params: dict, x: np.ndarray) -> np.ndarray:
    H = params["b1"].size
    arrs = [np.ascontiguousarray(params[k], dtype=np.float64) for k in ("W1", "b1", "W2", "b2", "w3", "b3")]
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 2)
    y = np.empty(x.shape[0], dtype=np.float64)
    lib().or_mlp_forward(H, *[_p(a) for a in arrs], _p(x), x.shape[0], _p(y))
    return y


def mlp_grad(params: dict, x: np.ndarray, t: np.ndarray):
    H = params["b1"].size
    names = ("W1", "b1", "W2", "b2", "w3", "b3")
    arrs = [np.ascontiguousarray(params[k], dtype=np.float64) for k in names]
    grads = [np.zeros_like(a) for a in arrs]
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 2)
    t = np.ascontiguousarray(t, dtype=np.float64)
    loss = lib().or_mlp_grad(H, *[_p(a) for a in arrs], _p(x), _p(t), x.shape[0],
                             *[_p(g) for g in grads])
    return loss, dict(zip(names, grads))


# ---------------------------------------------------------------- piecewise polynomials
def pwp_table(K: int = 15, deg: int = 3):
    """Piecewise polynomial table (rows 0..K x 4 coefficients in the local
    variable s) and its squared L2 error."""
    L = lib()
    if not getattr(L, "_pwp_sig", False):
        L.or_pwp_table.restype = C.c_double
        L.or_pwp_table.argtypes = [C.c_int, C.c_int, C.c_void_p]
        L.or_sample_pwp.restype = None
        L.or_sample_pwp.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_void_p]
        L._pwp_sig = True
    c = np.zeros(4 * (K + 1), dtype=np.float64)
    e2 = L.or_pwp_table(K, deg, _p(c))
    return c.reshape(K + 1, 4), e2


def sample_pwp(coef_f32, u):
    pwp_table(1, 1)  # binds the signatures
    c = np.ascontiguousarray(coef_f32, dtype=np.float32).reshape(-1)
    u = np.ascontiguousarray(u, dtype=np.float32)
    out = np.empty(u.size, dtype=np.float64)
    lib().or_sample_pwp(_p(c), c.size // 4 - 1, _p(u), u.size, _p(out))
    return out
