"""Python binding of libaicdf (approximate inverse-CDF random variables on GB300).

Argument marshalling only: every step of the computation runs in the CUDA
library ``libaicdf.so`` built in-tree by ``build.py`` (``__graft_entry__.build()``).
There is no CPU fallback; if the library is missing every call raises.

Functions mirror the C ABI in ``include/aicdf.h`` (without the ``aicdf_``
prefix).  Device buffers are torch CUDA tensors (or raw integer pointers);
streams default to torch's current stream.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libaicdf.so")

# enums (include/aicdf.h)
OK, ERR_ARG, ERR_CUDA, ERR_NOCONVERGE, ERR_DOMAIN, ERR_STATE, ERR_NOMEM, ERR_UNSUPPORTED = range(8)
PWC, PWL, EXACT, EXACT_LIB, PWP = 0, 1, 2, 3, 4
Z_E, Z_C, Z_I, Z_V = 0, 1, 2, 3
F32, F16 = 0, 1
MODEL_GBM, MODEL_CIR = 0, 1
SCHEME_EM, SCHEME_MILSTEIN = 0, 1
PAYOFF_X, PAYOFF_CALL, PAYOFF_ASIAN = 0, 1, 2
KIND_APPROX2, KIND_CORR4, KIND_EXACT2, KIND_PLAIN, KIND_PLAIN_APPROX = range(5)
SUMS = 5  # AICDF_SUMS_PER_TERM: (sum Y, sum Y^2, sum Y^3, sum Y^4, n) per term

_lock = threading.Lock()
_lib = None


class AicdfError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.aicdf_status_str(status).decode() if _lib is not None else str(status)
        if status == ERR_CUDA and _lib is not None:
            msg += f" (cudaError {_lib.aicdf_last_cuda_error()})"
        super().__init__(f"{where}: {msg}")
        self.status = status


class SdeParams(C.Structure):
    _fields_ = [("model", C.c_int), ("scheme", C.c_int), ("payoff", C.c_int), ("reserved", C.c_int),
                ("X0", C.c_double), ("T", C.c_double), ("K", C.c_double), ("mu", C.c_double),
                ("sigma", C.c_double), ("kappa", C.c_double), ("theta", C.c_double),
                ("discount", C.c_double)]


EST_NESTED, EST_REGULAR, EST_PLAIN, EST_ADAPTIVE = 0, 1, 2, 3
MAX_LEVELS = 24


class MlmcOpts(C.Structure):
    _fields_ = [("eps", C.c_double), ("estimator", C.c_int), ("L_min", C.c_int), ("L_max", C.c_int),
                ("fixed_L", C.c_int), ("n_pilot", C.c_uint64), ("seed", C.c_uint64),
                ("weak_order", C.c_double)]


class MlmcResult(C.Structure):
    _fields_ = [("estimate", C.c_double), ("variance", C.c_double), ("bias", C.c_double),
                ("gpu_ms", C.c_double), ("wall_ms", C.c_double), ("L", C.c_int),
                ("converged", C.c_int), ("n_terms", C.c_int), ("launches", C.c_int),
                ("paths", (C.c_uint64 * 2) * MAX_LEVELS), ("mean", (C.c_double * 2) * MAX_LEVELS),
                ("var", (C.c_double * 2) * MAX_LEVELS), ("kurt", (C.c_double * 2) * MAX_LEVELS),
                ("cost_ns", (C.c_double * 2) * MAX_LEVELS), ("exact_level", C.c_int * MAX_LEVELS)]

    def as_dict(self):
        L, t = self.L, self.n_terms
        lv = range(L + 1) if t == 2 or self.paths[0][0] else [L]
        return {"estimate": self.estimate, "variance": self.variance, "bias": self.bias,
                "gpu_ms": self.gpu_ms, "wall_ms": self.wall_ms, "L": L, "converged": bool(self.converged),
                "launches": self.launches,
                "levels": [{"l": l, "paths": list(self.paths[l])[:t], "mean": list(self.mean[l])[:t],
                            "var": list(self.var[l])[:t], "kurt": list(self.kurt[l])[:t],
                            "cost_ns": list(self.cost_ns[l])[:t], "exact_level": bool(self.exact_level[l])}
                           for l in lv]}


class BatchTerm(C.Structure):
    _fields_ = [("set", C.c_uint32), ("level", C.c_int32), ("kind", C.c_int32), ("tag", C.c_uint32),
                ("n_paths", C.c_uint64), ("path_offset", C.c_uint64)]


class Schedule(C.Structure):
    _fields_ = [("tile_paths", C.c_int), ("block_threads", C.c_int), ("blocks_per_sm", C.c_int),
                ("var16", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# name -> (restype, argtypes); every entry point of include/aicdf.h
_P, _I, _U32, _U64, _SZ, _D = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_size_t, C.c_double
SIGNATURES = {
    "aicdf_status_str": (C.c_char_p, [_I]),
    "aicdf_last_cuda_error": (_I, []),
    "aicdf_version": (_I, []),
    "aicdf_table_build": (_I, [_I, _I, _I, C.POINTER(_P)]),
    "aicdf_table_destroy": (None, [_P]),
    "aicdf_table_get": (_I, [_P, _P, _P, _I, C.POINTER(_I)]),
    "aicdf_table_info": (_I, [_P, C.POINTER(_I), C.POINTER(_I)]),
    "aicdf_sample": (_I, [_P, _I, _P, _U64, _U64, _SZ, _P, _I, _P]),
    "aicdf_sample_to_host": (_I, [_P, _I, _U64, _U64, _SZ, _P, _I, _P, _SZ, _P]),
    "aicdf_sample_bits": (_I, [_P, _I, _I, _U64, _U64, _SZ, _P, _I, _P]),
    "aicdf_mlmc_level_workspace_bytes": (_SZ, []),
    "aicdf_mlmc_level": (_I, [_P, _P, _I, _I, _U64, _U64, _U64, _U32, _P, _P, _SZ, _P]),
    "aicdf_mlmc_allocate": (_I, [_I, _P, _P, _D, _P, _P]),
    "aicdf_mlmc_level_noalloc": (_I, [_P, _P, _I, _I, _U64, _U64, _U64, _U32, _P, _P]),
    "aicdf_batch_create": (_I, [_P, _I, _P, _I, _P, _U64, C.POINTER(_P)]),
    "aicdf_batch_destroy": (None, [_P]),
    "aicdf_batch_workspace_bytes": (_SZ, [_P, _P]),
    "aicdf_batch_run": (_I, [_P, _P, _P, _P, _SZ, _P]),
    "aicdf_batch_info": (_I, [_P, _P, C.POINTER(_I), C.POINTER(_I)]),
    "aicdf_batch_autotune": (_I, [_P, _I, _P, _P, _SZ, _P, C.c_char_p, _P, C.POINTER(_D)]),
    "aicdf_ncx2_ppf": (_I, [_P, _P, _D, _SZ, _P, _P, _P]),
    "aicdf_ncx2_targets": (_I, [_D, C.c_float, C.c_float, _U64, _U32, _SZ, _P, _P, _P, _P, _P]),
    "aicdf_surrogate_create": (_I, [_D, _U64, C.POINTER(_P)]),
    "aicdf_surrogate_destroy": (None, [_P]),
    "aicdf_surrogate_param_count": (_I, []),
    "aicdf_surrogate_get_params": (_I, [_P, _P, _I]),
    "aicdf_surrogate_set_params": (_I, [_P, _P, _I]),
    "aicdf_surrogate_save": (_I, [_P, C.c_char_p]),
    "aicdf_surrogate_load": (_I, [C.c_char_p, _P]),
    "aicdf_surrogate_eval": (_I, [_P, _P, _P, _SZ, _P, _P]),
    "aicdf_surrogate_grad": (_I, [_P, _P, _P, _P, _SZ, _P, _P]),
    "aicdf_surrogate_train_step": (_I, [_P, _P, _P, _P, _SZ, C.c_float, _P, _P]),
    "aicdf_surrogate_train": (_I, [_P, _P, _P, _P, _SZ, _SZ, _I, C.c_float, C.c_float, _P, _P]),
    "aicdf_cir_level": (_I, [_P, _P, _I, _I, _U64, _U64, _U64, _U32, _P, _P, _SZ, _P, _P]),
    "aicdf_ncx2_table_build": (_I, [_D, _I, _I, _I, _P]),
    "aicdf_ncx2_table_destroy": (None, [_P]),
    "aicdf_ncx2_table_info": (_I, [_P, _P, _P, _P, _P]),
    "aicdf_ncx2_table_get": (_I, [_P, _P, _SZ, _P]),
    "aicdf_ncx2_table_eval": (_I, [_P, _P, _P, _SZ, _P, _P]),
    "aicdf_cir_level_table": (_I, [_P, _P, _I, _I, _U64, _U64, _U64, _U32, _P, _P, _SZ, _P, _P]),
    "aicdf_mlmc_run_workspace_bytes": (_SZ, []),
    "aicdf_mlmc_run": (_I, [_P, _P, _P, _P, _P, _SZ, _P]),
    "aicdf_mlmc_run_sets_workspace_bytes": (_SZ, [_I]),
    "aicdf_mlmc_run_sets": (_I, [_P, _I, _P, _P, _P, _P, _SZ, _P]),
}


def lib():
    """Load libaicdf.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != OK:
        raise AicdfError(status, where)


def _sums(x, terms: int = 1):
    """Pointer of a sums buffer after checking that it holds SUMS values per
    term (a shorter buffer would be overrun by the device writes)."""
    if hasattr(x, "numel") and hasattr(x, "element_size"):
        if x.element_size() != 8 or x.numel() < SUMS * terms:
            raise ValueError(f"sums must hold {SUMS * terms} float64 values ({SUMS} per term)")
    return _ptr(x)


def _ptr(x):
    """Device/host pointer of a torch tensor, numpy array or int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Table:
    """Owning handle of an aicdf_table (host FP64 coefficients)."""

    def __init__(self, method: int, n: int, construction: int = Z_E):
        L = lib()
        h = C.c_void_p()
        _check(L.aicdf_table_build(method, n, construction, C.byref(h)), "table_build")
        self.handle = h
        self.method = method
        self.n = n

    def coefficients(self):
        import numpy as np
        cnt = {PWC: self.n, PWL: self.n + 1, PWP: 4 * (self.n + 1)}[self.method]
        c0 = np.zeros(cnt, dtype=np.float64)
        c1 = np.zeros(cnt, dtype=np.float64)
        got = C.c_int()
        _check(lib().aicdf_table_get(self.handle, c0.ctypes.data, c1.ctypes.data, cnt, C.byref(got)),
               "table_get")
        if self.method == PWP:
            return (c0.reshape(self.n + 1, 4),)
        return (c0,) if self.method == PWC else (c0, c1)

    def info(self):
        m, n = C.c_int(), C.c_int()
        _check(lib().aicdf_table_info(self.handle, C.byref(m), C.byref(n)), "table_info")
        return m.value, n.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.aicdf_table_destroy(h)
            self.handle = None


def table_build(method: int, n: int, construction: int = Z_E) -> Table:
    return Table(method, n, construction)


def _th(table):
    return None if table is None else table.handle


def sample(table, method: int, out, u=None, seed: int = 0, offset: int = 0, n: int | None = None,
           out_dtype: int | None = None, stream=None):
    """aicdf_sample: fill device buffer `out` (torch float32/float16 tensor)."""
    if n is None:
        n = out.numel()
    if out_dtype is None:
        import torch
        out_dtype = F16 if out.dtype == torch.float16 else F32
    _check(lib().aicdf_sample(_th(table), method, _ptr(u), seed, offset, n, _ptr(out), out_dtype,
                              _stream(stream)), "sample")
    return out


def sample_bits(table, method: int, bits: int, out, seed: int = 0, offset: int = 0, n: int | None = None,
                out_dtype: int | None = None, stream=None):
    """aicdf_sample_bits: the method evaluated at B-bit truncated Philox uniforms."""
    if n is None:
        n = out.numel()
    if out_dtype is None:
        import torch
        out_dtype = F16 if out.dtype == torch.float16 else F32
    _check(lib().aicdf_sample_bits(_th(table), method, bits, seed, offset, n, _ptr(out), out_dtype,
                                   _stream(stream)), "sample_bits")
    return out


def sample_to_host(table, method: int, host_out, staging, seed: int = 0, offset: int = 0,
                   n: int | None = None, out_dtype: int | None = None, stream=None):
    """aicdf_sample_to_host: generate into `staging` (device) and copy to `host_out`."""
    if n is None:
        n = host_out.numel()
    if out_dtype is None:
        import torch
        out_dtype = F16 if host_out.dtype == torch.float16 else F32
    nbytes = staging.numel() * staging.element_size()
    _check(lib().aicdf_sample_to_host(_th(table), method, seed, offset, n, _ptr(host_out), out_dtype,
                                      _ptr(staging), nbytes, _stream(stream)), "sample_to_host")
    return host_out


def sde_params(model=MODEL_GBM, scheme=SCHEME_EM, payoff=PAYOFF_CALL, X0=1.0, T=1.0, K=1.0,
               mu=0.05, sigma=0.2, kappa=0.0, theta=0.0, discount=None) -> SdeParams:
    import math
    if discount is None:
        discount = math.exp(-mu * T) if (model == MODEL_GBM and payoff == PAYOFF_CALL) else 1.0
    return SdeParams(model, scheme, payoff, 0, X0, T, K, mu, sigma, kappa, theta, discount)


def mlmc_level_workspace_bytes() -> int:
    return lib().aicdf_mlmc_level_workspace_bytes()


def mlmc_level(params: SdeParams, table: Table, level: int, kind: int, n_paths: int, sums,
               workspace, path_offset: int = 0, seed: int = 0, tag: int = 1, stream=None):
    """aicdf_mlmc_level: sums (device float64[SUMS]) <- [sum Y, sum Y^2, sum Y^3, sum Y^4, n]."""
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().aicdf_mlmc_level(C.byref(params), table.handle, level, kind, n_paths, path_offset,
                                  seed, tag, _sums(sums), _ptr(workspace), nbytes, _stream(stream)),
           "mlmc_level")
    return sums


def mlmc_level_noalloc(params: SdeParams, table: Table, level: int, kind: int, n_paths: int, sums,
                       path_offset: int = 0, seed: int = 0, tag: int = 1, stream=None):
    """aicdf_mlmc_level_noalloc: like mlmc_level, for callers that cannot
    allocate device memory; the scratch lives in a fixed array inside the
    library, shared by all calls (serialise calls that could overlap)."""
    _check(lib().aicdf_mlmc_level_noalloc(C.byref(params), table.handle, level, kind, n_paths,
                                          path_offset, seed, tag, _sums(sums), _stream(stream)),
           "mlmc_level_noalloc")
    return sums


def mlmc_allocate(v, c, eps: float):
    """aicdf_mlmc_allocate (host): optimal path counts and total time."""
    import numpy as np
    v = np.ascontiguousarray(v, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    m = np.zeros(v.size, dtype=np.float64)
    tot = C.c_double()
    _check(lib().aicdf_mlmc_allocate(v.size, v.ctypes.data, c.ctypes.data, eps, m.ctypes.data,
                                     C.byref(tot)), "mlmc_allocate")
    return tot.value, m


def mlmc_run_workspace_bytes() -> int:
    return lib().aicdf_mlmc_run_workspace_bytes()


def mlmc_run(params: SdeParams, table: Table, eps: float, workspace, estimator: int = EST_NESTED,
             L_min: int = 2, L_max: int = 20, fixed_L: int = -1, n_pilot: int = 10000, seed: int = 0,
             weak_order: float = 1.0, stream=None) -> MlmcResult:
    """aicdf_mlmc_run: estimate E[P] to RMSE eps (synchronous)."""
    o = MlmcOpts(eps, estimator, L_min, L_max, fixed_L, n_pilot, seed, weak_order)
    r = MlmcResult()
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().aicdf_mlmc_run(C.byref(params), table.handle, C.byref(o), C.byref(r), _ptr(workspace),
                                nbytes, _stream(stream)), "mlmc_run")
    return r


def mlmc_run_sets_workspace_bytes(n_sets: int) -> int:
    return lib().aicdf_mlmc_run_sets_workspace_bytes(n_sets)


def mlmc_run_sets(sets, table: Table, eps: float, workspace, estimator: int = EST_NESTED, L_min: int = 2,
                  L_max: int = 20, fixed_L: int = -1, n_pilot: int = 10000, seed: int = 0,
                  weak_order: float = 1.0, stream=None):
    """aicdf_mlmc_run_sets: one estimate per parameter set, all sets' paths in
    shared batched launches (synchronous).  Returns a list of MlmcResult."""
    o = MlmcOpts(eps, estimator, L_min, L_max, fixed_L, n_pilot, seed, weak_order)
    arr = (SdeParams * len(sets))(*sets)
    res = (MlmcResult * len(sets))()
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().aicdf_mlmc_run_sets(arr, len(sets), table.handle, C.byref(o), res, _ptr(workspace), nbytes,
                                     _stream(stream)), "mlmc_run_sets")
    return list(res)


class Batch:
    """Owning handle of an aicdf_batch: many MLMC terms in one persistent launch."""

    def __init__(self, sets, terms, table: Table, seed: int = 0):
        L = lib()
        self._sets = (SdeParams * len(sets))(*sets)
        self._terms = (BatchTerm * len(terms))(*terms)
        self.n_terms = len(terms)
        h = C.c_void_p()
        _check(L.aicdf_batch_create(self._sets, len(sets), self._terms, len(terms), table.handle, seed,
                                    C.byref(h)), "batch_create")
        self.handle = h

    def workspace_bytes(self, sched: Schedule) -> int:
        return lib().aicdf_batch_workspace_bytes(self.handle, C.byref(sched))

    def run(self, sched: Schedule, sums, workspace, stream=None):
        nbytes = workspace.numel() * workspace.element_size()
        _check(lib().aicdf_batch_run(self.handle, C.byref(sched), _sums(sums, self.n_terms), _ptr(workspace), nbytes,
                                     _stream(stream)), "batch_run")
        return sums

    def info(self, sched: Schedule):
        n, g = C.c_int(), C.c_int()
        _check(lib().aicdf_batch_info(self.handle, C.byref(sched), C.byref(n), C.byref(g)), "batch_info")
        return n.value, g.value

    def autotune(self, sums, workspace, var16: int = 0, cache_path: str | None = None, stream=None):
        best = Schedule()
        ms = C.c_double()
        nbytes = workspace.numel() * workspace.element_size()
        _check(lib().aicdf_batch_autotune(self.handle, var16, _sums(sums, self.n_terms), _ptr(workspace), nbytes,
                                          _stream(stream), cache_path.encode() if cache_path else None,
                                          C.byref(best), C.byref(ms)), "batch_autotune")
        return best, ms.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.aicdf_batch_destroy(h)
            self.handle = None


# ------------------------------------------------------------------ NCX2, surrogate, CIR
CIR_EXACT, CIR_SURROGATE, CIR_DIFF, CIR_GAUSS, CIR_DIFF_GAUSS, CIR_TABLE, CIR_DIFF_TABLE = range(7)
MLP_OFFSETS = {"W1": (0, (64, 2)), "b1": (128, (64,)), "W2": (192, (64, 64)), "b2": (4288, (64,)),
               "w3": (4352, (64,)), "b3": (4416, (1,))}


def ncx2_ppf(u, lam, nu: float, out, status, stream=None):
    """aicdf_ncx2_ppf: out[i] = C^{-1}_nu(u[i]; lam[i]) (u float32, lam/out float64, device)."""
    _check(lib().aicdf_ncx2_ppf(_ptr(u), _ptr(lam), nu, u.numel(), _ptr(out), _ptr(status),
                                _stream(stream)), "ncx2_ppf")
    return out


def ncx2_targets(nu: float, n: int, u, lam, p, status, seed: int = 0, tag: int = 1,
                 loglam_lo: float = -4.0, loglam_hi: float = 4.0, stream=None):
    """aicdf_ncx2_targets: exact training targets P_nu(u; nu/(lam+nu)) (device float32)."""
    _check(lib().aicdf_ncx2_targets(nu, loglam_lo, loglam_hi, seed, tag, n, _ptr(u), _ptr(lam), _ptr(p),
                                    _ptr(status), _stream(stream)), "ncx2_targets")


class Surrogate:
    """Owning handle of the learned P_nu(U; y) surrogate (device weights)."""

    def __init__(self, nu: float, seed: int = 0, _handle=None):
        h = _handle
        if h is None:
            h = C.c_void_p()
            _check(lib().aicdf_surrogate_create(nu, seed, C.byref(h)), "surrogate_create")
        self.handle = h
        self.nu = nu
        self.n_params = lib().aicdf_surrogate_param_count()

    def save(self, path: str):
        """aicdf_surrogate_save: nu and the weights to a host file."""
        _check(lib().aicdf_surrogate_save(self.handle, os.fsencode(path)), "surrogate_save")

    @classmethod
    def load(cls, path: str, nu: float | None = None):
        """aicdf_surrogate_load: a new handle from a file written by save()."""
        h = C.c_void_p()
        _check(lib().aicdf_surrogate_load(os.fsencode(path), C.byref(h)), "surrogate_load")
        import struct
        with open(path, "rb") as f:
            f.read(8)
            file_nu = struct.unpack("<d", f.read(8))[0]
        return cls(file_nu if nu is None else nu, _handle=h)

    def get_params(self):
        import numpy as np
        p = np.zeros(4420, dtype=np.float32)
        _check(lib().aicdf_surrogate_get_params(self.handle, p.ctypes.data, p.size), "surrogate_get_params")
        return p[: self.n_params]

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().aicdf_surrogate_set_params(self.handle, p.ctypes.data, p.size), "surrogate_set_params")

    def params_dict(self):
        p = self.get_params().astype("float64")
        return {k: p[o:o + int(__import__("numpy").prod(s))].reshape(s) for k, (o, s) in MLP_OFFSETS.items()}

    def eval(self, u, lam, out, stream=None):
        _check(lib().aicdf_surrogate_eval(self.handle, _ptr(u), _ptr(lam), u.numel(), _ptr(out),
                                          _stream(stream)), "surrogate_eval")
        return out

    def grad(self, u, lam, target, grad_out, stream=None):
        _check(lib().aicdf_surrogate_grad(self.handle, _ptr(u), _ptr(lam), _ptr(target), u.numel(),
                                          _ptr(grad_out), _stream(stream)), "surrogate_grad")
        return grad_out

    def train_step(self, u, lam, target, lr: float, loss=None, stream=None):
        _check(lib().aicdf_surrogate_train_step(self.handle, _ptr(u), _ptr(lam), _ptr(target), u.numel(),
                                                lr, _ptr(loss), _stream(stream)), "surrogate_train_step")

    def train(self, u, lam, target, batch: int, epochs: int, lr: float, lr_final: float, loss=None,
              stream=None):
        _check(lib().aicdf_surrogate_train(self.handle, _ptr(u), _ptr(lam), _ptr(target), u.numel(), batch,
                                           epochs, lr, lr_final, _ptr(loss), _stream(stream)),
               "surrogate_train")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.aicdf_surrogate_destroy(h)
            self.handle = None


def cir_level(params: SdeParams, surrogate, level: int, kind: int, n_paths: int, sums, workspace, status,
              path_offset: int = 0, seed: int = 0, tag: int = 1, stream=None):
    """aicdf_cir_level: sums <- [sum Y, sum Y^2, sum Y^3, sum Y^4, n] for a CIR kind (see aicdf.h)."""
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().aicdf_cir_level(C.byref(params), None if surrogate is None else surrogate.handle, level,
                                 kind, n_paths, path_offset, seed, tag, _sums(sums), _ptr(workspace), nbytes,
                                 _ptr(status), _stream(stream)), "cir_level")
    return sums


class Ncx2Table:
    """aicdf_ncx2_table_*: the Section 5.1 tabulated inverse for one nu."""

    def __init__(self, nu: float, K: int = 16, n_knots: int = 16, degree: int = 1):
        h = C.c_void_p()
        _check(lib().aicdf_ncx2_table_build(float(nu), K, n_knots, degree, C.byref(h)), "ncx2_table_build")
        self.handle = h
        self.nu, self.K, self.n_knots, self.degree = float(nu), K, n_knots, degree

    def coefficients(self) -> np.ndarray:
        """FP64 coefficients as (n_knots, 2 halves, K+1 rows, 4 powers)."""
        import numpy as np
        n = C.c_size_t()
        _check(lib().aicdf_ncx2_table_get(self.handle, None, 0, C.byref(n)), "ncx2_table_get")
        c = np.zeros(n.value, dtype=np.float64)
        _check(lib().aicdf_ncx2_table_get(self.handle, c.ctypes.data, n.value, C.byref(n)), "ncx2_table_get")
        return c.reshape(self.n_knots, 2, self.K + 1, 4)

    def info(self):
        nu, K, nk, d = C.c_double(), C.c_int(), C.c_int(), C.c_int()
        _check(lib().aicdf_ncx2_table_info(self.handle, C.byref(nu), C.byref(K), C.byref(nk), C.byref(d)),
               "ncx2_table_info")
        return nu.value, K.value, nk.value, d.value

    def eval(self, u, lam, out, stream=None):
        """out <- C~^{-1}_nu(u; lam) (device float32 tensors of equal length)."""
        _check(lib().aicdf_ncx2_table_eval(self.handle, _ptr(u), _ptr(lam), out.numel(), _ptr(out),
                                           _stream(stream)), "ncx2_table_eval")
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.aicdf_ncx2_table_destroy(h)
            self.handle = None


def cir_level_table(params: SdeParams, table: Ncx2Table, level: int, kind: int, n_paths: int, sums, workspace,
                    status, path_offset: int = 0, seed: int = 0, tag: int = 1, stream=None):
    """aicdf_cir_level_table: sums <- [sum Y, sum Y^2, sum Y^3, sum Y^4, n] with the tabulated approximation."""
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().aicdf_cir_level_table(C.byref(params), table.handle, level, kind, n_paths, path_offset, seed,
                                       tag, _sums(sums), _ptr(workspace), nbytes, _ptr(status), _stream(stream)),
           "cir_level_table")
    return sums
