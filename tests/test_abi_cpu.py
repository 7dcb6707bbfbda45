"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/*.h, and its host-side logic (table build, allocation,
argument validation) agrees with the oracle and the header's contract."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2012_09715_gb300 import build as b
    b.build()
    import paper_2012_09715_gb300 as P
    P.lib()
    return P


def _declared_symbols():
    syms = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(aicdf_[a-z0-9_]+)\s*\(", text):
            syms.add(m.group(1))
    return syms


def test_library_exports_every_declared_symbol(P):
    syms = _declared_symbols()
    assert len(syms) >= 10
    L = C.CDLL(P.LIB_PATH)
    missing = [s for s in sorted(syms) if not hasattr(L, s)]
    assert not missing, missing
    # and the binding wraps every one of them
    assert syms <= set(P.SIGNATURES), sorted(syms - set(P.SIGNATURES))


def test_status_strings_and_version(P):
    L = P.lib()
    for s in range(8):
        assert L.aicdf_status_str(s)
    assert L.aicdf_version() >= 100


def test_table_build_matches_oracle(P, orc):
    """The library's FP64 table build (its own inverse CDF, centred-basis
    normal equations, expm1 form of Z^E) agrees with the oracle's."""
    for K in (1, 4, 15, 16, 24):
        t = P.table_build(P.PWL, K)
        a, b = t.coefficients()
        oa, ob = orc.pwl_table(K, 0.5)
        # both sides are within ~2e-12 of mpmath: the moments M1 - m M0 lose
        # a few digits to cancellation in FP64
        assert np.allclose(a, oa, rtol=5e-12, atol=1e-14)
        assert np.allclose(b, ob, rtol=5e-12, atol=1e-14)
        assert t.info() == (P.PWL, K)
    for n in (2, 8, 1024, 4096):
        for cons in (P.Z_E, P.Z_C, P.Z_I, P.Z_V):
            q = P.table_build(P.PWC, n, cons).coefficients()[0]
            oq = orc.pwc_table(n, cons)
            # the oracle's plain form n (phi(z_k) - phi(z_{k+1})) cancels near
            # u = 1/2: its absolute error is ~ n * 1e-16 (mpmath confirms the
            # library side to 1e-15 there)
            assert np.allclose(q, oq, rtol=1e-11, atol=n * 2e-16), (n, cons)
            assert np.array_equal(q.astype(np.float32), oq.astype(np.float32)), (n, cons)
    # the FP32 tables the kernels use are identical on both sides
    t = P.table_build(P.PWL, 15)
    a, b = t.coefficients()
    oa, ob = orc.pwl_table(15, 0.5)
    assert np.array_equal(a.astype(np.float32), oa.astype(np.float32))
    assert np.array_equal(b.astype(np.float32), ob.astype(np.float32))
    q = P.table_build(P.PWC, 1024).coefficients()[0]
    assert np.array_equal(q.astype(np.float32), orc.pwc_table(1024, 0).astype(np.float32))


def test_table_build_rejects_bad_arguments(P):
    L = P.lib()
    h = C.c_void_p()
    for m, n, c in ((P.PWC, 1000, 0), (P.PWC, 1, 0), (P.PWC, 8192, 0), (P.PWC, 64, 7), (P.PWC, 64, 4),
                    (P.PWL, 0, 0), (P.PWL, 32, 0), (9, 15, 0)):
        assert L.aicdf_table_build(m, n, c, C.byref(h)) == P.ERR_ARG
    assert L.aicdf_table_build(P.PWL, 15, 0, None) == P.ERR_ARG


def test_allocation_matches_oracle(P, orc):
    rng = np.random.default_rng(0)
    v = rng.random(9) * 1e-3
    c = 2.0 ** np.arange(9)
    T, m = P.mlmc_allocate(v, c, 1e-4)
    To, mo = orc.mlmc_alloc(v, c, 1e-4)
    assert T == pytest.approx(To, rel=1e-14)
    assert np.allclose(m, mo, rtol=1e-14)
    with pytest.raises(P.AicdfError):
        P.mlmc_allocate([1.0], [0.0], 1e-3)
    with pytest.raises(P.AicdfError):
        P.mlmc_allocate([1.0], [1.0], 0.0)


def test_sample_argument_validation_without_gpu(P):
    """Invalid requests are refused before anything touches the device."""
    L = P.lib()
    t = P.table_build(P.PWL, 15)
    tc = P.table_build(P.PWC, 1024)
    fake = 1 << 40
    # wrong table for the method, table given to an exact method, bad dtype/method
    assert L.aicdf_sample(tc.handle, P.PWL, None, 0, 0, 16, fake, P.F32, None) == P.ERR_ARG
    assert L.aicdf_sample(t.handle, P.EXACT, None, 0, 0, 16, fake, P.F32, None) == P.ERR_ARG
    assert L.aicdf_sample(t.handle, P.PWL, None, 0, 0, 16, fake, 5, None) == P.ERR_ARG
    assert L.aicdf_sample(t.handle, 11, None, 0, 0, 16, fake, P.F32, None) == P.ERR_ARG
    # misaligned output / input, null output
    assert L.aicdf_sample(t.handle, P.PWL, None, 0, 0, 16, fake + 2, P.F32, None) == P.ERR_ARG
    assert L.aicdf_sample(t.handle, P.PWL, fake + 1, 0, 0, 16, fake, P.F32, None) == P.ERR_ARG
    assert L.aicdf_sample(t.handle, P.PWL, None, 0, 0, 16, None, P.F32, None) == P.ERR_ARG
    # n = 0 is a no-op
    assert L.aicdf_sample(t.handle, P.PWL, None, 0, 0, 0, None, P.F32, None) == P.OK
    # tables too large for the kernels are refused, not truncated
    big = P.table_build(P.PWL, 20)
    assert L.aicdf_sample(big.handle, P.PWL, None, 0, 0, 16, fake, P.F32, None) == P.ERR_UNSUPPORTED
    # truncated-bit sampling: unsupported widths, bad dtype, misaligned output
    assert L.aicdf_sample_bits(t.handle, P.PWL, 12, 0, 0, 16, fake, P.F32, None) == P.ERR_UNSUPPORTED
    assert L.aicdf_sample_bits(t.handle, P.PWL, 0, 0, 0, 16, fake, P.F32, None) == P.ERR_ARG
    assert L.aicdf_sample_bits(t.handle, P.PWL, 24, 0, 0, 16, fake, P.F32, None) == P.ERR_ARG
    assert L.aicdf_sample_bits(t.handle, P.PWL, 16, 0, 0, 16, fake, 3, None) == P.ERR_ARG
    assert L.aicdf_sample_bits(t.handle, P.PWL, 16, 0, 0, 16, fake + 2, P.F32, None) == P.ERR_ARG
    assert L.aicdf_sample_bits(tc.handle, P.PWL, 16, 0, 0, 16, fake, P.F32, None) == P.ERR_ARG
    assert L.aicdf_sample_bits(t.handle, P.PWL, 16, 0, 0, 0, None, P.F32, None) == P.OK
    # host pipeline: staging too small
    assert L.aicdf_sample_to_host(t.handle, P.PWL, 0, 0, 16, fake, P.F32, fake, 1024, None) == P.ERR_ARG


def test_mlmc_argument_validation_without_gpu(P):
    L = P.lib()
    t = P.table_build(P.PWL, 15)
    prm = P.sde_params()
    ws_bytes = P.mlmc_level_workspace_bytes()
    fake = 1 << 40
    call = lambda prm, lvl, kind, n, sums=fake, ws=fake, wsb=ws_bytes: L.aicdf_mlmc_level(
        C.byref(prm), t.handle, lvl, kind, n, 0, 0, 1, sums, ws, wsb, None)
    assert call(prm, -1, P.KIND_CORR4, 10) == P.ERR_ARG
    assert call(prm, 3, 9, 10) == P.ERR_ARG
    assert call(prm, 3, P.KIND_CORR4, 0) == P.ERR_ARG
    assert call(prm, 3, P.KIND_CORR4, 10, wsb=16) == P.ERR_ARG
    assert call(prm, 3, P.KIND_CORR4, 10, sums=fake + 4) == P.ERR_ARG
    bad = P.sde_params(sigma=float("nan"))
    assert call(bad, 3, P.KIND_CORR4, 10) == P.ERR_DOMAIN
    bad = P.sde_params(T=0.0)
    assert call(bad, 3, P.KIND_CORR4, 10) == P.ERR_DOMAIN
    assert L.aicdf_mlmc_level(None, t.handle, 3, 1, 10, 0, 0, 1, fake, fake, ws_bytes, None) == P.ERR_ARG
    # the path average is for the CIR per-step calls only; unknown payoffs everywhere
    assert call(P.sde_params(payoff=P.PAYOFF_ASIAN), 3, P.KIND_CORR4, 10) == P.ERR_ARG
    assert call(P.sde_params(payoff=3), 3, P.KIND_CORR4, 10) == P.ERR_ARG


def test_pwp_table_matches_oracle(P, orc):
    """Library (shifted-Legendre projection, exponential substitution on the
    singular interval) and oracle (normal equations, z-substitution) build the
    same polynomial tables."""
    for K in (8, 15):
        for deg in (1, 2, 3):
            c = P.table_build(P.PWP, K, deg).coefficients()[0]
            o, _ = orc.pwp_table(K, deg)
            assert np.allclose(c, o, rtol=1e-9, atol=1e-11), (K, deg)
            assert np.array_equal(c.astype(np.float32), o.astype(np.float32)) or \
                np.max(np.abs(c.astype(np.float32) - o.astype(np.float32))) <= 1e-6


def test_ncx2_table_matches_oracle(P, orc):
    """Section 5.1 tables: the library's host FP64 build (its own root finder,
    Legendre projection) and the oracle's give the same RMSE against the exact
    inverse and the same approximation to 2e-5 relative (the largest gap sits
    in the deepest lower tail, where the two quadratures are cut differently)."""
    for nu, deg in ((1.0, 1), (0.8889, 3)):
        t = P.Ncx2Table(nu, 16, 16, deg)
        assert t.info() == (nu, 16, 16, deg)
        c = t.coefficients()
        o = orc.ncx2_poly_table(nu, 16, 16, deg)
        for lam in (0.5, 100.0):
            assert orc.ncx2_poly_rmse(c, nu, lam) == pytest.approx(orc.ncx2_poly_rmse(o, nu, lam), rel=1e-6)
        us = np.concatenate([np.linspace(1e-6, 1 - 1e-6, 401), 10.0 ** -np.arange(3, 16),
                             1 - 10.0 ** -np.arange(3, 16)])
        for lam in (0.3, 30.0):
            a = np.array([orc.ncx2_poly_ppf(c, nu, u, lam) for u in us])
            b = np.array([orc.ncx2_poly_ppf(o, nu, u, lam) for u in us])
            assert np.max(np.abs(a - b) / (1 + np.abs(b))) < 2e-5


def test_ncx2_table_argument_validation(P):
    L = P.lib()
    h = C.c_void_p()
    for nu, K, nk, d in ((0.0, 16, 16, 1), (-1.0, 16, 16, 1), (1.0, 0, 16, 1), (1.0, 31, 16, 1),
                         (1.0, 16, 1, 1), (1.0, 16, 65, 1), (1.0, 16, 16, 0), (1.0, 16, 16, 4)):
        assert L.aicdf_ncx2_table_build(nu, K, nk, d, C.byref(h)) == P.ERR_ARG
    assert L.aicdf_ncx2_table_build(1.0, 16, 16, 1, None) == P.ERR_ARG
    fake = 1 << 40
    big = P.Ncx2Table(2.0, 30, 32, 1)  # 32 x 2 x 31 rows: too many for a launch parameter
    assert L.aicdf_ncx2_table_eval(big.handle, fake, fake, 16, fake, None) == P.ERR_UNSUPPORTED
    t = P.Ncx2Table(2.0, 16, 16, 1)
    assert L.aicdf_ncx2_table_eval(t.handle, fake + 2, fake, 16, fake, None) == P.ERR_ARG
    assert L.aicdf_ncx2_table_eval(t.handle, fake, fake, 0, fake, None) == P.OK
    # CIR with the table: nu must match 4 kappa theta / sigma^2, and only its kinds
    prm = P.sde_params(model=P.MODEL_CIR, payoff=P.PAYOFF_X, X0=1.0, T=1.0, mu=0.0, sigma=1.0, kappa=0.5,
                       theta=1.0, discount=1.0)                      # nu = 2
    ws = P.mlmc_level_workspace_bytes()
    call = lambda tab, kind: L.aicdf_cir_level_table(C.byref(prm), tab.handle, 3, kind, 10, 0, 0, 1, fake, fake,
                                                     ws, fake, None)
    assert call(t, P.CIR_SURROGATE) == P.ERR_ARG
    bad = P.sde_params(model=P.MODEL_CIR, payoff=3, X0=1.0, T=1.0, mu=0.0, sigma=1.0, kappa=0.5, theta=1.0,
                       discount=1.0)
    assert L.aicdf_cir_level_table(C.byref(bad), t.handle, 3, P.CIR_TABLE, 10, 0, 0, 1, fake, fake, ws, fake,
                                   None) == P.ERR_ARG
    assert call(P.Ncx2Table(1.0, 16, 16, 1), P.CIR_DIFF_TABLE) == P.ERR_DOMAIN
    assert L.aicdf_cir_level(C.byref(prm), None, 3, P.CIR_TABLE, 10, 0, 0, 1, fake, fake, ws, fake, None) == P.ERR_ARG


def test_ncx2_tables_build_across_nu(P, orc):
    """The host build converges at every quadrature node for nu from 0.3 to 100
    (knots down to y = 1/225, i.e. lambda up to 224 nu, and tails down to
    1e-20), and the nu = 100 linear table has Table 5a's RMSE at lambda = 100."""
    for nu, deg in ((0.3, 1), (5.0, 3), (10.0, 3), (50.0, 1), (100.0, 1)):
        t = P.Ncx2Table(nu, 16, 16, deg)
        assert t.info()[0] == nu
    c = P.Ncx2Table(100.0, 16, 16, 1).coefficients()
    assert abs(orc.ncx2_poly_rmse(c, 100.0, 100.0) - 0.161) <= 0.0006


def test_surrogate_load_rejects_bad_files(P, tmp_path):
    """aicdf_surrogate_load refuses a missing file, a foreign file and a
    truncated one before it creates anything (no device needed)."""
    L = P.lib()
    h = C.c_void_p()
    assert L.aicdf_surrogate_load(os.fsencode(str(tmp_path / "none.bin")), C.byref(h)) == P.ERR_ARG
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a surrogate file at all")
    assert L.aicdf_surrogate_load(os.fsencode(str(bad)), C.byref(h)) == P.ERR_ARG
    short = tmp_path / "short.bin"
    short.write_bytes(b"AICDFSG1" + np.float64(0.889).tobytes() + np.int32(4417).tobytes() + b"\0" * 100)
    assert L.aicdf_surrogate_load(os.fsencode(str(short)), C.byref(h)) == P.ERR_ARG
    assert not h.value
    assert L.aicdf_surrogate_save(None, os.fsencode(str(bad))) == P.ERR_ARG
