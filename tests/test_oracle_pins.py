"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: numbers
printed in the paper, closed forms stated in its proofs, invariants of the
theorems, independent libraries (numpy, scipy, mpmath) and brute force.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _trunc_sig(x, sig):
    """Truncate toward zero to `sig` significant figures."""
    if x == 0:
        return 0.0
    e = math.floor(math.log10(abs(x))) - sig + 1
    return math.trunc(x / 10.0 ** e) * 10.0 ** e


# ---------------------------------------------------------------- Philox
def test_philox_w64_matches_numpy(orc):
    """The word-size-generic Philox, instantiated at W=64, equals numpy's
    independent Philox4x64-10 (numpy bumps the counter before each block)."""
    cases = [([0, 0, 0, 0], [0, 0]), ([5, 7, 9, 11], [123, 456]),
             ([2**64 - 1, 3, 0, 2**63], [2**64 - 1, 17])]
    for ctr, key in cases:
        bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
        ref = bg.random_raw(4)
        nxt = list(ctr)
        nxt[0] = (nxt[0] + 1) % 2**64
        if nxt[0] == 0:
            nxt[1] = (nxt[1] + 1) % 2**64
        got = orc.philox4(nxt, key, wbits=64)
        assert [int(x) for x in got] == [int(x) for x in ref], (ctr, key)


def test_philox_w32_uniformity(orc):
    """Philox4x32-10 words: chi-square on 256 bins and bit balance."""
    u = orc.uniforms(seed=0, offset=0, n=1 << 16)
    hist, _ = np.histogram(u, bins=256, range=(0.0, 1.0))
    e = u.size / 256
    chi2 = ((hist - e) ** 2 / e).sum()
    # 255 dof: mean 255, sd ~22.6; 6 sigma band
    assert 120 < chi2 < 390, chi2
    assert abs(u.mean() - 0.5) < 5 * (1 / math.sqrt(12 * u.size))


def test_philox_stream_mapping(orc):
    """Sample i of the standalone stream is word i%4 of block i//4."""
    u = orc.uniforms(seed=0x1234_5678_9ABC, offset=8, n=8)
    for i in range(8):
        j = (8 + i) // 4
        w = orc.philox4([j & 0xFFFFFFFF, j >> 32, 0, 0], [0x5678_9ABC, 0x1234], 32)
        assert u[i] == np.float32(orc.u01(int(w[(8 + i) % 4])))


def test_u01_grid(orc):
    """Open, FP32-exact midpoint grid of 2^23 cells: the top bit picks the
    half and the low 22 bits the cell, mirrored in the upper half, so that
    u(x) + u(x ^ 2^31) = 1; u in [2^-24, 1-2^-24], never 1/2, and bits 22..30
    are ignored."""
    xs = [0, 1, 511, 512, 0x3FFFFF, 0x400000, 0x7FFFFF, 0x800000, 0x7FFFFFFF, 0x80000000, 0xFFFFFE00,
          0xFFFFFFFF, 0x12345678]
    for x in xs:
        a, b = orc.u01(x), orc.u01(x ^ 0x80000000)
        assert a + b == 1.0 and a != 0.5
        assert float(np.float32(a)) == a and float(np.float32(1.0 - a)) == 1.0 - a
        assert orc.u01(x ^ 0x7FC00000) == a  # bits 22..30
        assert (a < 0.5) == (x < 0x80000000)
    assert orc.u01(0) == 2.0 ** -24 and orc.u01(0x80000000) == 1.0 - 2.0 ** -24
    assert orc.u01(0x3FFFFF) == 0.5 - 2.0 ** -24 and orc.u01(0xBFFFFFFF) == 0.5 + 2.0 ** -24
    assert orc.u01(0x0000_1235) == (2 * 0x1235 + 1) * 2.0 ** -24
    assert orc.u01(0x8000_1235) == 1.0 - (2 * 0x1235 + 1) * 2.0 ** -24
    # distinct (top bit, low 22 bits) give distinct cells
    rng = np.random.default_rng(3)
    ws = np.unique(rng.integers(0, 1 << 23, 4000)).tolist()
    us = {orc.u01(((w >> 22) << 31) | (w & 0x3FFFFF)) for w in ws}
    assert len(us) == len(ws)


@pytest.mark.parametrize("bits", [1, 8, 10, 16])
def test_truncated_uniform_stream_mapping(orc, bits):
    """Sample s = 4F j + 4h + t of the B-bit stream is field h of word t of
    Philox call j, at the midpoint (m + 1/2) 2^-B of its cell."""
    F = 32 // bits
    off, n = 4 * F * 3 + 5, 4 * F * 2 + 7
    seed = 0xABCDEF0123
    u = orc.uniforms_bits(seed=seed, offset=off, n=n, bits=bits)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(n):
        s = off + i
        j, r = divmod(s, 4 * F)
        h, t = divmod(r, 4)
        w = int(orc.philox4([j, 0, 0, 0], key, 32)[t])
        m = (w >> (h * bits)) & ((1 << bits) - 1)
        assert u[i] == np.float32((m + 0.5) / 2.0 ** bits), (bits, i)


def test_truncated_uniforms_equidistributed_and_fields_independent(orc):
    """8-bit stream: chi-square over the 256 cells, and over 16 x 16 cells of
    the top nibbles of fields 0 and 1 of the same word."""
    u = orc.uniforms_bits(seed=3, offset=0, n=1 << 17, bits=8)
    m = np.floor(u.astype(np.float64) * 256).astype(int)
    assert np.all((m + 0.5) / 256 == u)
    hist = np.bincount(m, minlength=256)
    e = m.size / 256
    assert 120 < ((hist - e) ** 2 / e).sum() < 390
    blk = m.reshape(-1, 16)                   # one Philox call = 16 samples
    a, b = blk[:, 0:4].ravel() >> 4, blk[:, 4:8].ravel() >> 4
    joint = np.bincount(a * 16 + b, minlength=256)
    e2 = a.size / 256
    assert 120 < ((joint - e2) ** 2 / e2).sum() < 390


def test_truncated_uniform_inverse_is_midpoint_pwc(orc):
    """Section 1 / Section 2.2: inverting a B-bit uniform exactly gives the
    piecewise constant approximation on 2^B equal intervals with the midpoint
    values Z^C, whose squared L2 error decays like 2^-q / q (Giles et al.)."""
    for q in (4, 8):
        u = ((np.arange(2 ** q) + 0.5) / 2 ** q).astype(np.float32)
        assert np.array_equal(orc.phiinv(u), orc.pwc_table(2 ** q, 1))
    r = [orc.pwc_l2err2(orc.pwc_table(2 ** q, 1)) * q * 2 ** q for q in (6, 8, 10, 12)]
    assert max(r) / min(r) < 1.6, r
    # a PWC table on 2^q <= 2^B intervals reads cell m >> (B - q) of a B-bit uniform
    t = orc.pwc_table(64, 0).astype(np.float32)
    u = ((np.arange(256) + 0.5) / 256).astype(np.float32)
    z, idx = orc.sample_pwc(t, u)
    assert np.array_equal(idx, np.arange(256) >> 2)


def test_unit_variance_construction(orc):
    """Construction 3 rescales Z^E to unit variance: n = 2 gives the Rademacher
    values +-1 (Section 1); the mean square is 1 for every n."""
    q2 = orc.pwc_table(2, 3)
    assert np.allclose(q2, [-1.0, 1.0], rtol=0, atol=1e-14)
    for n in (4, 64, 1024):
        q = orc.pwc_table(n, 3)
        e = orc.pwc_table(n, 0)
        assert np.mean(q * q) == pytest.approx(1.0, abs=1e-13)
        assert np.allclose(q / e, q[0] / e[0], rtol=1e-12)


# ---------------------------------------------------------------- Phi^-1
def test_phiinv_against_scipy_and_mpmath(orc):
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(0)
    u = np.concatenate([rng.random(4000), 10.0 ** -rng.uniform(1, 40, 500),
                        [2.0 ** -24, 0.5 - 2.0 ** -24, 0.25, 0.75]]).astype(np.float32)
    u = u[(u > 0) & (u < 1)]
    z = orc.phiinv(u)
    ref = sp.ndtri(u.astype(np.float64))
    assert np.allclose(z, ref, rtol=2e-14, atol=0), np.max(np.abs(z - ref) / np.abs(ref))
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 90   # erfinv(1 - 2u) loses digits as u -> 0: carry plenty
    for uu in [2.0 ** -24, 1e-30, 0.02, 0.3, 0.5 - 2.0 ** -24, 0.9]:
        exact = float(-mpmath.sqrt(2) * mpmath.erfinv(1 - 2 * mpmath.mpf(uu)))
        assert abs(orc.phiinv_f64(uu) - exact) <= 4e-16 * abs(exact)


def test_phiinv_symmetry_and_roundtrip(orc):
    from scipy.special import ndtr
    k = np.arange(0, 1 << 23, 4099, dtype=np.int64)
    u = ((2 * k + 1) * 2.0 ** -24).astype(np.float32)
    z = orc.phiinv(u)
    zr = orc.phiinv((1.0 - u.astype(np.float64)).astype(np.float32))
    assert np.array_equal(zr, -z)          # exact antisymmetry on the grid
    lo = u < 0.5
    assert np.allclose(ndtr(z[lo]), u[lo].astype(np.float64), rtol=1e-14)
    assert orc.phiinv_f64(0.5) == 0.0
    assert orc.phiinv_f64(0.0) == -math.inf and orc.phiinv_f64(1.0) == math.inf


# ---------------------------------------------------------------- PWC table
def test_pwc_listing_values(orc):
    """The listing's printed table entries are Z^E truncated to one decimal."""
    q = orc.pwc_table(1024, 0)
    for idx, val in _read_golden("pwc_listing_values.txt"):
        assert math.trunc(q[int(idx)] * 10) / 10 == pytest.approx(float(val), abs=1e-12)


def test_pwc_conditional_mean_by_quadrature(orc):
    """Z^E_k = N * int_{I_k} Phi^{-1}(u) du, checked by independent quadrature."""
    from scipy.integrate import quad
    from scipy.special import ndtri
    n = 1024
    q = orc.pwc_table(n, 0)
    for k in [0, 1, 100, 511, 512, 900, 1022, 1023]:
        val, err = quad(lambda t: ndtri(t), k / n, (k + 1) / n, epsabs=1e-14, epsrel=1e-13, limit=200)
        assert q[k] == pytest.approx(n * val, rel=1e-9, abs=1e-12), k


def test_pwc_theorem21_conditions(orc):
    """Conditions (symmetry, intermediate values, bounded growth) of Theorem 2.1,
    and the tail bound Q_K <= z_K + 1.25 q^{-1/2} of Corollary 2.3 (q >= 10)."""
    from scipy.special import ndtri
    for q_exp in [10, 11, 12, 13]:
        n = 2 ** q_exp
        for cons in (0, 1, 2):
            Q = orc.pwc_table(n, cons)
            assert np.allclose(Q, -Q[::-1], atol=1e-12)
            u = np.arange(n + 1) / n
            z = ndtri(u)
            assert np.all(Q[1:-1] >= z[1:-2] - 1e-12) and np.all(Q[1:-1] <= z[2:-1] + 1e-12)
            zK = z[n - 1]
            assert zK - 1e-12 <= Q[-1] <= zK + 1.25 / math.sqrt(q_exp)
        QE, QC, QI = (orc.pwc_table(n, c) for c in (0, 1, 2))
        up = slice(n // 2, n)
        assert np.all(QE[up] >= QC[up] - 1e-12) and np.all(QC[up] >= QI[up] - 1e-12)


def test_pwc_l2_error_and_rate(orc):
    """RMSE of 1024 intervals is about 1e-2 (Section 2.2 / Section 4.1), the
    closed form agrees with quadrature, and ||Q - Phi^{-1}||_p^p / (2^-q q^{-p/2})
    stays bounded as q grows (Theorem 2.1, p = 2 and 4)."""
    from numpy.polynomial.legendre import leggauss
    from scipy.special import ndtri
    from scipy.integrate import quad
    q1024 = orc.pwc_table(1024, 0)
    rmse = math.sqrt(orc.pwc_l2err2(q1024))
    assert 0.005 < rmse < 0.02
    xg, wg = leggauss(24)

    def lpp(n, p):
        Q = orc.pwc_table(n, 0)
        z = ndtri(np.arange(n + 1) / n)
        tot = 0.0
        # interior intervals in z-space: int |Q_k - z|^p phi(z) dz (Gauss-Legendre)
        a, b = z[1:-2], z[2:-1]
        Qi = Q[1:-1]
        zz = 0.5 * (b - a)[:, None] * xg[None, :] + 0.5 * (a + b)[:, None]
        f = np.abs(Qi[:, None] - zz) ** p * np.exp(-0.5 * zz ** 2) / math.sqrt(2 * math.pi)
        tot += (0.5 * (b - a) * (f * wg[None, :]).sum(axis=1)).sum()
        # the two singular end intervals by adaptive quadrature
        for k, (lo, hi) in ((0, (-np.inf, z[1])), (n - 1, (z[n - 1], np.inf))):
            tot += quad(lambda t: abs(Q[k] - t) ** p * math.exp(-0.5 * t * t) / math.sqrt(2 * math.pi),
                        lo, hi, epsabs=1e-16, limit=200)[0]
        return tot

    assert lpp(1024, 2) == pytest.approx(rmse ** 2, rel=1e-6)
    for p in (2, 4):
        ratios = [lpp(2 ** q, p) / (2.0 ** -q * q ** (-p / 2)) for q in (6, 8, 10, 12)]
        assert max(ratios) / min(ratios) < 4.0, ratios
        assert ratios[-1] <= ratios[0] * 1.5, ratios


# ---------------------------------------------------------------- PWL table
def test_pwl_listing_coefficients(orc):
    a, b = orc.pwl_table(15, 0.5)
    for idx, av, bv in _read_golden("pwl_listing_coefficients.txt"):
        i = int(idx)
        assert _trunc_sig(a[i], 2) == pytest.approx(float(av), abs=1e-9), (i, a[i])
        assert _trunc_sig(b[i], 2) == pytest.approx(float(bv), rel=1e-9, abs=1e-9), (i, b[i])


def test_pwl_singular_interval_closed_form(orc):
    """alpha = 2 phi(z_b)/b - 3 Phi(sqrt2 z_b)/(b^2 sqrt pi),
    beta = 6/b^3 (Phi(sqrt2 z_b)/sqrt pi - b phi(z_b))  (proof of Theorem 2.4)."""
    from scipy.special import ndtri, ndtr
    for K in (8, 15, 16, 20):
        a, b = orc.pwl_table(K, 0.5)
        bb = 2.0 ** -K
        zb = ndtri(bb)
        ph = math.exp(-0.5 * zb * zb) / math.sqrt(2 * math.pi)
        P2 = ndtr(math.sqrt(2) * zb)
        alpha = 2 * ph / bb - 3 * P2 / (bb * bb * math.sqrt(math.pi))
        beta = 6 / bb ** 3 * (P2 / math.sqrt(math.pi) - bb * ph)
        assert a[K] == pytest.approx(alpha, rel=1e-9)
        assert b[K] == pytest.approx(beta, rel=1e-9)
        assert b[K] == pytest.approx(-3 / (bb * zb), rel=0.35)   # beta ~ -3/(b z_b)


def test_pwl_normal_equations_mpmath(orc):
    """Coefficients solve the L2 normal equations, integrals by mpmath quadrature."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    a, b = orc.pwl_table(15, 0.5)
    finv = lambda t: -mpmath.sqrt(2) * mpmath.erfinv(1 - 2 * t)
    for k in (1, 2, 7, 14, 15):
        hi = mpmath.mpf(2) ** -k
        lo = mpmath.mpf(0) if k == 15 else hi / 2
        m0 = mpmath.quad(finv, [lo, hi])
        m1 = mpmath.quad(lambda t: t * finv(t), [lo, hi])
        s11, s12, s22 = hi - lo, (hi ** 2 - lo ** 2) / 2, (hi ** 3 - lo ** 3) / 3
        det = s11 * s22 - s12 * s12
        al = (m0 * s22 - m1 * s12) / det
        be = (s11 * m1 - s12 * m0) / det
        assert a[k] == pytest.approx(float(al), rel=1e-11), k
        assert b[k] == pytest.approx(float(be), rel=1e-11), k


def test_pwl_l2_error(orc):
    """RMSE of 15 dyadic intervals is ~1e-2 and plateaus (Section 2.3): the
    closed form agrees with quadrature, and more intervals barely help."""
    from numpy.polynomial.legendre import leggauss
    from scipy.special import ndtri
    a, b = orc.pwl_table(15, 0.5)
    e2 = orc.pwl_l2err2(a, b)
    assert 0.003 < math.sqrt(e2) < 0.02
    xg, wg = leggauss(60)
    tot = 0.0
    for k in range(1, 16):
        hi = 2.0 ** -k
        lo = 0.0 if k == 15 else hi / 2
        if k == 15:  # singular interval: integrate in z-space
            zl, zh = -40.0, ndtri(hi)
            zz = 0.5 * (zh - zl) * xg + 0.5 * (zh + zl)
            from scipy.special import ndtr
            uu = ndtr(zz)
            f = (a[k] + b[k] * uu - zz) ** 2 * np.exp(-0.5 * zz ** 2) / math.sqrt(2 * math.pi)
            tot += 0.5 * (zh - zl) * (f * wg).sum()
        else:
            uu = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
            f = (a[k] + b[k] * uu - ndtri(uu)) ** 2
            tot += 0.5 * (hi - lo) * (f * wg).sum()
    assert 2 * tot == pytest.approx(e2, rel=1e-5)
    e_inf = orc.pwl_l2err2(*orc.pwl_table(40, 0.5))
    prev = None
    for K in range(4, 25):
        eK = orc.pwl_l2err2(*orc.pwl_table(K, 0.5))
        assert eK >= e_inf - 1e-15
        assert eK - e_inf <= 2.0 ** -(K - 1)          # tail term o(r^{K-1})
        if prev is not None:
            assert eK <= prev + 1e-15
        prev = eK
    assert math.sqrt(orc.pwl_l2err2(*orc.pwl_table(16, 0.5))) == pytest.approx(math.sqrt(e2), rel=0.01)


def test_pwl_rate_in_r(orc):
    """Central term O((1-r)^{2p}) of Theorem 2.4 for p = 2: with the tail made
    negligible, log ||D-Phi^{-1}||_2^2 against log(1-r) has slope ~4."""
    rs = [0.7, 0.8, 0.9]
    errs = []
    for r in rs:
        K = int(math.ceil(math.log(1e-13) / math.log(r))) + 1
        errs.append(orc.pwl_l2err2(*orc.pwl_table(K, r), r=r))
    slope = np.polyfit(np.log([1 - r for r in rs]), np.log(errs), 1)[0]
    assert 3.3 < slope < 4.7, (slope, errs)


def test_pwl_peano_bound(orc):
    """max_a -6 a^2 (Phi^{-1})''(a) ~ 2.59 at a ~ 0.177, with
    (Phi^{-1})''(u) = z / phi(z)^2, and the pointwise error on the
    non-singular dyadic intervals stays below 2.59 ((1-r)/r)^2."""
    a_grid = np.linspace(0.05, 0.45, 40001)
    z = np.array([orc.phiinv_f64(t) for t in a_grid])
    phi = np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)
    g = -6 * a_grid ** 2 * z / phi ** 2
    i = int(np.argmax(g))
    assert g[i] == pytest.approx(2.5845, abs=2e-3)
    assert a_grid[i] == pytest.approx(0.177, abs=2e-3)
    al, be = orc.pwl_table(15, 0.5)
    for k in range(1, 15):
        hi = 2.0 ** -k
        uu = np.linspace(hi / 2, hi, 200, endpoint=False)
        err = np.abs(al[k] + be[k] * uu - np.array([orc.phiinv_f64(t) for t in uu]))
        assert err.max() <= 2.59


# ---------------------------------------------------------------- piecewise polynomials
def test_pwp_degree1_equals_closed_form_pwl(orc):
    """The quadrature route of the polynomial tables, at degree 1, reproduces the
    closed-form L2 lines (proof of Theorem 2.4) in the local variable s."""
    for K in (8, 15, 16):
        c, e2 = orc.pwp_table(K, 1)
        a, b = orc.pwl_table(K, 0.5)
        for k in range(1, K + 1):
            hi = 2.0 ** -k
            lo = 0.0 if k == K else hi / 2
            assert c[k, 0] == pytest.approx(a[k] + b[k] * lo, rel=1e-11, abs=1e-12)
            assert c[k, 1] == pytest.approx(b[k] * (hi - lo), rel=1e-10)
        assert e2 == pytest.approx(orc.pwl_l2err2(a, b), rel=1e-9)


def test_pwp_cubic_error_and_orthogonality(orc):
    """Piecewise cubic on 16 dyadic intervals reaches an L2 error around 1e-4,
    far below the linear plateau ~1e-2 (Section 2.3, Fig. 2 discussion); the
    residual is orthogonal to 1, s, s^2, s^3 on every interval (independent
    adaptive quadrature)."""
    from scipy.integrate import quad
    from scipy.special import ndtri
    c16, e16 = orc.pwp_table(16, 3)
    l16 = orc.pwl_l2err2(*orc.pwl_table(16, 0.5))
    assert 5e-5 < math.sqrt(e16) < 5e-4
    assert math.sqrt(l16) / math.sqrt(e16) > 10
    c, _ = orc.pwp_table(15, 3)
    for k in (1, 5, 14):
        hi = 2.0 ** -k
        lo = hi / 2
        for j in range(4):
            f = lambda u: ((u - lo) / (hi - lo)) ** j * (ndtri(u) - np.polyval(c[k, ::-1], (u - lo) / (hi - lo)))
            val = quad(f, lo, hi, epsabs=1e-16, epsrel=1e-12, limit=200)[0]
            assert abs(val) < 1e-12 * (hi - lo) * 10, (k, j, val)


def test_pwp_sampler_bruteforce(orc):
    """Grid uniforms near every interval edge: the sampler evaluates the cubic
    of the interval containing min(u, 1-u) in its local variable, with the sign
    restored (Algorithm 1 with Horner's rule)."""
    c, _ = orc.pwp_table(15, 3)
    c32 = c.astype(np.float32)
    ks = []
    for k in range(1, 24):
        m = int(2 ** 24 * 2.0 ** -k)
        for d in (-3, -1, 1, 3):
            if 0 < m + d < 2 ** 24 and (m + d) % 2:
                ks += [m + d, 2 ** 24 - (m + d)]
    u = (np.array(ks) * 2.0 ** -24).astype(np.float32)
    z = orc.sample_pwp(c32, u)
    ud = u.astype(np.float64)
    v = np.where(ud < 0.5, ud, 1 - ud)
    _, ex = np.frexp(v)
    k = np.minimum(-ex, 15)
    b = 2.0 ** -k
    s = np.where(k < 15, (v - b / 2) / (b / 2), v / b)
    want = sum(c32[k, j].astype(np.float64) * s ** j for j in range(4))
    assert np.allclose(z, np.where(ud < 0.5, want, -want), rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- samplers
def test_samplers_bruteforce_grid(orc):
    """Every point of the uniform grid near every interval edge: the PWL index
    equals ceil(-log2 v) - 1 capped at 15 (Section 3.3), the PWC index equals
    floor(N u) (Section 3.2), and values are the table formulas."""
    a, b = orc.pwl_table(15, 0.5)
    a32, b32 = a.astype(np.float32), b.astype(np.float32)
    q32 = orc.pwc_table(1024, 0).astype(np.float32)
    edges = [2.0 ** -k for k in range(1, 24)] + [m / 1024 for m in range(1025)]
    ks = set()
    for e in edges:
        c = int(round(e * 2 ** 24))
        for d in range(-7, 8, 2):
            m = c + d
            if 0 < m < 2 ** 24 and m % 2 == 1:
                ks.add(m)
                ks.add(2 ** 24 - m)
    m = np.array(sorted(ks), dtype=np.int64)
    u = (m * 2.0 ** -24).astype(np.float32)
    z, idx = orc.sample_pwl(a32, b32, u)
    ud = u.astype(np.float64)
    v = np.where(ud < 0.5, ud, 1.0 - ud)
    _, ex = np.frexp(v)                       # v = f 2^ex, f in [1/2, 1)
    want_idx = np.minimum(-ex, 15)            # ceil(-log2 v) - 1 for v in (0, 1/2]
    want_idx = np.where(v == 0.5, 0, want_idx)
    assert np.array_equal(idx, want_idx)
    zz = a32[want_idx].astype(np.float64) + b32[want_idx].astype(np.float64) * v
    assert np.array_equal(z, np.where(ud < 0.5, zz, -zz))
    zc, ic = orc.sample_pwc(q32, u)
    assert np.array_equal(ic, np.minimum(np.floor(ud * 1024).astype(np.int64), 1023))
    assert np.array_equal(zc, q32[ic].astype(np.float64))


def test_samplers_edge_cases(orc):
    a, b = orc.pwl_table(15, 0.5)
    a32, b32 = a.astype(np.float32), b.astype(np.float32)
    u = np.array([0.5, 0.0, 1.0, np.nan, -0.25, 1.5, 2.0 ** -140], dtype=np.float32)
    z, idx = orc.sample_pwl(a32, b32, u)
    assert z[0] == 0.0 and math.copysign(1.0, z[0]) == -1.0    # u = 1/2 -> -0
    assert z[1] == a32[15] and z[2] == -a32[15]
    assert np.isnan(z[3]) and np.isnan(z[4]) and np.isnan(z[5])
    assert idx[6] == 15
    q32 = orc.pwc_table(1024, 0).astype(np.float32)
    zc, ic = orc.sample_pwc(q32, u)
    assert list(ic[:3]) == [512, 0, 1023] and np.isnan(zc[3:6]).all()


def test_pwc_exact_discrete_law(orc):
    """On the 2^23-point grid every PWC value has probability exactly 1/N, so the
    sampled distribution is the discrete law of Q (Section 2.2)."""
    k = np.arange(1 << 23, dtype=np.int64)
    u = ((2 * k + 1) * 2.0 ** -24).astype(np.float32)
    q32 = orc.pwc_table(1024, 0).astype(np.float32)
    _, ic = orc.sample_pwc(q32, u)
    assert np.array_equal(np.bincount(ic, minlength=1024), np.full(1024, 8192))


# ---------------------------------------------------------------- MLMC
def _gbm(orc, payoff, scheme=0, approx=0):
    return orc.sde_params(model=orc.MODEL_GBM, scheme=scheme, payoff=payoff, approx=approx,
                          X0=1.0, T=1.0, K=1.0, mu=0.05, sigma=0.2, discount=1.0)


def test_mlmc_em_exact_moments(orc):
    """E[X_N] = X0 (1 + mu dt)^N for exact and approximate variates (both have
    zero mean), and E[X_N^2] = ((1 + mu dt)^2 + sigma^2 dt E[Z^2])^N  (Section 4)."""
    a, b = orc.pwl_table(15, 0.5)
    tab = (a, b)
    # E[Z~^2] = int D^2 = 2 sum_k int_{I_k} (alpha + beta u)^2 du
    sq = 0.0
    for k in range(1, 16):
        hi = 2.0 ** -k
        lo = 0.0 if k == 15 else hi / 2
        sq += a[k] ** 2 * (hi - lo) + a[k] * b[k] * (hi * hi - lo * lo) + b[k] ** 2 * (hi ** 3 - lo ** 3) / 3
    EZ2a = 2 * sq
    prm = _gbm(orc, orc.PAYOFF_X)
    n = 40000
    for level in (0, 3):
        N = 2 ** level
        dt = 1.0 / N
        for kind, ez2 in ((orc.KIND_PLAIN, 1.0), (orc.KIND_PLAIN_APPROX, EZ2a)):
            y = orc.mlmc_paths(prm, tab, level, kind, n, seed=11, tag=7)
            m1 = (1 + 0.05 * dt) ** N
            m2 = ((1 + 0.05 * dt) ** 2 + 0.04 * dt * ez2) ** N
            se1 = y.std() / math.sqrt(n)
            se2 = (y ** 2).std() / math.sqrt(n)
            assert abs(y.mean() - m1) < 4.5 * se1
            assert abs((y ** 2).mean() - m2) < 4.5 * se2


def _pwl_even_moments(a, b, K=15):
    """E[D(U)^k] for k = 0..6 of the piecewise-linear approximation on (0, 1):
    D is odd about 1/2, so odd moments vanish and the even ones are twice the
    integrals of (alpha_k + beta_k u)^k over the lower-half intervals."""
    m = np.zeros(7)
    for k in range(1, K + 1):
        hi = 2.0 ** -k
        lo = 0.0 if k == K else hi / 2
        line = np.polynomial.Polynomial([a[k], b[k]])
        for p in (2, 4, 6):
            F = (line ** p).integ()
            m[p] += 2 * (F(hi) - F(lo))
    m[0] = 1.0
    return m


def _milstein_factor_moments(mu, sigma, h, mz):
    """E[f^k], k = 1..3, of the GBM Milstein step factor f = A + B Z + C Z^2
    (A = 1 + mu h - sigma^2 h / 2, B = sigma sqrt(h), C = sigma^2 h / 2), from
    the moments mz[0..6] of Z (Section 4, Fig. 3b: X' = X f)."""
    A, B, C = 1 + mu * h - 0.5 * sigma ** 2 * h, sigma * math.sqrt(h), 0.5 * sigma ** 2 * h
    f = np.polynomial.Polynomial([A, B, C])
    out = []
    for k in (1, 2, 3):
        coef = (f ** k).coef
        out.append(sum(c * mz[j] for j, c in enumerate(coef)))
    return out


def test_mlmc_milstein_gbm_moments(orc):
    """GBM Milstein with P(X) = X: the step factors are independent, so
    E[X_N^k] = X0^k (E f^k)^N.  For exact variates E f = 1 + mu h and
    E f^2 = (1 + mu h)^2 + sigma^2 h + sigma^4 h^2 / 2; for the approximate ones
    the moments of D enter through the same polynomial.  sigma = 0.5 makes the
    Milstein term large enough that a wrong sign or factor in it (both change
    E f^2 or E f^3 by 10-20 standard errors here) fails the test."""
    a, b = orc.pwl_table(15, 0.5)
    mz_exact = np.array([1.0, 0.0, 1.0, 0.0, 3.0, 0.0, 15.0])
    mz_pwl = _pwl_even_moments(a, b)
    mu, sigma = 0.05, 0.5
    # the expansion reproduces the closed forms for the exact Gaussian
    for h in (1.0, 0.125):
        e1, e2, _ = _milstein_factor_moments(mu, sigma, h, mz_exact)
        assert e1 == pytest.approx(1 + mu * h, rel=1e-14)
        assert e2 == pytest.approx((1 + mu * h) ** 2 + sigma ** 2 * h + sigma ** 4 * h * h / 2, rel=1e-14)
    prm = orc.sde_params(model=orc.MODEL_GBM, scheme=orc.SCHEME_MILSTEIN, payoff=orc.PAYOFF_X,
                         X0=1.0, T=1.0, mu=mu, sigma=sigma, discount=1.0)
    n = 40000
    for level in (0, 2):
        N = 2 ** level
        h = 1.0 / N
        for kind, mz in ((orc.KIND_PLAIN, mz_exact), (orc.KIND_PLAIN_APPROX, mz_pwl)):
            y = orc.mlmc_paths(prm, (a, b), level, kind, n, seed=13, tag=17)
            want = _milstein_factor_moments(mu, sigma, h, mz)
            for k in (1, 2, 3):
                yk = y ** k
                se = yk.std() / math.sqrt(n)
                assert abs(yk.mean() - want[k - 1] ** N) < 4.5 * se, (level, kind, k)


def test_mlmc_milstein_strong_order(orc):
    """Milstein has strong order 1, so the two-way exact variance
    V[P_l - P_(l-1)] of P(X) = X falls like h^2: slope -2 per level, against -1
    for Euler-Maruyama (Section 4, Fig. 3a/3b).  GBM with the config's
    parameters, and CIR with the Feller condition well satisfied (kappa = 0.5,
    theta = X0 = 1, sigma = 0.3), where sqrt(|X|) never meets 0 and the
    Milstein term sigma^2 (dW^2 - h) / 4 gives order 1 as well.  A wrong sign or
    factor in either Milstein term brings the slope back to about -1.  (For
    this CIR set Euler-Maruyama's order-1/2 term sigma^4 h / 8 per unit time
    is small, so at levels 2..6 its slope reads about -1.5: the test asks that
    it stay well above Milstein's.)"""
    a, b = orc.pwl_table(15, 0.5)
    gbm = dict(model=orc.MODEL_GBM, payoff=orc.PAYOFF_X, X0=1.0, T=1.0, mu=0.05, sigma=0.2, discount=1.0)
    cir = dict(model=orc.MODEL_CIR, payoff=orc.PAYOFF_X, X0=1.0, T=1.0, sigma=0.3, kappa=0.5, theta=1.0,
               discount=1.0)
    for base in (gbm, cir):
        slopes = {}
        for scheme in (orc.SCHEME_EM, orc.SCHEME_MILSTEIN):
            prm = orc.sde_params(scheme=scheme, **base)
            v = [orc.mlmc_paths(prm, (a, b), level, orc.KIND_EXACT2, 20000, seed=4, tag=3).var()
                 for level in (2, 4, 6)]
            slopes[scheme] = (math.log2(v[2]) - math.log2(v[0])) / 4
        assert -2.4 < slopes[orc.SCHEME_MILSTEIN] < -1.7, (base["model"], slopes)
        em_lo = -1.3 if base is gbm else -1.7
        assert em_lo < slopes[orc.SCHEME_EM] < -0.7, (base["model"], slopes)
        assert slopes[orc.SCHEME_EM] > slopes[orc.SCHEME_MILSTEIN] + 0.4, (base["model"], slopes)


def test_mlmc_milstein_cir_mean_exact(orc):
    """The CIR Milstein step adds sigma^2 (dW^2 - h) / 4, whose mean is zero for
    exact variates, so E[X_N] = theta + (X0 - theta)(1 - kappa h)^N as for
    Euler-Maruyama; with the approximate variates E[dW~^2] = h E[D^2], which
    moves the fixed point to theta + sigma^2 (E[D^2] - 1) / (4 kappa)."""
    a, b = orc.pwl_table(15, 0.5)
    m2 = _pwl_even_moments(a, b)[2]
    kappa, theta, sigma, X0 = 0.5, 0.04, 0.3, 0.09
    prm = orc.sde_params(model=orc.MODEL_CIR, scheme=orc.SCHEME_MILSTEIN, payoff=orc.PAYOFF_X, X0=X0,
                         T=1.0, sigma=sigma, kappa=kappa, theta=theta, discount=1.0)
    for level in (2, 5):
        N = 2 ** level
        h = 1.0 / N
        for kind, th in ((orc.KIND_PLAIN, theta),
                         (orc.KIND_PLAIN_APPROX, theta + sigma ** 2 * (m2 - 1) / (4 * kappa))):
            y = orc.mlmc_paths(prm, (a, b), level, kind, 30000, seed=6, tag=10)
            want = th + (X0 - th) * (1 - kappa * h) ** N
            assert abs(y.mean() - want) < 4.5 * y.std() / math.sqrt(y.size), (level, kind)


def test_mlmc_telescoping_black_scholes(orc):
    """Nested MLMC sum over levels of APPROX2 + CORR4 means matches the
    Black-Scholes call (S0 = K = 1, r = 0.05, sigma = 0.2, T = 1) within the
    Euler-Maruyama weak bias plus sampling error (Section 4, Section 4.1)."""
    from scipy.stats import norm
    r, s = 0.05, 0.2
    d1 = (r + 0.5 * s * s) / s
    bs = norm.cdf(d1) - math.exp(-r) * norm.cdf(d1 - s)
    assert bs == pytest.approx(0.1045058357, abs=1e-9)
    a, b = orc.pwl_table(15, 0.5)
    prm = orc.sde_params(payoff=orc.PAYOFF_CALL, mu=r, sigma=s)
    est, var = 0.0, 0.0
    for level, n2, n4 in ((0, 200000, 4000), (1, 100000, 4000), (2, 60000, 4000), (3, 40000, 4000),
                          (4, 20000, 2000), (5, 10000, 2000)):
        s2 = orc.mlmc_level(prm, (a, b), level, orc.KIND_APPROX2, n2, seed=3, tag=100 + level)
        s4 = orc.mlmc_level(prm, (a, b), level, orc.KIND_CORR4, n4, seed=3, tag=200 + level)
        for (S1, S2, _, _, N) in (s2, s4):
            m = S1 / N
            est += m
            var += (S2 / N - m * m) / N
    bias_bound = 0.1045 * 2.0 ** -5 * 2   # EM weak error is O(dt); generous constant
    assert abs(est - bs) < 4 * math.sqrt(var) + bias_bound


def test_mlmc_level_power_sums(orc):
    """The level sums carry sum Y^k, k = 1..4 (Section 4.1 sample moments and
    the kurtosis).  For GBM Euler-Maruyama with P(X) = X the step factors
    f = 1 + mu h + sigma sqrt(h) Z are independent, so E[Y^k] = X0^k (E f^k)^N
    with E f^k from the Gaussian moments 1, 0, 1, 0, 3; each power sum / n
    must match within 4.5 standard errors, and a dropped or mis-indexed power
    fails.  The fourth-moment ratio of a one-step PLAIN term is the Gaussian 3
    less a small correction, which the same sums reproduce."""
    mz = np.array([1.0, 0.0, 1.0, 0.0, 3.0, 0.0, 15.0, 0.0, 105.0])
    mu, sigma = 0.05, 0.2
    prm = _gbm(orc, orc.PAYOFF_X)
    a, b = orc.pwl_table(15, 0.5)
    n = 60000
    for level in (0, 2):
        N = 2 ** level
        h = 1.0 / N
        f = np.polynomial.Polynomial([1 + mu * h, sigma * math.sqrt(h)])
        want = [sum(c * mz[j] for j, c in enumerate((f ** k).coef)) ** N for k in (1, 2, 3, 4)]
        sums = orc.mlmc_level(prm, (a, b), level, orc.KIND_PLAIN, n, seed=21, tag=5)
        y = orc.mlmc_paths(prm, (a, b), level, orc.KIND_PLAIN, n, seed=21, tag=5)   # for the SEs
        assert sums[4] == n
        for k in (1, 2, 3, 4):
            se = (y ** k).std() / math.sqrt(n)
            assert abs(sums[k - 1] / n - want[k - 1]) < 4.5 * se, (level, k, sums[k - 1] / n, want[k - 1])
    # level 0: Y = X0 f, kurtosis of f = 3 exactly (a Gaussian), from the sums
    s = orc.mlmc_level(prm, (a, b), 0, orc.KIND_PLAIN, 200000, seed=22, tag=6)
    m, e2, e3, e4 = (s[k] / s[4] for k in range(4))
    v = e2 - m * m
    kurt = (e4 - 4 * m * e3 + 6 * m * m * e2 - 3 * m ** 4) / v ** 2
    assert abs(kurt - 3.0) < 0.1, kurt


def test_mlmc_cir_mean_exact(orc):
    """Truncated Euler-Maruyama for CIR has E[X_N] = theta + (X0 - theta)(1 - kappa dt)^N
    exactly, because the noise term has zero mean given X_n."""
    prm = orc.sde_params(model=orc.MODEL_CIR, payoff=orc.PAYOFF_X, X0=0.04, T=1.0,
                         sigma=0.3, kappa=0.5, theta=0.04, discount=1.0)
    prm.X0 = 0.09
    a, b = orc.pwl_table(15, 0.5)
    for level in (2, 5):
        N = 2 ** level
        y = orc.mlmc_paths(prm, (a, b), level, orc.KIND_PLAIN, 30000, seed=5, tag=9)
        want = 0.04 + (0.09 - 0.04) * (1 - 0.5 / N) ** N
        assert abs(y.mean() - want) < 4.5 * y.std() / math.sqrt(y.size)


def test_mlmc_variance_structure(orc):
    """Fig. 3 / Table 2 shape: two-way exact variance decays ~2^-l (strong order
    1/2), the four-way variance is ~2^-13..2^-14 of it for PWC/PWL, flat in l."""
    prm_l = _gbm(orc, orc.PAYOFF_X, approx=orc.APPROX_PWL)
    prm_c = _gbm(orc, orc.PAYOFF_X, approx=orc.APPROX_PWC)
    a, b = orc.pwl_table(15, 0.5)
    q = orc.pwc_table(1024, 0)
    v2, rl, rc = [], [], []
    for level in (2, 4, 6):
        n = 20000
        y2 = orc.mlmc_paths(prm_l, (a, b), level, orc.KIND_EXACT2, n, seed=1, tag=1)
        y4 = orc.mlmc_paths(prm_l, (a, b), level, orc.KIND_CORR4, n, seed=1, tag=1)
        y4c = orc.mlmc_paths(prm_c, q, level, orc.KIND_CORR4, n, seed=1, tag=1)
        v2.append(y2.var())
        rl.append(math.log2(y4.var() / y2.var()))
        rc.append(math.log2(y4c.var() / y2.var()))
    slope = (math.log2(v2[2]) - math.log2(v2[0])) / 4
    assert -1.25 < slope < -0.75, v2
    assert all(abs(x - (-14)) < 1.5 for x in rl), rl
    assert all(abs(x - (-13)) < 2.0 for x in rc), rc
    assert max(rl) - min(rl) < 1.0 and max(rc) - min(rc) < 1.0


def test_mlmc_pwp_linear_rows_reproduce_pwl_paths(orc):
    """A degree-1 polynomial table is the piecewise linear approximation written
    in the local variable s, so coupled paths driven by it equal the PWL paths up
    to the FP32 rounding of the two coefficient sets (a wrong row, local
    variable or sign in the polynomial branch of the path code fails this)."""
    a, b = orc.pwl_table(15, 0.5)
    c1, _ = orc.pwp_table(15, 1)
    for kind in (orc.KIND_APPROX2, orc.KIND_CORR4, orc.KIND_PLAIN_APPROX):
        yl = orc.mlmc_paths(_gbm(orc, orc.PAYOFF_X, approx=orc.APPROX_PWL), (a, b), 3, kind, 3000,
                            seed=2, tag=5)
        yp = orc.mlmc_paths(_gbm(orc, orc.PAYOFF_X, approx=orc.APPROX_PWP), c1, 3, kind, 3000,
                            seed=2, tag=5)
        # the coefficient rounding moves Y by ~1e-5 of its own scale
        assert np.max(np.abs(yl - yp)) < 1e-4 * np.max(np.abs(yl)), kind
        assert np.max(np.abs(yl)) > 0


def test_mlmc_cubic_variance_drop(orc):
    """Fig. 3 / Table 6, with the variance predicted from the table's own error.

    Writing Z~ = Z - e, the first-order effect of e_n cancels between the fine
    and the coarse path (the coarse increment sums the same two variates); what
    remains is e_n sigma^2 h Z_(n+-1), so Var(four-way) ~ N delta^2 sigma^4 h^2
    = 2 delta^2 Var(two-way), delta^2 = E[e^2] the squared L2 error.  PWL (K=15)
    has delta = 6.5e-3: 2 delta^2 = 2^-13.5 (the paper's 2^-14).  For the cubic,
    the regular intervals give delta = 1.0e-4 (the paper's ~1e-4): 2^-25.6, the
    paper's 2^-25; the singular interval adds 93% of delta^2 through rare u near
    0, so the full expectation is 2^-21.7 and finite-sample estimates lie
    between the two."""
    from scipy.integrate import quad
    from scipy.special import ndtri
    c3, e2 = orc.pwp_table(15, 3)
    reg = 0.0
    for k in range(1, 15):
        hi = 2.0 ** -k
        lo = hi / 2
        reg += 2 * quad(lambda u: (ndtri(u) - np.polyval(c3[k, ::-1], (u - lo) / (hi - lo))) ** 2, lo, hi,
                        epsabs=1e-20, limit=200)[0]
    assert 0.9e-4 < math.sqrt(reg) < 1.1e-4 and reg < 0.1 * e2
    lo_pred, hi_pred = math.log2(2 * reg), math.log2(2 * e2)
    assert -26 < lo_pred < -25 and -22 < hi_pred < -21.5
    prm = _gbm(orc, orc.PAYOFF_X, approx=orc.APPROX_PWP)
    prm_l = _gbm(orc, orc.PAYOFF_X, approx=orc.APPROX_PWL)
    a, b = orc.pwl_table(15, 0.5)
    for level in (2, 3):
        n = 20000
        y2 = orc.mlmc_paths(prm, c3, level, orc.KIND_EXACT2, n, seed=1, tag=1)
        y4 = orc.mlmc_paths(prm, c3, level, orc.KIND_CORR4, n, seed=1, tag=1)
        y4l = orc.mlmc_paths(prm_l, (a, b), level, orc.KIND_CORR4, n, seed=1, tag=1)
        r = math.log2(y4.var() / y2.var())
        rl = math.log2(y4l.var() / y2.var())
        assert lo_pred - 1.5 < r < hi_pred + 1.0, (level, r)
        assert r < rl - 8, (level, r, rl)


def test_cost_model_tables(orc):
    """Table 2 and Table 6 speed-ups follow from the allocation formulas of
    Section 4.1 with C~ = c^ + c~ and v~ = v^."""
    for name, lv, cr, sp, eff, mm, mM in _read_golden("savings_tables.txt"):
        lv, cr, sp, eff, mm = float(lv), float(cr), float(sp), float(eff), float(mm)
        vhat, chat, ctil = 1.0, cr, 1.0
        Vt, Ct = 2.0 ** lv, chat + ctil
        eps = 1e-3
        That, mhat = orc.mlmc_alloc([vhat], [chat], eps)
        Ttil, mtil = orc.mlmc_alloc([vhat, Vt], [ctil, Ct], eps)
        speed = That / Ttil
        assert speed == pytest.approx(sp, abs=1.0 if cr > 100 else 0.006), name
        assert 100 * speed / cr == pytest.approx(eff, abs=0.06), name
        assert mtil[0] / mhat[0] == pytest.approx(mm, abs=0.011), name
        if mM != "nan":
            assert mtil[0] / mtil[1] == pytest.approx(float(mM), rel=0.025), name


# ---------------------------------------------------------------- NCX2
def test_gammp_against_scipy(orc):
    from scipy.special import gammainc
    for a in (0.1, 0.5, 1.0, 2.5, 10.0, 57.3, 400.0):
        for x in (1e-3, 0.3, 1.0, 3.0, 9.5, 50.0, 380.0, 500.0):
            assert orc.gammp(a, x) == pytest.approx(gammainc(a, x), rel=1e-12, abs=1e-15)


def test_ncx2_closed_forms_and_scipy(orc):
    from scipy.stats import ncx2
    for u in (1e-6, 0.1, 0.5, 0.9, 0.999999):
        # the quantile is found from F = 1 - Q, so near u -> 1 its error is
        # ~1e-16 / f(x) in absolute terms: allow that conditioning
        x = -2 * math.log1p(-u)
        cond = 1e-15 / (0.5 * math.exp(-0.5 * x))
        assert orc.ncx2_ppf(u, 2.0, 0.0) == pytest.approx(x, rel=1e-12, abs=cond)
    for nu, lam in ((0.8889, 1.37), (1.0, 10.0), (5.0, 0.5), (2.0, 113.0), (10.0, 200.0)):
        for u in (0.001, 0.2, 0.5, 0.8, 0.999):
            assert orc.ncx2_ppf(u, nu, lam) == pytest.approx(ncx2.ppf(u, nu, lam), rel=1e-8)
        for x in (0.05, 1.0, nu + lam):
            assert orc.ncx2_cdf(x, nu, lam) == pytest.approx(ncx2.cdf(x, nu, lam), rel=1e-9, abs=1e-14)


def test_ncx2_moments_by_quadrature(orc):
    """mean nu + lambda and variance 2(nu + 2 lambda) of the quantile function."""
    from numpy.polynomial.legendre import leggauss
    xg, wg = leggauss(400)
    u = 0.5 * (xg + 1)
    for nu, lam in ((1.0, 5.0), (4.0, 2.0)):
        x = np.array([orc.ncx2_ppf(t, nu, lam) for t in u])
        m = 0.5 * (wg * x).sum()
        v = 0.5 * (wg * x * x).sum() - m * m
        assert m == pytest.approx(nu + lam, rel=2e-3)
        assert v == pytest.approx(2 * (nu + 2 * lam), rel=2e-2)


def test_ncx2_P_limits(orc):
    """P_x(U; y) -> Phi^{-1}(U) as y -> 0 and -> C_x^{-1}(U)/(2 sqrt x) - sqrt(x)/2
    as y -> 1 (Section 5.1)."""
    from scipy.stats import chi2
    for u in (0.05, 0.3, 0.7, 0.95):
        assert orc.ncx2_P(u, 1.0, 1e-5) == pytest.approx(orc.phiinv_f64(u), abs=0.01)
        y1 = orc.ncx2_P(u, 3.0, 1.0 - 1e-9)
        assert y1 == pytest.approx(chi2.ppf(u, 3.0) / (2 * math.sqrt(3.0)) - math.sqrt(3.0) / 2, abs=1e-6)


def test_ncx2_upper_tail_against_scipy(orc):
    """The directly summed upper tail and its quantile match scipy's ncx2.sf /
    ncx2.isf, down to tail probabilities far below the FP64 spacing at 1."""
    from scipy.stats import ncx2
    for nu, lam in ((1.0, 1.0), (2.0, 30.0), (10.0, 224.0)):
        for v in (0.3, 1e-3, 1e-9, 1e-15, 1e-25):
            x = orc.ncx2_isf(v, nu, lam)
            assert orc.ncx2_sf(x, nu, lam) == pytest.approx(v, rel=1e-10)
            assert x == pytest.approx(ncx2.isf(v, nu, lam), rel=2e-7)
        for u in (0.2, 0.6):
            x = orc.ncx2_ppf(u, nu, lam)
            assert orc.ncx2_sf(x, nu, lam) == pytest.approx(1 - u, rel=1e-12)


def _ncx2_tables():
    out = {}
    for row in _read_golden("ncx2_rmse_table5.txt"):
        out[(int(row[0]), int(row[1]), int(row[2]))] = float(row[3])
    return out


def test_ncx2_tables_reproduce_table5(orc):
    """Section 5.1 approximation (two halves, 16 dyadic intervals per half, 16
    knots equally spaced in sqrt(y), linear interpolation in sqrt(y), L2 fits):
    its RMSE against the exact inverse reproduces the values printed in Table 5
    (a: linear, b: cubic) to their three decimals."""
    want = _ncx2_tables()
    cases = {(1, 1): (1, 10, 200), (1, 10): (5, 100), (3, 1): (1, 50, 200), (3, 10): (10, 100)}
    for (deg, nu), lams in cases.items():
        c = orc.ncx2_poly_table(nu, 16, 16, deg)
        for lam in lams:
            r = orc.ncx2_poly_rmse(c, nu, lam)
            assert abs(r - want[(deg, nu, lam)]) <= 0.0006, (deg, nu, lam, r)


def test_ncx2_table_limits(orc):
    """Knot y = 0 is the Gaussian limit: the lower half equals the L2 polynomial
    tables of Phi^{-1} on the same intervals and the upper half its negation;
    knot y = 1 is the central chi^2 limit, and the tables reproduce scipy's
    chi2 quantile there to their fit error."""
    from scipy.stats import chi2
    K, nu = 16, 4.0
    c = orc.ncx2_poly_table(nu, K, 16, 3)
    g, _ = orc.pwp_table(K, 3)
    assert np.allclose(c[0, 0, 1:], g[1:], rtol=1e-7, atol=1e-9)
    assert np.allclose(c[0, 1, 1:], -g[1:], rtol=1e-7, atol=1e-9)
    assert c[0, 0, 0, 0] == pytest.approx(0.0, abs=1e-12)
    for u in (0.01, 0.2, 0.5, 0.8, 0.99):
        want = chi2.ppf(u, nu)
        assert orc.ncx2_poly_ppf(c, nu, u, 0.0) == pytest.approx(want, abs=2e-3 * (1 + want))
    # between knots the interpolation is linear in sqrt(y)
    y0, y1 = (3 / 15) ** 2, (4 / 15) ** 2
    ym = ((3.5 / 15)) ** 2
    for u in (0.1, 0.7):
        p0, p1, pm = (orc.ncx2_poly_P(c, u, y) for y in (y0, y1, ym))
        assert pm == pytest.approx(0.5 * (p0 + p1), abs=1e-13)


# ---------------------------------------------------------------- MLP
def test_mlp_gradient_finite_differences(orc):
    rng = np.random.default_rng(4)
    H = 8
    p = {"W1": rng.normal(size=(H, 2)), "b1": rng.normal(size=H) * 0.1,
         "W2": rng.normal(size=(H, H)) / math.sqrt(H), "b2": rng.normal(size=H) * 0.1,
         "w3": rng.normal(size=H) / math.sqrt(H), "b3": np.array([0.05])}
    x = rng.normal(size=(17, 2))
    t = rng.normal(size=17)
    loss, g = orc.mlp_grad(p, x, t)
    assert loss == pytest.approx(np.mean((orc.mlp_forward(p, x) - t) ** 2), rel=1e-13)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for j in range(min(flat.size, 6)):
            old = flat[j]
            flat[j] = old + h
            lp = np.mean((orc.mlp_forward(p, x) - t) ** 2)
            flat[j] = old - h
            lm = np.mean((orc.mlp_forward(p, x) - t) ** 2)
            flat[j] = old
            assert g[name].reshape(-1)[j] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-9)
