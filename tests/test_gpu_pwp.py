"""GPU parity of the piecewise polynomial (degree 1..3) method against the oracle.

Tolerance: the oracle evaluates each row's FP32 coefficients c_j in its local
variable s (|s| <= 1) in FP64.  The GPU evaluates the same polynomial written
in v, d_j = alpha^j sum_{i>=j} C(i, j) beta^(i-j) c_i (s = alpha v + beta; the
d_j formed in FP64 and rounded once to FP32), by Horner's rule with three
FMAs: the rounding of the d_j and of each FMA is at most ~3 * 2^-24 *
sum_j |d_j| v^j.  The test allows 4 * 2^-24 * (sum_j |c_j| + sum_j |d_j| v^j)
plus 2 ulp of the result.  MLMC paths use the per-path bound of the
level-kernel tests.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_2012_09715_gb300 import build as b
    b.build()
    import paper_2012_09715_gb300 as P
    P.lib()
    return P


@pytest.fixture(scope="module")
def tables(P):
    out = {}
    for K in (8, 15):
        for deg in (1, 2, 3):
            t = P.table_build(P.PWP, K, deg)
            out[(K, deg)] = (t, t.coefficients()[0].astype(np.float32))
    return out


def _gpu(P, table, n, seed=0, offset=0, u=None, dtype="f32"):
    import torch
    tdt = torch.float32 if dtype == "f32" else torch.float16
    out = torch.full((n,), float("nan"), dtype=tdt, device="cuda")
    uu = None if u is None else torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda()
    P.sample(table, P.PWP, out, u=uu, seed=seed, offset=offset, n=n)
    torch.cuda.synchronize()
    return out.float().cpu().numpy().astype(np.float64)


def _rows_in_v(c32):
    """Each row's coefficients in v (FP64): s = alpha v + beta."""
    K = c32.shape[0] - 1
    c = c32.astype(np.float64)
    d = np.zeros_like(c)
    for r in range(K + 1):
        alpha, beta = (2.0 ** K, 0.0) if r == K else (2.0 ** (r + 1), -1.0)
        for j in range(4):
            d[r, j] = alpha ** j * sum(math.comb(i, j) * beta ** (i - j) * c[r, i] for i in range(j, 4))
    return d


def _row_bound(c32, u):
    """4 * 2^-24 * (sum_j |c_j| + sum_j |d_j| v^j) of the row each u falls in
    (oracle row rule)."""
    ud = u.astype(np.float64)
    v = np.where(ud < 0.5, ud, 1.0 - ud)
    K = c32.shape[0] - 1
    with np.errstate(divide="ignore", invalid="ignore"):
        _, ex = np.frexp(np.where(np.isfinite(v) & (v > 0), v, 0.25))
    k = np.where(v >= 0.5, 0, np.minimum(-ex, K))
    k = np.where(np.isfinite(v) & (v > 0), k, K)
    vv = np.where(np.isfinite(v), np.abs(v), 0.0)
    d = np.abs(_rows_in_v(c32))[k]
    dv = d[:, 0] + vv * (d[:, 1] + vv * (d[:, 2] + vv * d[:, 3]))
    return 4 * 2.0 ** -24 * (np.abs(c32.astype(np.float64)).sum(axis=1)[k] + dv)


def _assert_close(z, ref, bound):
    both_nan = np.isnan(z) & np.isnan(ref)
    tol = bound + 2 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    ok = both_nan | (np.abs(z - ref) <= tol)
    assert ok.all(), (np.flatnonzero(~ok)[:5], z[~ok][:5], ref[~ok][:5])


@pytest.mark.parametrize("K,deg", [(15, 3), (15, 1), (15, 2), (8, 3)])
@pytest.mark.parametrize("n,offset", [(1, 0), (5, 6), (4097, 8), ((1 << 20) + 13, 0)])
def test_pwp_philox_parity(P, tables, orc, K, deg, n, offset):
    t, c32 = tables[(K, deg)]
    u = orc.uniforms(seed=21, offset=offset, n=n)
    ref = orc.sample_pwp(c32, u)
    z = _gpu(P, t, n, seed=21, offset=offset)
    _assert_close(z, ref, _row_bound(c32, u))


def test_pwp_f16_output(P, tables, orc):
    t, c32 = tables[(15, 3)]
    n = 40003
    u = orc.uniforms(seed=3, offset=0, n=n)
    ref = orc.sample_pwp(c32, u)
    z = _gpu(P, t, n, seed=3, dtype="f16")
    r16 = ref.astype(np.float32).astype(np.float16).astype(np.float64)
    # one FP16 spacing, widened by the FP32 evaluation's own bound (which
    # matters only near z = 0, where FP16's spacing is finest)
    tol = np.spacing(np.abs(r16).astype(np.float16)).astype(np.float64) + _row_bound(c32, u)
    assert np.all(np.abs(z - r16) <= tol)


def _edge_uniforms():
    tiny = [1e-45, 1e-40, 1.2e-38, 1e-30, 1e-12, 1.7e-8, 2.0 ** -25, 2.0 ** -24, 3e-8, 1e-7]
    specials = [0.0, 1.0, 0.5, np.nan, -0.25, 1.5, -0.0, np.inf,
                np.nextafter(np.float32(0.5), np.float32(0)), np.nextafter(np.float32(0.5), np.float32(1)),
                1.0 - 2.0 ** -24, 0.25, 0.75]
    edges = []
    for k in range(1, 25):
        e = np.float32(2.0 ** -k)
        edges += [e, np.nextafter(e, np.float32(0)), np.nextafter(e, np.float32(1)), np.float32(1) - e]
    rng = np.random.default_rng(5)
    rand = rng.random(5000).astype(np.float32)
    logu = (10.0 ** -rng.uniform(0, 37, 2000)).astype(np.float32)
    return np.concatenate([np.array(tiny + specials, dtype=np.float32), np.array(edges, dtype=np.float32),
                           rand, logu, 1 - logu]).astype(np.float32)


@pytest.mark.parametrize("K,deg", [(15, 3), (8, 2)])
def test_pwp_input_mode_edge_cases(P, tables, orc, K, deg):
    """Caller-given u: interval edges, subnormals, +-0, 1, 1/2, NaN, out of range."""
    t, c32 = tables[(K, deg)]
    u = _edge_uniforms()
    for n in (u.size, u.size - 3):
        uu = u[:n]
        ref = orc.sample_pwp(c32, uu)
        z = _gpu(P, t, n, u=uu)
        _assert_close(z, ref, _row_bound(c32, uu))
        i = int(np.flatnonzero(uu == 0.5)[0])
        assert z[i] == 0.0 and math.copysign(1.0, z[i]) == -1.0
        # -0 and +0 both take the singular row's value at s = 0
        zero = np.flatnonzero(uu == 0.0)
        assert np.all(z[zero] == np.float32(c32[K, 0]))


def test_pwp_counters_beyond_32_bits(P, tables, orc):
    t, c32 = tables[(15, 3)]
    for off in ((1 << 34) + 8, (1 << 34) - 4000):
        n = 8195
        u = orc.uniforms(seed=13, offset=off, n=n)
        ref = orc.sample_pwp(c32, u)
        _assert_close(_gpu(P, t, n, seed=13, offset=off), ref, _row_bound(c32, u))


def test_pwp_statistics(P, tables):
    """Sample mean/variance of 2^24 cubic variates against the table's own moments
    (the cubic is within 4e-4 RMS of Phi^{-1}: variance within 2e-3 of 1)."""
    import torch
    t, _ = tables[(15, 3)]
    out = torch.empty(1 << 24, dtype=torch.float32, device="cuda")
    P.sample(t, P.PWP, out, seed=99)
    x = out.double()
    assert abs(x.mean().item()) < 5 / math.sqrt(x.numel())
    assert abs(x.var().item() - 1.0) < 2e-3


# ------------------------------------------------------------------ MLMC
@pytest.fixture(scope="module")
def lvl(P):
    import torch
    ws = torch.empty(P.mlmc_level_workspace_bytes(), dtype=torch.uint8, device="cuda")
    sums = torch.zeros(P.SUMS, dtype=torch.float64, device="cuda")
    return ws, sums


def _level(P, lvl, gp, table, level, kind, n, off=0, seed=0, tag=1):
    ws, sums = lvl
    P.mlmc_level(gp, table, level, kind, n, sums, ws, path_offset=off, seed=seed, tag=tag)
    return sums.cpu().numpy().copy()


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("model", ["gbm_call", "cir_x"])
def test_pwp_mlmc_per_path(P, orc, tables, lvl, scheme, model):
    t, c32 = tables[(15, 3)]
    if model == "gbm_call":
        kw = dict(model=0, payoff=1, X0=1.0, T=1.0, K=1.0, mu=0.05, sigma=0.2)
        S = 2.0
    else:
        kw = dict(model=1, payoff=0, X0=0.04, T=1.0, K=0.0, mu=0.0, sigma=0.3, kappa=0.5, theta=0.04,
                  discount=1.0)
        S = 0.4
    gp = P.sde_params(scheme=scheme, **kw)
    op = orc.sde_params(scheme=scheme, approx=orc.APPROX_PWP, **kw)
    for level in (0, 2, 5):
        tol = 4 * (2 ** level + 2) * 2.0 ** -23 * S
        for kind in range(5):
            for p in (0, 31, 123456789):
                y = _level(P, lvl, gp, t, level, kind, 1, off=p, seed=17, tag=kind + 1)[0]
                yr = orc.mlmc_paths(op, c32, level, kind, 1, path_offset=p, seed=17, tag=kind + 1)[0]
                assert abs(y - yr) <= tol, (model, scheme, level, kind, p, y, yr)


def test_pwp_mlmc_level_sums_match_oracle(P, orc, tables, lvl):
    t, c32 = tables[(15, 3)]
    kw = dict(model=0, payoff=1, X0=1.0, T=1.0, K=1.0, mu=0.05, sigma=0.2)
    gp = P.sde_params(**kw)
    op = orc.sde_params(approx=orc.APPROX_PWP, **kw)
    for level, kind in ((0, 0), (3, 0), (3, 4)):
        n = 20000
        g = _level(P, lvl, gp, t, level, kind, n, off=777, seed=4, tag=9)
        o = orc.mlmc_level(op, c32, level, kind, n, path_offset=777, seed=4, tag=9)
        assert g[4] == n
        assert abs(g[0] - o[0]) <= 1e-4 * (abs(o[0]) + math.sqrt(o[1] * n)) + 1e-9
        assert g[1] == pytest.approx(o[1], rel=1e-4, abs=1e-12)


def test_pwp_cubic_variance_drop_on_gpu(P, tables, lvl):
    """Four-way / two-way variance for the cubic (GBM, P(X) = X, EM): far below
    the PWL value 2^-13.5 and inside [2^-27, 2^-20.5], the band between the
    regular-interval prediction 2 delta_reg^2 = 2^-25.6 (Table 6's 2^-25) and
    the full-error prediction 2 delta^2 = 2^-21.7."""
    t, _ = tables[(15, 3)]
    gp = P.sde_params(payoff=P.PAYOFF_X, discount=1.0)
    tl = P.table_build(P.PWL, 15)
    for level in (3, 6):
        n = 400000
        s2 = _level(P, lvl, gp, t, level, 2, n, seed=6, tag=1)
        s4 = _level(P, lvl, gp, t, level, 1, n, seed=6, tag=1)
        s4l = _level(P, lvl, gp, tl, level, 1, n, seed=6, tag=1)
        v2 = s2[1] / n - (s2[0] / n) ** 2
        v4 = s4[1] / n - (s4[0] / n) ** 2
        v4l = s4l[1] / n - (s4l[0] / n) ** 2
        r = math.log2(v4 / v2)
        assert -27.0 < r < -20.5, (level, r)
        assert r < math.log2(v4l / v2) - 6, (level, r)


def test_pwp_batch_matches_level_kernel(P, tables):
    import torch
    t, _ = tables[(15, 3)]
    sets = [P.sde_params(), P.sde_params(payoff=P.PAYOFF_X, discount=1.0, scheme=P.SCHEME_MILSTEIN)]
    rng = np.random.default_rng(4)
    terms = []
    for s in range(2):
        for level in range(6):
            for kind in range(5):
                terms.append(P.BatchTerm(s, level, kind, 50 + 7 * s + 3 * level + kind,
                                         int(rng.integers(1, 30000)), int(rng.integers(0, 1 << 20))))
    b = P.Batch(sets, terms, t, seed=5)
    sums = torch.zeros(P.SUMS * len(terms), dtype=torch.float64, device="cuda")
    sched = P.Schedule(2048, 128, 0, 0)
    ws = torch.empty(b.workspace_bytes(sched), dtype=torch.uint8, device="cuda")
    b.run(sched, sums, ws)
    got = sums.cpu().numpy().reshape(-1, P.SUMS)
    lws = torch.empty(P.mlmc_level_workspace_bytes(), dtype=torch.uint8, device="cuda")
    ls = torch.zeros(P.SUMS, dtype=torch.float64, device="cuda")
    for i, tm in enumerate(terms):
        P.mlmc_level(sets[tm.set], t, tm.level, tm.kind, tm.n_paths, ls, lws, path_offset=tm.path_offset,
                     seed=5, tag=tm.tag)
        ref = ls.cpu().numpy()
        assert got[i, 4] == tm.n_paths
        scale = math.sqrt(tm.n_paths * ref[1]) + 1e-30
        assert abs(got[i, 0] - ref[0]) <= 2e-6 * scale, (i, got[i], ref)
        assert got[i, 1] == pytest.approx(ref[1], rel=2e-6, abs=1e-30)
