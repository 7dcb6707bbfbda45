"""GPU parity of the fused MLMC level kernel against the CPU oracle.

* Per path: a call with n_paths = 1 returns that path's Y; it must match the
  oracle's FP64 path to within the FP32 rounding the kernel's path arithmetic
  can accumulate: each fine step rounds the state multiplier and the product
  (<= ~1.2e-7 relative), the kind combines up to 4 paths, so
  |dY| <= 4 * (2^l + 2) * 2^-23 * S, S the scale of the state.
* Level sums: within 3 standard errors of the oracle's sums on the same paths
  (the estimator contract), and far tighter in practice.
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
def env(P):
    import torch
    tl = P.table_build(P.PWL, 15)
    tc = P.table_build(P.PWC, 1024)
    ws = torch.empty(P.mlmc_level_workspace_bytes(), dtype=torch.uint8, device="cuda")
    sums = torch.zeros(P.SUMS, dtype=torch.float64, device="cuda")
    a, b = tl.coefficients()
    q = tc.coefficients()[0]
    return dict(tl=tl, tc=tc, ws=ws, sums=sums, pwl=(a, b), pwc=q)


MODELS = {
    "gbm_call": dict(model=0, payoff=1, X0=1.0, T=1.0, K=1.0, mu=0.05, sigma=0.2),
    "gbm_x": dict(model=0, payoff=0, X0=1.0, T=1.0, K=1.0, mu=0.05, sigma=0.2, discount=1.0),
    "cir_x": dict(model=1, payoff=0, X0=0.04, T=1.0, K=0.0, mu=0.0, sigma=0.3, kappa=0.5,
                  theta=0.04, discount=1.0),
}


def _params(P, orc, name, scheme, approx):
    kw = dict(MODELS[name])
    gp = P.sde_params(scheme=scheme, **kw)
    op = orc.sde_params(scheme=scheme, approx=approx, **kw)
    return gp, op


def _level(P, env, gp, table, level, kind, n, off=0, seed=0, tag=1):
    P.mlmc_level(gp, table, level, kind, n, env["sums"], env["ws"], path_offset=off, seed=seed, tag=tag)
    return env["sums"].cpu().numpy().copy()


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("approx", ["pwl", "pwc"])
def test_per_path_parity(P, orc, env, name, scheme, approx):
    oap = orc.APPROX_PWL if approx == "pwl" else orc.APPROX_PWC
    gp, op = _params(P, orc, name, scheme, oap)
    table = env["tl"] if approx == "pwl" else env["tc"]
    otab = env["pwl"] if approx == "pwl" else env["pwc"]
    S = 2.0 * max(MODELS[name]["X0"], 1.0 if MODELS[name]["model"] == 0 else 0.2)
    for level in (0, 1, 2, 5):
        tol = 4 * (2 ** level + 2) * 2.0 ** -23 * S
        for kind in range(5):
            for p in (0, 1, 31, 1000, 123456789):
                y = _level(P, env, gp, table, level, kind, 1, off=p, seed=17, tag=kind + 1)[0]
                yr = orc.mlmc_paths(op, otab, level, kind, 1, path_offset=p, seed=17, tag=kind + 1)[0]
                assert abs(y - yr) <= tol, (name, scheme, approx, level, kind, p, y, yr)


@pytest.mark.parametrize("level", [0, 3, 6])
@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_level_sums_within_3se(P, orc, env, level, kind):
    gp, op = _params(P, orc, "gbm_call", 0, orc.APPROX_PWL)
    n = 20000 if level < 6 else 5000
    g = _level(P, env, gp, env["tl"], level, kind, n, off=777, seed=4, tag=9)
    o = orc.mlmc_level(op, env["pwl"], level, kind, n, path_offset=777, seed=4, tag=9)
    assert g[4] == n
    var = max(o[1] / n - (o[0] / n) ** 2, 0.0)
    se = math.sqrt(var / n)
    assert abs(g[0] / n - o[0] / n) <= 3 * se + 1e-12
    # same paths, same uniforms: the sums agree far inside the statistical band
    assert abs(g[0] - o[0]) <= 1e-4 * (abs(o[0]) + math.sqrt(o[1] * n)) + 1e-9
    # per path, FP32 rounding adds up like a random walk over the 2^l + 2 steps
    # (each <= 2^-24 of the path scale S = 2); an error d_i moves sum Y^2 by
    # 2 Y_i d_i, which sums to about 2 sqrt(sum Y^2) |d|.  For the four-way
    # terms |Y| is itself small, so this, not a fraction of sum Y^2, sets the band.
    d = math.sqrt(2 ** level + 2) * 2.0 ** -24 * 2.0
    assert abs(g[1] - o[1]) <= 1e-4 * o[1] + 8 * math.sqrt(o[1]) * d + 1e-12
    # sum Y^3 and sum Y^4: a per-path error of at most D (the per-path parity
    # bound) moves y^3 by <= 3 y^2 D + 3 |y| D^2 + D^3 and y^4 by <= 4 |y|^3 D +
    # 6 y^2 D^2 + ..., with sum |y|^3 <= sqrt(sum y^2 sum y^4); the FP32
    # running sums add at most (paths per thread) 2^-24 of sum |y|^k (one or
    # two paths per thread here)
    D = 4 * (2 ** level + 2) * 2.0 ** -23 * 2.0
    abs3 = math.sqrt(o[1] * o[3])
    assert abs(g[2] - o[2]) <= 1e-5 * abs3 + 3 * D * o[1] + 3 * D * D * math.sqrt(n * o[1]) + n * D ** 3 + 1e-30
    assert abs(g[3] - o[3]) <= 1e-5 * o[3] + 4 * D * abs3 + 7 * D * D * o[1] + 1e-30


def test_determinism_and_additivity(P, orc, env):
    gp, _ = _params(P, orc, "gbm_call", 0, orc.APPROX_PWL)
    n = 3_000_001
    s1 = _level(P, env, gp, env["tl"], 4, 1, n, seed=8, tag=2)
    s2 = _level(P, env, gp, env["tl"], 4, 1, n, seed=8, tag=2)
    assert np.array_equal(s1, s2)                     # bit-identical reruns
    parts = [(0, 1_000_000), (1_000_000, 1_234_567), (2_234_567, 765_434)]
    tot = np.zeros(P.SUMS)
    for off, m in parts:
        tot += _level(P, env, gp, env["tl"], 4, 1, m, off=off, seed=8, tag=2)
    assert tot[4] == n
    # a different split regroups the per-thread FP32 chunks: the sums agree to
    # the chunk rounding, ~1e-6 of sum |Y| <= 1e-6 sqrt(n sum Y^2)
    scale = math.sqrt(n * s1[1])
    assert abs(tot[0] - s1[0]) <= 1e-6 * scale
    assert tot[1] == pytest.approx(s1[1], rel=1e-6)


def test_full_size_gbm_config(P, orc, env):
    """The nested-MLMC workload of the benchmark (GBM call, levels 0..8,
    N_l = round(10^(7 - 3l/8))): sampled paths equal the oracle's, and the
    estimate of the call price agrees with Black-Scholes within 3 SE + the
    Euler-Maruyama weak bias at level 8."""
    from scipy.stats import norm
    gp, op = _params(P, orc, "gbm_call", 0, orc.APPROX_PWL)
    est, var = 0.0, 0.0
    for level in range(9):
        n = int(round(10 ** (7 - 3 * level / 8)))
        for kind, tag in ((0, 100 + level), (1, 200 + level)):
            s = _level(P, env, gp, env["tl"], level, kind, n, seed=0, tag=tag)
            m = s[0] / n
            est += m
            var += (s[1] / n - m * m) / n
        for p in (0, n // 2, n - 1):
            y = _level(P, env, gp, env["tl"], level, 1, 1, off=p, seed=0, tag=200 + level)[0]
            yr = orc.mlmc_paths(op, env["pwl"], level, 1, 1, path_offset=p, seed=0, tag=200 + level)[0]
            assert abs(y - yr) <= 4 * (2 ** level + 2) * 2.0 ** -23 * 2.0
    r, s = 0.05, 0.2
    d1 = (r + 0.5 * s * s) / s
    bs = norm.cdf(d1) - math.exp(-r) * norm.cdf(d1 - s)
    assert abs(est - bs) <= 3 * math.sqrt(var) + 0.1045 * 2.0 ** -8 * 2


def test_variance_reduction_of_correction(P, orc, env):
    """Four-way variance / two-way exact variance ~ 2^-14 (PWL) and ~2^-13
    (PWC) for P(X) = X (Section 4.1, Table 2), measured on the GPU."""
    gp, _ = _params(P, orc, "gbm_x", 0, orc.APPROX_PWL)
    for table, want in ((env["tl"], -14), (env["tc"], -13)):
        for level in (3, 6):
            n = 400000
            s2 = _level(P, env, gp, table, level, 2, n, seed=6, tag=1)
            s4 = _level(P, env, gp, table, level, 1, n, seed=6, tag=1)
            v2 = s2[1] / n - (s2[0] / n) ** 2
            v4 = s4[1] / n - (s4[0] / n) ** 2
            assert abs(math.log2(v4 / v2) - want) < 2.0, (level, math.log2(v4 / v2))
