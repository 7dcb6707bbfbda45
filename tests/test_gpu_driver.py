"""GPU checks of the MLMC driver (Section 4.1): nested, regular and plain
estimators reach the target RMSE around the Black-Scholes price."""
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


def _bs():
    from scipy.stats import norm
    r, s = 0.05, 0.2
    d1 = (r + 0.5 * s * s) / s
    return norm.cdf(d1) - math.exp(-r) * norm.cdf(d1 - s)


@pytest.mark.parametrize("estimator", ["EST_NESTED", "EST_REGULAR", "EST_ADAPTIVE"])
def test_driver_reaches_rmse(P, estimator):
    import torch
    tl = P.table_build(P.PWL, 15)
    ws = torch.empty(P.mlmc_run_workspace_bytes(), dtype=torch.uint8, device="cuda")
    prm = P.sde_params()
    eps = 5e-4
    r = P.mlmc_run(prm, tl, eps, ws, estimator=getattr(P, estimator), seed=1)
    d = r.as_dict()
    assert d["converged"]
    assert r.variance <= eps * eps / 2 * 1.05
    assert r.bias <= eps / math.sqrt(2)
    # within 4 standard deviations of the estimator plus the bias allowance
    assert abs(r.estimate - _bs()) <= 4 * math.sqrt(r.variance) + eps / math.sqrt(2)
    if estimator == "EST_NESTED":
        # the correction terms need far fewer paths than the approximate ones
        # (per level they can tie at the pilot count)
        assert sum(lv["paths"][1] for lv in d["levels"]) < sum(lv["paths"][0] for lv in d["levels"])
        for lv in d["levels"]:
            assert lv["paths"][1] <= lv["paths"][0]


def test_driver_plain_and_reproducible(P):
    import torch
    tl = P.table_build(P.PWL, 15)
    ws = torch.empty(P.mlmc_run_workspace_bytes(), dtype=torch.uint8, device="cuda")
    prm = P.sde_params()
    eps = 1e-3
    r1 = P.mlmc_run(prm, tl, eps, ws, estimator=P.EST_PLAIN, fixed_L=5, seed=2)
    r2 = P.mlmc_run(prm, tl, eps, ws, estimator=P.EST_PLAIN, fixed_L=5, seed=2)
    assert r1.estimate == r2.estimate and r1.paths[5][0] == r2.paths[5][0]
    assert r1.variance <= eps * eps / 2 * 1.05
    # plain MC at L = 5 carries the Euler-Maruyama weak bias of level 5
    assert abs(r1.estimate - _bs()) <= 4 * math.sqrt(r1.variance) + 0.1045 * 2.0 ** -5 * 2
    with pytest.raises(P.AicdfError):
        P.mlmc_run(prm, tl, eps, ws, estimator=P.EST_PLAIN)   # plain needs fixed_L


def test_driver_sets_single_set_equals_run(P):
    """One set through the multi-set driver takes exactly the rounds of
    aicdf_mlmc_run (same tags, same allocations): bit-identical results."""
    import torch
    tl = P.table_build(P.PWL, 15)
    prm = P.sde_params()
    ws = torch.empty(max(P.mlmc_run_workspace_bytes(), P.mlmc_run_sets_workspace_bytes(1)), dtype=torch.uint8,
                     device="cuda")
    for est in (P.EST_NESTED, P.EST_REGULAR, P.EST_ADAPTIVE):
        r = P.mlmc_run(prm, tl, 5e-4, ws, estimator=est, seed=4)
        (q,) = P.mlmc_run_sets([prm], tl, 5e-4, ws, estimator=est, seed=4)
        assert q.estimate == r.estimate and q.variance == r.variance and q.L == r.L
        assert [list(q.paths[l]) for l in range(r.L + 1)] == [list(r.paths[l]) for l in range(r.L + 1)]


@pytest.mark.parametrize("table", ["PWL", "PWP3"])
def test_driver_sets_many_cir_sets(P, table):
    """64 CIR sets (truncated Euler-Maruyama, X0 = theta): E[X_T] = theta at every
    level, so each set's estimate is within 4 of its own standard deviations of
    theta; every set converges, and sets of one run use their own streams.  The
    same with the piecewise cubic table (whose rows the kernels read in v), where
    the four-way terms' variance is ~2^-20 of the two-way terms'."""
    import torch
    from paper_2012_09715_gb300 import inputs
    sw = inputs.sweep_sets(64, seed=3)
    sets = [P.sde_params(model=P.MODEL_CIR, payoff=P.PAYOFF_X, X0=float(sw["X0"][i]), T=1.0, K=0.0, mu=0.0,
                         sigma=float(sw["sigma"][i]), kappa=float(sw["kappa"][i]), theta=float(sw["theta"][i]),
                         discount=1.0) for i in range(64)]
    tl = P.table_build(P.PWL, 15) if table == "PWL" else P.table_build(P.PWP, 15, 3)
    ws = torch.empty(P.mlmc_run_sets_workspace_bytes(len(sets)), dtype=torch.uint8, device="cuda")
    eps = 1e-3
    res = P.mlmc_run_sets(sets, tl, eps, ws, estimator=P.EST_NESTED, seed=7)
    assert len(res) == 64
    ests = []
    for prm, r in zip(sets, res):
        assert r.converged
        assert r.variance <= eps * eps / 2 * 1.05
        assert abs(r.estimate - prm.theta) <= 4 * math.sqrt(r.variance) + 1e-12, (prm.theta, r.estimate)
        ests.append(r.estimate - prm.theta)
    assert len(set(ests)) == len(ests)  # no two sets share a stream
    assert res[0].launches == res[-1].launches >= 2
    if table == "PWP3":
        ratios = [r.var[l][1] / r.var[l][0] for r in res for l in range(1, r.L + 1) if r.var[l][0] > 0]
        assert np.median(ratios) < 2.0 ** -15, np.median(ratios)


def test_adaptive_keeps_the_pair_where_it_pays(P):
    """The adaptive estimator (per level the cheaper of the nested pair and the
    exact two-way term by the Section 4.1 cost model).  With the piecewise
    linear table the GBM call's four-way variance is ~2^-14 of the two-way
    one, so the nested pair stays at every level.  With the two-interval
    piecewise constant table (Z^E = +-0.80, squared L2 error 1 - 2/pi) the
    four-way variance is of the two-way one's order and the pair never pays:
    every level runs an exact two-way term on its own stream -- which is then
    the regular estimator on other streams -- and the estimate stays within
    its error of the Black-Scholes price."""
    import torch
    ws = torch.empty(P.mlmc_run_workspace_bytes(), dtype=torch.uint8, device="cuda")
    eps = 2e-4
    for table, want_exact in ((P.table_build(P.PWL, 15), False), (P.table_build(P.PWC, 2), True)):
        r = P.mlmc_run(P.sde_params(), table, eps, ws, estimator=P.EST_ADAPTIVE, seed=6)
        d = r.as_dict()
        assert r.converged and r.variance <= eps * eps / 2 * 1.05
        assert all(lv["exact_level"] == want_exact for lv in d["levels"]), d["levels"]
        for lv in d["levels"]:
            if want_exact:
                assert lv["paths"][1] == 0 and lv["paths"][0] > 0
            else:
                assert 0 < lv["paths"][1] <= lv["paths"][0]
        assert abs(r.estimate - _bs()) <= 4 * math.sqrt(r.variance) + eps / math.sqrt(2)
