"""GPU checks of the MLMC driver (Section 4.1): nested, regular and plain
estimators reach the target RMSE around the Black-Scholes price."""
import math

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


@pytest.mark.parametrize("estimator", ["EST_NESTED", "EST_REGULAR"])
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
