"""Host logic of the benchmark's nested-versus-exact helper (Section 4.1's
optimal split of paths between the approximate term and the correction, from
pilot variances and timed pilot costs, with the correction's kurtosis floor),
driven by a fake term runner whose sums have known moments."""
import math

import numpy as np
import pytest


def _fake_run(terms):
    """run(kind, n, offset, tag) -> (power sums of n draws, ms): each kind has
    mean mu, variance v, fourth central moment k v^2 (third central 0) and a
    cost in ms per path."""
    calls = []

    def run(kind, n, off, tag):
        mu, v, k, ms = terms[kind]
        m2 = v + mu * mu
        m3 = mu ** 3 + 3 * mu * v
        m4 = mu ** 4 + 6 * mu * mu * v + k * v * v
        calls.append((kind, n, off))
        return np.array([n * mu, n * m2, n * m3, n * m4, n], dtype=np.float64), n * ms
    return run, calls


def test_optimal_split_and_pilots():
    import bench
    terms = {"exact": (1.0, 0.6, 3.0, 4e-4), "approx": (0.999, 0.6, 3.0, 1e-5),
             "diff": (1e-3, 0.6 * 2.0 ** -14, 3.0, 3.5e-4)}
    run, calls = _fake_run(terms)
    eps = 1e-3
    r = bench._nested_vs_exact(run, eps, n0=4096, n0c=1024)
    # exact only: the pilot plus the rest up to var / eps^2 paths
    # (the pilot variance is E[Y^2] - E[Y]^2 in FP64: one path either way)
    assert abs(r["exact"]["paths"] - math.ceil(0.6 / eps ** 2)) <= 1
    assert r["exact"]["estimate"] == pytest.approx(1.0)
    # nested: m_i = eps^-2 sqrt(V_i / C_i) sum_j sqrt(V_j C_j) (Section 4.1)
    va, ca, vc, cc = 0.6, 1e-5, 0.6 * 2.0 ** -14, 3.5e-4
    k = (math.sqrt(va * ca) + math.sqrt(vc * cc)) / eps ** 2
    na, nc = math.ceil(k * math.sqrt(va / ca)), max(1024, math.ceil(k * math.sqrt(vc / cc)))
    assert abs(r["nested"]["paths_approx"] - na) <= 1
    assert r["nested"]["paths_correction"] == nc == 1024  # the optimum is below the pilot
    assert r["nested"]["estimate"] == pytest.approx(0.999 + 1e-3)
    assert r["nested"]["rmse_est"] == pytest.approx(math.sqrt(va / na + vc / nc), rel=1e-6)
    assert r["nested"]["rmse_est"] <= eps * 1.001
    assert r["nested"]["correction_pilot_kurtosis"] == pytest.approx(3.0)
    # the correction ran its pilot only (paths 0 .. 1023), the approximate
    # term its pilot and then the rest from path 4096 on
    assert [(n, off) for kind, n, off in calls if kind == "diff"] == [(1024, 0)]
    assert [(n, off) for kind, n, off in calls if kind == "approx"] == [(4096, 0), (r["nested"]["paths_approx"] - 4096, 4096)]


def test_kurtosis_floor_raises_the_correction():
    """A heavy-tailed correction (kurtosis k) whose share f of the estimator
    variance is not negligible keeps at least (k - 1)(4 f)^2 paths, so that
    its variance estimate cannot move the RMSE by more than ~25% of its share."""
    import bench
    terms = {"exact": (1.0, 0.6, 3.0, 4e-4), "approx": (0.99, 0.6, 3.0, 1e-5),
             "diff": (1e-2, 0.6 * 2.0 ** -6, 1e6, 3.5e-4)}
    run, _ = _fake_run(terms)
    r = bench._nested_vs_exact(run, 1e-3, n0=4096, n0c=1024)
    va, ca, vc, cc = 0.6, 1e-5, 0.6 * 2.0 ** -6, 3.5e-4
    k = (math.sqrt(va * ca) + math.sqrt(vc * cc)) / 1e-6
    na, nc0 = math.ceil(k * math.sqrt(va / ca)), max(1024, math.ceil(k * math.sqrt(vc / cc)))
    share = (vc / nc0) / (va / na + vc / nc0)
    floor = math.ceil((1e6 - 1.0) * (4.0 * share) ** 2)
    assert floor > nc0
    assert abs(r["nested"]["paths_correction"] - floor) <= max(2, floor * 1e-6)
    assert r["nested"]["correction_pilot_kurtosis"] == pytest.approx(1e6, rel=1e-6)
