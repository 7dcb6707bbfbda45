"""GPU checks of the batched persistent MLMC launch: every term's sums equal
those of the single-term level kernel (itself checked against the oracle) up
to the regrouping of FP32 chunks, are deterministic across graph replays and
schedules, and agree with the oracle within 3 standard errors."""
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


def _sets(P):
    return [P.sde_params(),  # GBM call
            P.sde_params(payoff=P.PAYOFF_X, discount=1.0, scheme=P.SCHEME_MILSTEIN),
            P.sde_params(model=P.MODEL_CIR, payoff=P.PAYOFF_X, X0=0.04, mu=0.0, sigma=0.3,
                         kappa=0.5, theta=0.04, discount=1.0),
            P.sde_params(model=P.MODEL_CIR, scheme=P.SCHEME_MILSTEIN, payoff=P.PAYOFF_CALL, X0=0.05,
                         K=0.05, mu=0.0, sigma=0.2, kappa=1.5, theta=0.06, discount=1.0)]


def _terms(P):
    terms = []
    rng = np.random.default_rng(1)
    for s in range(4):
        for level in range(0, 8):
            for kind in range(5):
                n = int(rng.integers(1, 60000))
                terms.append(P.BatchTerm(s, level, kind, 1000 + 37 * s + 5 * level + kind, n,
                                         int(rng.integers(0, 1 << 20))))
    return terms


def _level_sums(P, prm, table, t, ws, sums, seed):
    P.mlmc_level(prm, table, t.level, t.kind, t.n_paths, sums, ws, path_offset=t.path_offset,
                 seed=seed, tag=t.tag)
    return sums.cpu().numpy().copy()


@pytest.mark.parametrize("method", ["PWL", "PWC"])
def test_batch_matches_level_kernel(P, method):
    import torch
    table = P.table_build(getattr(P, method), 15 if method == "PWL" else 1024)
    sets, terms = _sets(P), _terms(P)
    b = P.Batch(sets, terms, table, seed=3)
    sums = torch.zeros(P.SUMS * len(terms), dtype=torch.float64, device="cuda")
    sched = P.Schedule(2048, 128, 0, 0)
    ws = torch.empty(b.workspace_bytes(sched), dtype=torch.uint8, device="cuda")
    b.run(sched, sums, ws)
    got = sums.cpu().numpy().reshape(-1, P.SUMS)
    lws = torch.empty(P.mlmc_level_workspace_bytes(), dtype=torch.uint8, device="cuda")
    ls = torch.zeros(P.SUMS, dtype=torch.float64, device="cuda")
    for i, t in enumerate(terms):
        ref = _level_sums(P, sets[t.set], table, t, lws, ls, 3)
        assert got[i, 4] == t.n_paths
        scale = math.sqrt(t.n_paths * ref[1]) + 1e-30
        assert abs(got[i, 0] - ref[0]) <= 2e-6 * scale, (i, got[i], ref)
        assert got[i, 1] == pytest.approx(ref[1], rel=2e-6, abs=1e-30)
        # Y^3, Y^4: the same paths regrouped into other FP32 chunks
        assert abs(got[i, 2] - ref[2]) <= 4e-6 * math.sqrt(ref[1] * ref[3]) + 1e-30, (i, got[i], ref)
        assert got[i, 3] == pytest.approx(ref[3], rel=4e-6, abs=1e-30)


@pytest.mark.parametrize("slots", [1, 5, 9, 17, 33, 65, 129, 256, 257, 600])
def test_term_reduction_widths(P, slots):
    """The term sums come from a term's tile partials, added by P = 1 .. 32
    lanes per term (at most 8 tiles a lane) or by a block for terms of more
    than 256 tiles; the widest term of a plan sets the form.  A level-0 term
    of `slots` tiles of 256 paths (the last one ragged) beside two small terms
    must give the level kernel's sums in every form, and the same bits on a
    graph replay."""
    import torch
    table = P.table_build(P.PWL, 15)
    sets = [P.sde_params()]
    n = slots * 256 - 77
    terms = [P.BatchTerm(0, 0, P.KIND_APPROX2, 11, n, 5), P.BatchTerm(0, 0, P.KIND_CORR4, 12, 300, 7),
             P.BatchTerm(0, 3, P.KIND_APPROX2, 13, 200, 0)]
    b = P.Batch(sets, terms, table, seed=17)
    sched = P.Schedule(256, 128, 0, 0)
    sums = torch.zeros(P.SUMS * len(terms), dtype=torch.float64, device="cuda")
    ws = torch.empty(b.workspace_bytes(sched), dtype=torch.uint8, device="cuda")
    b.run(sched, sums, ws)
    got = sums.cpu().numpy().reshape(-1, P.SUMS).copy()
    b.run(sched, sums, ws)  # graph replay
    assert np.array_equal(got, sums.cpu().numpy().reshape(-1, P.SUMS))
    assert b.info(sched)[0] >= slots
    lws = torch.empty(P.mlmc_level_workspace_bytes(), dtype=torch.uint8, device="cuda")
    ls = torch.zeros(P.SUMS, dtype=torch.float64, device="cuda")
    for i, t in enumerate(terms):
        ref = _level_sums(P, sets[0], table, t, lws, ls, 17)
        assert got[i, 4] == t.n_paths
        scale = math.sqrt(t.n_paths * ref[1]) + 1e-30
        assert abs(got[i, 0] - ref[0]) <= 2e-6 * scale, (i, got[i], ref)
        assert got[i, 1] == pytest.approx(ref[1], rel=2e-6, abs=1e-30)
        assert abs(got[i, 2] - ref[2]) <= 4e-6 * math.sqrt(ref[1] * ref[3]) + 1e-30, (i, got[i], ref)
        assert got[i, 3] == pytest.approx(ref[3], rel=4e-6, abs=1e-30)


def test_batch_deterministic_across_replays_and_schedules(P):
    import torch
    table = P.table_build(P.PWL, 15)
    sets, terms = _sets(P), _terms(P)
    b = P.Batch(sets, terms, table, seed=9)
    sums = torch.zeros(P.SUMS * len(terms), dtype=torch.float64, device="cuda")
    res = []
    for sched in (P.Schedule(4096, 256, 0, 0), P.Schedule(4096, 256, 0, 0), P.Schedule(256, 64, 2, 0)):
        ws = torch.empty(b.workspace_bytes(sched), dtype=torch.uint8, device="cuda")
        b.run(sched, sums, ws)
        b.run(sched, sums, ws)      # graph replay
        res.append(sums.cpu().numpy().reshape(-1, P.SUMS).copy())
    assert np.array_equal(res[0], res[1])
    scale = np.sqrt(res[0][:, 4] * res[0][:, 1]) + 1e-30
    assert np.all(np.abs(res[0][:, 0] - res[2][:, 0]) <= 2e-6 * scale)


def test_batch_against_oracle(P, orc):
    import torch
    table = P.table_build(P.PWL, 15)
    a, bb = table.coefficients()
    sets = _sets(P)
    osets = [orc.sde_params(model=s.model, scheme=s.scheme, payoff=s.payoff, X0=s.X0, T=s.T, K=s.K,
                            mu=s.mu, sigma=s.sigma, kappa=s.kappa, theta=s.theta, discount=s.discount)
             for s in sets]
    terms = [P.BatchTerm(s, level, kind, 50 + s * 16 + level * 2 + (kind == 1), 4000, 123)
             for s in range(4) for level in (0, 2, 5) for kind in (0, 1)]
    b = P.Batch(sets, terms, table, seed=21)
    sums = torch.zeros(P.SUMS * len(terms), dtype=torch.float64, device="cuda")
    sched = P.Schedule(1024, 128, 0, 0)
    ws = torch.empty(b.workspace_bytes(sched), dtype=torch.uint8, device="cuda")
    b.run(sched, sums, ws)
    got = sums.cpu().numpy().reshape(-1, P.SUMS)
    for i, t in enumerate(terms):
        o = orc.mlmc_level(osets[t.set], (a, bb), t.level, t.kind, t.n_paths, path_offset=t.path_offset,
                           seed=21, tag=t.tag)
        n = t.n_paths
        se = math.sqrt(max(o[1] / n - (o[0] / n) ** 2, 0.0) / n)
        assert abs(got[i, 0] / n - o[0] / n) <= 3 * se + 1e-12, (i, got[i], o)


def test_fp16_variates_keep_the_correction_unbiased(P):
    """Rounding the approximate variates to FP16 changes the two-way term a
    little; the four-way correction absorbs it, so APPROX2 + CORR4 keeps the
    same level mean as EXACT2 (Section 4.1)."""
    import torch
    table = P.table_build(P.PWL, 15)
    sets = [P.sde_params(payoff=P.PAYOFF_X, discount=1.0)]
    level, n = 4, 1 << 21
    terms = [P.BatchTerm(0, level, P.KIND_APPROX2, 1, n, 0), P.BatchTerm(0, level, P.KIND_CORR4, 2, n, 0),
             P.BatchTerm(0, level, P.KIND_EXACT2, 3, n, 0)]
    b = P.Batch(sets, terms, table, seed=5)
    sums = torch.zeros(3 * P.SUMS, dtype=torch.float64, device="cuda")
    out = {}
    for v16 in (0, 1):
        sched = P.Schedule(8192, 256, 0, v16)
        ws = torch.empty(b.workspace_bytes(sched), dtype=torch.uint8, device="cuda")
        b.run(sched, sums, ws)
        out[v16] = sums.cpu().numpy().reshape(-1, P.SUMS).copy()
    for v16 in (0, 1):
        s = out[v16]
        m = s[:, 0] / n
        v = s[:, 1] / n - m * m
        nested, exact = m[0] + m[1], m[2]
        assert abs(nested - exact) <= 4 * math.sqrt((v[0] + v[1] + v[2]) / n)
    # FP16 rounding is visible in the correction's variance but stays small
    v4 = [out[k][1, 1] / n - (out[k][1, 0] / n) ** 2 for k in (0, 1)]
    v2 = out[0][2, 1] / n - (out[0][2, 0] / n) ** 2
    assert v4[1] >= v4[0] * 0.9 and v4[1] < v2 * 2.0 ** -8


def test_autotune_and_cache(P, tmp_path):
    import torch
    table = P.table_build(P.PWL, 15)
    sets, terms = _sets(P), _terms(P)
    b = P.Batch(sets, terms, table, seed=1)
    sums = torch.zeros(P.SUMS * len(terms), dtype=torch.float64, device="cuda")
    biggest = max(b.workspace_bytes(P.Schedule(t * m, t, 0, 0)) for t in (128, 256) for m in (2, 8, 32, 128))
    ws = torch.empty(biggest, dtype=torch.uint8, device="cuda")
    cache = str(tmp_path / "tune.txt")
    best, ms = b.autotune(sums, ws, var16=0, cache_path=cache)
    assert best.block_threads in (128, 256) and best.tile_paths % best.block_threads == 0 and ms > 0
    best2, ms2 = b.autotune(sums, ws, var16=0, cache_path=cache)   # served from the cache
    assert best2.as_dict() == best.as_dict() and ms2 == pytest.approx(ms, rel=1e-5)
    b.run(best, sums, ws)
    assert np.all(np.isfinite(sums.cpu().numpy()))


def test_full_sweep_sampled_terms(P):
    """The 4096-set sweep (CIR, truncated Euler-Maruyama, levels 0..7) at full
    size: with FP32 variates, sampled terms equal the level kernel's sums;
    in the benchmark's launch configuration (FP16 approximate variates, tiles
    of 16384 level-0 paths, 128 threads) every term keeps its count and its
    mean moves from the FP32 one by far less than its standard error (the
    same uniforms; only the variates' FP16 rounding differs)."""
    import torch
    from paper_2012_09715_gb300 import inputs
    sw = inputs.sweep_sets(4096, seed=0)
    n2, n4 = inputs.sweep_counts(sw["n_base"], levels=8)
    sets = [P.sde_params(model=P.MODEL_CIR, payoff=P.PAYOFF_X, X0=float(sw["X0"][i]), T=1.0, K=0.0,
                         mu=0.0, sigma=float(sw["sigma"][i]), kappa=float(sw["kappa"][i]),
                         theta=float(sw["theta"][i]), discount=1.0) for i in range(4096)]
    terms = []
    for s in range(4096):
        for l in range(8):
            terms.append(P.BatchTerm(s, l, P.KIND_APPROX2, 2 * (8 * s + l) + 1, int(n2[s, l]), 0))
            terms.append(P.BatchTerm(s, l, P.KIND_CORR4, 2 * (8 * s + l) + 2, int(n4[s, l]), 0))
    table = P.table_build(P.PWL, 15)
    b = P.Batch(sets, terms, table, seed=0)
    sums = torch.zeros(P.SUMS * len(terms), dtype=torch.float64, device="cuda")
    sched = P.Schedule(8192, 256, 0, 0)
    ws = torch.empty(b.workspace_bytes(sched), dtype=torch.uint8, device="cuda")
    b.run(sched, sums, ws)
    got = sums.cpu().numpy().reshape(-1, P.SUMS)
    assert np.all(np.isfinite(got)) and np.array_equal(got[:, 4], [t.n_paths for t in terms])
    lws = torch.empty(P.mlmc_level_workspace_bytes(), dtype=torch.uint8, device="cuda")
    ls = torch.zeros(P.SUMS, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(0)
    for i in rng.choice(len(terms), 24, replace=False):
        t = terms[i]
        ref = _level_sums(P, sets[t.set], table, t, lws, ls, 0)
        scale = math.sqrt(t.n_paths * ref[1]) + 1e-30
        assert abs(got[i, 0] - ref[0]) <= 2e-6 * scale
    # the level-0 two-way means estimate E[X_T]: truncated EM keeps the exact
    # mean theta + (X0 - theta)(1 - kappa dt)^N, = theta here since X0 = theta
    m0 = got[0::16, 0] / got[0::16, 4]
    assert np.all(np.abs(m0 - sw["theta"]) < 6 * sw["sigma"] * np.sqrt(sw["theta"] / got[0::16, 4]) + 1e-6)
    # the benchmark's launch configuration
    s16 = P.Schedule(16384, 128, 0, 1)
    ws16 = torch.empty(b.workspace_bytes(s16), dtype=torch.uint8, device="cuda")
    b.run(s16, sums, ws16)
    g16 = sums.cpu().numpy().reshape(-1, P.SUMS)
    assert np.all(np.isfinite(g16)) and np.array_equal(g16[:, 4], got[:, 4])
    n = got[:, 4]
    se = np.sqrt(np.maximum(got[:, 1] / n - (got[:, 0] / n) ** 2, 0.0) / n)
    se16 = np.sqrt(np.maximum(g16[:, 1] / n - (g16[:, 0] / n) ** 2, 0.0) / n)
    d = np.abs(g16[:, 0] / n - got[:, 0] / n)
    # two-way terms: the rounding moves a path's Y by ~2^-11 of its size
    assert np.all(d[0::2] <= 0.5 * se[0::2] + 1e-12)
    # four-way terms: Y is itself the small gap between exact and approximate
    # paths, which the rounding changes by a comparable amount (it raises
    # their variance); their means still agree within the two estimates' errors
    assert np.all(d[1::2] <= 6.0 * (se[1::2] + se16[1::2]) + 1e-12)
