"""GPU checks of the non-central chi-squared path (Section 5): the FP64 exact
quantile against the oracle, the BF16 tensor-core MLP forward and gradient
against the oracle's FP64 network, training, and CIR paths with exact and
learned transitions.

Tolerances:
  * exact quantile: 1e-9 relative (both FP64, independent root finders);
  * MLP: the GPU rounds W2 and the layer-1 activations to BF16 (2^-9
    relative) and uses tanh.approx; with |W2|, |w3| ~ 0.3 and 64 terms per
    dot product the output error is ~8 * 0.3 * 2^-9 per layer, so
    |dy| <= 0.03 + 0.01 |y|, and gradients agree to 5% in norm (cosine > 0.995).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NU_CFG = 4 * 0.5 * 0.04 / 0.3 ** 2  # kappa = 0.5, theta = 0.04, sigma = 0.3 -> nu = 0.8889


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_2012_09715_gb300 import build as b
    b.build()
    import paper_2012_09715_gb300 as P
    P.lib()
    return P


def _bf16(x):
    import torch
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def test_ncx2_ppf_matches_oracle(P, orc):
    import torch
    rng = np.random.default_rng(0)
    us = np.concatenate([orc.uniforms(3, 0, 300), np.array([2.0 ** -24, 1 - 2.0 ** -24, 0.5], np.float32)])
    us = us.astype(np.float32)
    for nu in (NU_CFG, 2.0, 5.0):
        lam = np.exp(rng.uniform(-4.0, 5.0, us.size))
        lam[:3] = 0.0
        u_d = torch.from_numpy(us).cuda()
        l_d = torch.from_numpy(lam).cuda()
        out = torch.zeros(us.size, dtype=torch.float64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        P.ncx2_ppf(u_d, l_d, nu, out, st)
        got = out.cpu().numpy()
        assert st.item() == 0
        ref = np.array([orc.ncx2_ppf(float(u), nu, float(l)) for u, l in zip(us, lam)])
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-300), np.max(np.abs(got / ref - 1))
        if nu == 2.0:  # lambda = 0: -2 ln(1 - u)
            assert np.allclose(got[:3], -2 * np.log1p(-us[:3].astype(np.float64)), rtol=1e-10)


@pytest.mark.parametrize("nu", [0.03, 0.1, 0.3])
def test_ncx2_ppf_small_nu(P, orc, nu):
    """Small nu (the slow-decay CIR sets): the law's spike at 0 holds a large
    share of the mass at values below 1e-20; every quantile above that agrees
    with the oracle to 1e-8 relative, and the deeper ones are 0 or agree (a
    CIR step multiplies them by c ~ 1e-2: far below the resolution of X)."""
    import torch
    rng = np.random.default_rng(4)
    us = np.concatenate([orc.uniforms(9, 0, 400), (10.0 ** -np.arange(2, 12)).astype(np.float32)]).astype(np.float32)
    lam = np.exp(rng.uniform(-7.0, 4.6, us.size))
    lam[:20] = 0.0
    out = torch.zeros(us.size, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.ncx2_ppf(torch.from_numpy(us).cuda(), torch.from_numpy(lam).cuda(), nu, out, st)
    got = out.cpu().numpy()
    ref = np.array([orc.ncx2_ppf(float(u), nu, float(l)) for u, l in zip(us, lam)])
    assert np.all(np.isfinite(got)) and np.all(got >= 0.0)
    big = ref > 1e-20
    assert big.sum() > us.size // 4
    assert np.allclose(got[big], ref[big], rtol=1e-8, atol=0.0), np.max(np.abs(got[big] / ref[big] - 1))
    assert np.all((got[~big] == 0.0) | (np.abs(got[~big] - ref[~big]) <= 1e-8 * ref[~big]) | (got[~big] <= 1e-20))
    # monotone in u at fixed lambda wherever the quantile is above 1e-20
    u_sorted = np.sort(np.concatenate([us[:50], us[-10:]]))
    l_d = torch.full((u_sorted.size,), 0.5, dtype=torch.float64, device="cuda")
    o2 = torch.zeros(u_sorted.size, dtype=torch.float64, device="cuda")
    P.ncx2_ppf(torch.from_numpy(u_sorted).cuda(), l_d, nu, o2, st)
    q = o2.cpu().numpy()
    q = q[q > 1e-20]
    assert np.all(np.diff(q) >= 0.0)


def test_ncx2_targets_match_oracle(P, orc):
    import torch
    n = 4096
    u = torch.empty(n, device="cuda")
    lam = torch.empty(n, device="cuda")
    p = torch.empty(n, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.ncx2_targets(NU_CFG, n, u, lam, p, st, seed=1, tag=5)
    torch.cuda.synchronize()
    assert st.item() == 0
    uh, lh, ph = u.cpu().numpy(), lam.cpu().numpy(), p.cpu().numpy()
    assert uh.min() >= 2.0 ** -24 and uh.max() <= 1 - 2.0 ** -24
    assert np.log(lh).min() >= -4.0 - 1e-5 and np.log(lh).max() <= 4.0 + 1e-5
    for i in range(0, n, 37):
        y = NU_CFG / (float(lh[i]) + NU_CFG)
        ref = orc.ncx2_P(float(uh[i]), NU_CFG, y)
        assert abs(ph[i] - ref) <= 1e-5 * (1 + abs(ref)), (i, ph[i], ref)


def _sqrt_y(lam, nu=NU_CFG):
    return np.sqrt(nu / (np.maximum(lam, 0.0) + nu))


def _features(u, lam, nu=NU_CFG):
    """The network's inputs as aicdf.h defines them: s(u)/3 and 2 sqrt(y) - 1."""
    v = np.minimum(u, 1 - u)
    s = np.sqrt(np.maximum(-2 * np.log(2 * v), 0.0))
    x0 = np.where(u < 0.5, -s, s) / 3.0
    x1 = 2 * _sqrt_y(lam, nu) - 1
    return np.stack([x0, x1], axis=1)


def _compose(orc, u, lam, nn, nu=NU_CFG):
    """P~ = Phi^{-1}(u) + sqrt(y) N from the network output N (oracle Phi^{-1})."""
    return orc.phiinv(np.asarray(u, dtype=np.float32)) + _sqrt_y(lam, nu) * nn


def _random_params(rng):
    p = np.zeros(4417, dtype=np.float32)
    p[0:128] = rng.uniform(-1.5, 1.5, 128)
    p[128:192] = rng.uniform(-0.5, 0.5, 64)
    p[192:4288] = rng.uniform(-0.3, 0.3, 4096)
    p[4288:4352] = rng.uniform(-0.2, 0.2, 64)
    p[4352:4416] = rng.uniform(-0.3, 0.3, 64)
    p[4416] = 0.1
    return p


def _oracle_params(p):
    q = p.astype(np.float64)
    return {"W1": q[0:128].reshape(64, 2), "b1": q[128:192], "W2": _bf16(p[192:4288]).astype(np.float64).reshape(64, 64),
            "b2": q[4288:4352], "w3": q[4352:4416], "b3": q[4416:4417]}


def test_mlp_forward_matches_oracle(P, orc):
    import torch
    rng = np.random.default_rng(1)
    s = P.Surrogate(NU_CFG, seed=0)
    p = _random_params(rng)
    s.set_params(p)
    n = 1000  # not a multiple of 32: ragged last warp
    u = orc.uniforms(7, 0, n)
    lam = np.exp(rng.uniform(-4.5, 4.5, n)).astype(np.float32)
    out = torch.zeros(n, device="cuda")
    s.eval(torch.from_numpy(u).cuda(), torch.from_numpy(lam).cuda(), out)
    got = out.cpu().numpy().astype(np.float64)
    nn = orc.mlp_forward(_oracle_params(p), _features(u.astype(np.float64), lam.astype(np.float64)))
    ref = _compose(orc, u, lam.astype(np.float64), nn)
    z = orc.phiinv(u)
    # the network's error scaled by sqrt(y), and the FP32 inverse's 1e-6 relative
    sy = _sqrt_y(lam.astype(np.float64))
    err = np.abs(got - ref)
    assert np.all(err <= sy * (0.03 + 0.01 * np.abs(nn)) + 2e-6 * np.abs(z) + 1e-6), err.max()
    assert math.sqrt(np.mean(err ** 2)) <= 0.01


def test_mlp_gradient_matches_oracle(P, orc):
    import torch
    rng = np.random.default_rng(2)
    s = P.Surrogate(NU_CFG, seed=0)
    p = _random_params(rng)
    s.set_params(p)
    n = 2048
    u = orc.uniforms(9, 0, n)
    lam = np.exp(rng.uniform(-4, 4, n)).astype(np.float32)
    tgt = rng.normal(size=n).astype(np.float32)
    g = torch.zeros(4418, device="cuda")
    s.grad(torch.from_numpy(u).cuda(), torch.from_numpy(lam).cuda(), torch.from_numpy(tgt).cuda(), g)
    got = g.cpu().numpy().astype(np.float64)
    # the network's own target g = (P - Phi^{-1}(u)) / sqrt(y) for the P targets given
    gt = (tgt.astype(np.float64) - orc.phiinv(u)) / _sqrt_y(lam.astype(np.float64))
    loss, ref = orc.mlp_grad(_oracle_params(p), _features(u.astype(np.float64), lam.astype(np.float64)), gt)
    assert got[4417] / n == pytest.approx(loss, rel=0.05)
    offs = {"W1": (0, 128), "b1": (128, 192), "W2": (192, 4288), "b2": (4288, 4352), "w3": (4352, 4416),
            "b3": (4416, 4417)}
    for name, (a, b) in offs.items():
        gv, rv = got[a:b], ref[name].reshape(-1)
        assert np.linalg.norm(gv - rv) <= 0.05 * np.linalg.norm(rv) + 1e-6, name
        if b - a > 1:
            cos = gv @ rv / (np.linalg.norm(gv) * np.linalg.norm(rv))
            assert cos > 0.995, (name, cos)


def test_scheduled_training_equals_step_by_step(P):
    """aicdf_surrogate_train (features formed once per call, the epoch's
    gradient and Adam launches replayed as one graph and chained by
    programmatic dependent launch) against the same four Adam steps taken one
    call at a time (features formed in the gradient kernel, plain launches),
    from the same initial weights at a constant step size.  The two differ only
    in how the bias corrections 1 - b^t are rounded (host against device), a
    relative 1e-6 of each step."""
    import torch
    n, b = 4 * 8192, 8192
    u, lam, p = (torch.empty(n, device="cuda") for _ in range(3))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.ncx2_targets(NU_CFG, n, u, lam, p, st, seed=21, tag=1, loglam_lo=-6.0, loglam_hi=7.0)
    s1, s2 = P.Surrogate(NU_CFG, seed=5), P.Surrogate(NU_CFG, seed=5)
    p0 = s1.get_params()
    assert np.array_equal(p0, s2.get_params())
    l1, l2 = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    s1.train(u, lam, p, batch=b, epochs=1, lr=1e-3, lr_final=1e-3, loss=l1)
    for k in range(n // b):
        s2.train_step(u[k * b:(k + 1) * b], lam[k * b:(k + 1) * b], p[k * b:(k + 1) * b], 1e-3, loss=l2)
    torch.cuda.synchronize()
    assert st.item() == 0
    a1, a2 = s1.get_params().astype(np.float64), s2.get_params().astype(np.float64)
    moved = np.abs(a1 - p0)
    assert np.median(moved) > 1e-4          # four steps of ~lr each moved the weights
    assert np.max(np.abs(a1 - a2)) <= 1e-6, np.max(np.abs(a1 - a2))
    assert l1.item() == pytest.approx(l2.item(), rel=1e-3)


@pytest.fixture(scope="module")
def trained(P):
    """Surrogate trained on 2^20 exact targets (the benchmark trains on 2^22)."""
    import torch
    n = 1 << 20
    u = torch.empty(n, device="cuda")
    lam = torch.empty(n, device="cuda")
    p = torch.empty(n, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.ncx2_targets(NU_CFG, n, u, lam, p, st, seed=11, tag=1, loglam_lo=-6.0, loglam_hi=7.0)
    s = P.Surrogate(NU_CFG, seed=3)
    loss = torch.zeros(1, device="cuda")
    s.train(u, lam, p, batch=8192, epochs=48, lr=3e-3, lr_final=3e-5, loss=loss)
    torch.cuda.synchronize()
    assert st.item() == 0
    return s, float(loss.item())


def test_training_beats_the_gaussian_limit(P, trained):
    """On held-out exact targets the trained network's RMSE is far below that
    of the approximation without it (P -> Phi^{-1}(U), Section 5.1)."""
    import torch
    from scipy.special import ndtri
    s, last_loss = trained
    n = 1 << 16
    u = torch.empty(n, device="cuda")
    lam = torch.empty(n, device="cuda")
    p = torch.empty(n, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.ncx2_targets(NU_CFG, n, u, lam, p, st, seed=999, tag=2)
    out = torch.zeros(n, device="cuda")
    s.eval(u, lam, out)
    torch.cuda.synchronize()
    t = p.cpu().numpy().astype(np.float64)
    e_mlp = out.cpu().numpy() - t
    e_gauss = ndtri(u.cpu().numpy().astype(np.float64)) - t
    rmse_mlp = math.sqrt(np.mean(e_mlp ** 2))
    rmse_gauss = math.sqrt(np.mean(e_gauss ** 2))
    # also where the CIR workload lives (lambda ~ e^2 .. e^4)
    sel = np.log(lam.cpu().numpy()) > 2.0
    reg = (math.sqrt(np.mean(e_mlp[sel] ** 2)), math.sqrt(np.mean(e_gauss[sel] ** 2)))
    assert math.isfinite(last_loss) and last_loss < 0.01, last_loss
    assert rmse_mlp < rmse_gauss / 20, (rmse_mlp, rmse_gauss, reg)
    assert reg[0] < reg[1] / 10, (rmse_mlp, rmse_gauss, reg)


def test_cir_exact_mean_and_surrogate_gain(P, trained):
    """Exact transitions reproduce E[X_T] = theta + (X0 - theta) e^{-kappa T};
    the learned transitions cut the variance of the two-way difference well
    below the Gaussian-limit transitions (Section 5.2)."""
    import torch
    s, _ = trained
    prm = P.sde_params(model=P.MODEL_CIR, payoff=P.PAYOFF_X, X0=0.08, T=1.0, K=0.0, mu=0.0, sigma=0.3,
                       kappa=0.5, theta=0.04, discount=1.0)
    ws = torch.empty(P.mlmc_level_workspace_bytes(), dtype=torch.uint8, device="cuda")
    sums = torch.zeros(P.SUMS, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    n = 20000
    res = {}
    for kind in (P.CIR_EXACT, P.CIR_DIFF, P.CIR_DIFF_GAUSS, P.CIR_SURROGATE):
        P.cir_level(prm, s, 3, kind, n, sums, ws, st, seed=4, tag=1)
        v = sums.cpu().numpy()
        m = v[0] / n
        res[kind] = (m, v[1] / n - m * m)
    assert st.item() == 0
    want = 0.04 + (0.08 - 0.04) * math.exp(-0.5)
    m, var = res[P.CIR_EXACT]
    assert abs(m - want) <= 4 * math.sqrt(var / n)
    assert res[P.CIR_DIFF][1] < res[P.CIR_DIFF_GAUSS][1] / 4, res
    # same uniforms: E[X^] - E[X~] from the DIFF kind equals the difference of means
    assert abs(res[P.CIR_DIFF][0] - (res[P.CIR_EXACT][0] - res[P.CIR_SURROGATE][0])) < 1e-9


def test_eval_kernel_matches_path_kernel_surrogate(P, orc):
    """The batched evaluation (tcgen05 MMA, TMEM accumulator, tiles of 128)
    and the CIR path kernel's warp-level evaluation (mma.sync) compute the
    same network: a one-step surrogate path X_1 = c max(h + 2 sqrt(h) P~, 0)
    with h = lambda + nu equals the same formula on the evaluation kernel's P~
    at that path's uniform, to FP32 rounding."""
    import torch
    rng = np.random.default_rng(5)
    s = P.Surrogate(NU_CFG, seed=0)
    params = _random_params(rng)
    s.set_params(params)
    kappa, theta, sigma, X0 = 0.5, 0.04, 0.3, 0.04
    prm = P.sde_params(model=P.MODEL_CIR, payoff=P.PAYOFF_X, X0=X0, T=1.0, K=0.0, mu=0.0, sigma=sigma,
                       kappa=kappa, theta=theta, discount=1.0)
    ws = torch.empty(P.mlmc_level_workspace_bytes(), dtype=torch.uint8, device="cuda")
    sums = torch.zeros(P.SUMS, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    c = sigma ** 2 * (-math.expm1(-kappa)) / (4 * kappa)
    e = math.exp(-kappa)
    nu32 = np.float32(4 * kappa * theta / sigma ** 2)
    lam = np.float32(max(np.float32(X0), np.float32(0)) * np.float32(e / c))
    seed, tag, m = 3, 7, 64
    key = [seed & 0xFFFFFFFF, seed >> 32]
    u = np.array([orc.u01(int(orc.philox4([0, p, 0, tag], key, 32)[0])) for p in range(m)], dtype=np.float32)
    pt = torch.zeros(m, device="cuda")
    s.eval(torch.from_numpy(u).cuda(), torch.full((m,), float(lam), device="cuda"), pt)
    pt = pt.cpu().numpy()
    h = np.float32(lam + nu32)
    want = np.float32(c) * np.maximum(np.float32(2) * np.sqrt(h) * pt + h, np.float32(0))
    # the two kernels add the last layer's 64 products w3_k h_k (|h_k| <= 1) in
    # different orders, so their P~ agree to a few ulps of sum |w3|; near
    # X_1 = 0 the cancellation in h + 2 sqrt(h) P~ magnifies that by 2 sqrt(h) c
    tol_p = 4 * 2.0 ** -24 * (float(np.abs(params[4352:4416]).sum()) + 1.0)
    for p in range(m):
        P.cir_level(prm, s, 0, P.CIR_SURROGATE, 1, sums, ws, st, path_offset=p, seed=seed, tag=tag)
        got = sums[0].item()
        tol = 2e-6 * abs(float(want[p])) + c * 2 * math.sqrt(h) * tol_p
        assert abs(got - float(want[p])) <= tol, (p, got, want[p], tol)
    assert st.item() == 0


@pytest.mark.parametrize("n", [1, 127, 128, 129, 255, 257, 1000, 40000, 400001])
def test_eval_ragged_tiles(P, orc, n):
    """Tiles of 128 samples taken in pairs, with ragged ends (a half-empty
    last pair, a one-sample last tile) and, at 400001 samples, several pairs
    per CTA: every output is written, nothing past the end, and the outputs
    agree with the oracle's network."""
    import torch
    rng = np.random.default_rng(n)
    s = P.Surrogate(NU_CFG, seed=0)
    p = _random_params(rng)
    s.set_params(p)
    u = orc.uniforms(11, 0, n)
    lam = np.exp(rng.uniform(-4.0, 4.0, n)).astype(np.float32)
    out = torch.full((n + 64,), float("inf"), device="cuda")
    s.eval(torch.from_numpy(u).cuda(), torch.from_numpy(lam).cuda(), out[:n])
    got = out.cpu().numpy().astype(np.float64)
    assert np.all(np.isinf(got[n:]))
    assert np.all(np.isfinite(got[:n]))
    idx = np.unique(np.concatenate([np.arange(min(n, 300)), rng.integers(0, n, 200), [n - 1]]))
    nn = orc.mlp_forward(_oracle_params(p), _features(u[idx].astype(np.float64), lam[idx].astype(np.float64)))
    ref = _compose(orc, u[idx], lam[idx].astype(np.float64), nn)
    sy = _sqrt_y(lam[idx].astype(np.float64))
    assert np.all(np.abs(got[idx] - ref) <= sy * (0.03 + 0.01 * np.abs(nn)) + 2e-6 * np.abs(ref) + 1e-6)


# ---------------------------------------------------------------------------
# Learned CIR paths step by step against the oracle's network (Section 5.2)
R_TANH, R_BF16 = 2.0 ** -10.9, 2.0 ** -9                 # tanh.approx.f32 relative error; BF16 rounding


def _plumbing_params(rng):
    """Weights for the path test: the inputs move P~ by O(0.3) through the
    64 x 64 layer, whose small weights keep the GPU's BF16 / tanh.approx
    error -- the bound below -- near 1e-3."""
    p = np.zeros(4417, dtype=np.float32)
    p[0:128] = rng.uniform(-1.5, 1.5, 128)
    p[128:192] = rng.uniform(-0.5, 0.5, 64)
    p[192:4288] = rng.uniform(-0.05, 0.05, 4096)
    p[4288:4352] = rng.uniform(-0.3, 0.3, 64)
    p[4352:4416] = rng.uniform(-0.5, 0.5, 64)
    p[4416] = 0.1
    return p


def _net_layers(q, x0, x1):
    """The network in FP64 (W2 BF16-rounded as the GPU keeps it): output, the
    layer activations, and dy/dx0, dy/dx1 -- used for the error bound only;
    the path emulation takes its P~ from the oracle's mlp_forward."""
    a1 = q["W1"] @ np.array([x0, x1]) + q["b1"]
    t1 = np.tanh(a1)
    z2 = q["W2"] @ t1 + q["b2"]
    h2 = np.tanh(z2)
    y = float(q["w3"] @ h2 + q["b3"][0])
    g = (q["w3"] * (1 - h2 ** 2)) @ q["W2"] * (1 - t1 ** 2)   # dy/da1
    return y, t1, h2, float(g @ q["W1"][:, 0]), float(g @ q["W1"][:, 1])


def _net_error_bound(q, t1, h2, dydx0, dydx1, s):
    """Error of the GPU's P~ against the FP64 network at one evaluation, as
    (sd, wc).  sd: the rounding errors of the GPU network -- layer-1
    activations from tanh.approx (relative 2^-10.9) rounded to BF16 (2^-9),
    tanh.approx again after the 64 x 64 product -- taken as independent and
    uniform within their bounds and propagated linearly (standard deviation).
    wc: worst-case terms -- FP32 accumulation, and the inputs' FP32 error: the
    feature sqrt(-2 ln 2v) takes __logf (absolute error ~2^-21 near 1), which
    moves s by min(dL / s, sqrt(2 dL))."""
    var_h1 = (R_BF16 ** 2 + R_TANH ** 2) / 3.0 * t1 ** 2
    var_z2 = (q["W2"] ** 2) @ var_h1
    var_h2 = (1 - h2 ** 2) ** 2 * var_z2 + R_TANH ** 2 / 3.0 * h2 ** 2
    sd = math.sqrt(float((q["w3"] ** 2) @ var_h2))
    dL = 2.0 ** -21
    ds = min(dL / s, math.sqrt(2 * dL)) if s > 0 else math.sqrt(2 * dL)
    wc = (2.0 ** -18 * float(np.abs(q["w3"]) @ (np.abs(q["W2"]) @ np.abs(t1))) +
          2.0 ** -20 * (float(np.abs(q["w3"]) @ np.abs(h2)) + abs(float(q["b3"][0]))) +
          abs(dydx0) * (ds / 3 + 1e-7) + abs(dydx1) * 2.0 ** -21)
    return sd, wc


def _surrogate_step(orc, qd, nu, cc, e, u, x, feature_power=0.5):
    """One learned transition as aicdf.h defines it: lambda = max(X, 0) e / c,
    sqrt(y) = sqrt(nu / (lambda + nu)), features (s(u)/3, 2 sqrt(y) - 1), N from
    the oracle network, P~ = Phi^{-1}(u) + sqrt(y) N, X' = c max(h + 2 sqrt(h) P~,
    0).  Returns X' and the (sd, worst-case) parts of its error from this
    evaluation.  feature_power != 1/2 plants a wrong input (y^p for sqrt(y))."""
    lam = max(x, 0.0) * e / cc
    sy = math.sqrt(nu / (lam + nu))
    v = min(u, 1.0 - u)
    s = math.sqrt(max(-2.0 * math.log(2.0 * v), 0.0))
    x0 = (-s if u < 0.5 else s) / 3.0
    x1 = 2.0 * (nu / (lam + nu)) ** feature_power - 1.0
    nn = float(orc.mlp_forward(qd, np.array([[x0, x1]]))[0])
    y, t1, h2, d0, d1 = _net_layers(qd, x0, x1)
    assert abs(y - nn) <= 1e-12 * (1 + abs(nn))          # the bound describes the oracle's own network
    sd, wc = _net_error_bound(qd, t1, h2, d0, d1, s)
    z = orc.phiinv_f64(u)
    pt = z + sy * nn
    sd, wc = sy * sd, sy * (wc + abs(d1) * 1e-6) + 2e-6 * abs(z)   # FP32 sqrt(y); the FP32 inverse, 1e-6 rel.
    h = lam + nu
    k = 2.0 * cc * math.sqrt(h)
    return cc * max(h + 2.0 * math.sqrt(h) * pt, 0.0), k * sd, k * wc


def _emulate_surrogate_path(orc, qd, prm_q, level, p, seed, tag, feature_power=0.5):
    """Exact and learned CIR path of 2^level steps from the same uniforms, with
    the error of the learned one carried along: sd' = sqrt((L sd)^2 + sd_new^2)
    and wc' = L wc + wc_new + FP32 rounding of the step, L the step map's
    sensitivity to X (central difference of the FP64 map at the same u).
    Returns X^_T, X~_T and the band 6 sd + 1.5 wc."""
    q = prm_q
    nu = 4 * q["kappa"] * q["theta"] / q["sigma"] ** 2
    hstep = q["T"] / 2 ** level
    e = math.exp(-q["kappa"] * hstep)
    cc = q["sigma"] ** 2 * (-math.expm1(-q["kappa"] * hstep)) / (4 * q["kappa"])
    key = [seed & 0xFFFFFFFF, seed >> 32]
    xe = q["X0"]
    xa = float(np.float32(q["X0"]))
    sd = wc = 0.0
    for s in range(2 ** level):
        w = int(orc.philox4([s // 4, p & 0xFFFFFFFF, p >> 32, tag], key, 32)[s % 4])
        u = orc.u01(w)
        lam_e = xe * e / cc
        xe = cc * (orc.ncx2_ppf(u, nu, lam_e) if u <= 0.5 else orc.ncx2_isf(1.0 - u, nu, lam_e))
        xn, sd_new, wc_new = _surrogate_step(orc, qd, nu, cc, e, u, xa, feature_power)
        d = max(1e-9, 1e-4 * abs(xa))
        lo = max(xa - d, 0.0)
        L = abs(_surrogate_step(orc, qd, nu, cc, e, u, xa + d, feature_power)[0] -
                _surrogate_step(orc, qd, nu, cc, e, u, lo, feature_power)[0]) / (xa + d - lo)
        sd = math.sqrt((L * sd) ** 2 + sd_new ** 2)
        wc = L * wc + wc_new + 8 * 2.0 ** -24 * (abs(xn) + cc * (nu + max(xa, 0) * e / cc))
        xa = xn
    return xe, xa, 6 * sd + 1.5 * wc + 1e-9


@pytest.mark.parametrize("level", [0, 2, 4, 6])
def test_cir_surrogate_paths_match_oracle_network(P, orc, level):
    """aicdf_cir_level SURROGATE and DIFF paths, one at a time, against the
    step-by-step restatement above with the oracle's FP64 network (BF16 W2),
    at the CIR configuration (nu = 0.889), levels 0..6 (lambda from near 0 at
    X0 = 0.0005 to ~e^6 at level 6 from X0 = 0.3).  The emulation with a wrong
    input (y for sqrt(y)) is checked to fall outside the tolerance, so the band
    is tight enough to see such a mistake."""
    import torch
    rng = np.random.default_rng(17)
    params = _plumbing_params(rng)
    qd = _oracle_params(params)
    s = P.Surrogate(NU_CFG, seed=0)
    s.set_params(params)
    ws = torch.empty(P.mlmc_level_workspace_bytes(), dtype=torch.uint8, device="cuda")
    sums = torch.zeros(P.SUMS, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    seed, tag = 9, 4
    caught = 0
    for X0 in (0.04, 0.0005, 0.3):
        q = dict(kappa=0.5, theta=0.04, sigma=0.3, X0=X0, T=1.0)
        prm = P.sde_params(model=P.MODEL_CIR, payoff=P.PAYOFF_X, X0=X0, T=1.0, K=0.0, mu=0.0, sigma=0.3,
                           kappa=0.5, theta=0.04, discount=1.0)
        for p in ((0, 5, 77777) if level < 6 else (3,)):
            xe, xa, band = _emulate_surrogate_path(orc, qd, q, level, p, seed, tag)
            got = {}
            for kind in (P.CIR_EXACT, P.CIR_SURROGATE, P.CIR_DIFF):
                P.cir_level(prm, s, level, kind, 1, sums, ws, st, path_offset=p, seed=seed, tag=tag)
                got[kind] = sums[0].item()
            assert st.item() == 0
            assert band <= 0.02 * (abs(xa) + 0.04), (level, X0, p, band, xa)   # well inside the scale of X
            assert got[P.CIR_EXACT] == pytest.approx(xe, rel=1e-6, abs=1e-12)
            assert abs(got[P.CIR_SURROGATE] - xa) <= band, (level, X0, p, got[P.CIR_SURROGATE], xa, band)
            assert abs(got[P.CIR_DIFF] - (xe - xa)) <= band + 1e-6 * abs(xe), (level, X0, p)
            # the same path with y fed for sqrt(y) (a plausible slip) leaves the band
            _, xb, _ = _emulate_surrogate_path(orc, qd, q, level, p, seed, tag, feature_power=1.0)
            caught += abs(xb - xa) > 3 * band
    assert caught >= 3, caught


def test_save_and_load_round_trip(P, orc, tmp_path):
    """aicdf_surrogate_save / _load: the loaded handle has the same nu and
    weights and evaluates to the same bits."""
    import torch
    rng = np.random.default_rng(23)
    s = P.Surrogate(NU_CFG, seed=0)
    s.set_params(_random_params(rng))
    path = str(tmp_path / "sur.bin")
    s.save(path)
    t = P.Surrogate.load(path)
    assert t.nu == NU_CFG
    assert np.array_equal(s.get_params(), t.get_params())
    n = 4096
    u = torch.from_numpy(orc.uniforms(3, 0, n)).cuda()
    lam = torch.from_numpy(np.exp(rng.uniform(-6, 7, n)).astype(np.float32)).cuda()
    a, b = torch.zeros(n, device="cuda"), torch.ones(n, device="cuda")
    s.eval(u, lam, a)
    t.eval(u, lam, b)
    assert torch.equal(a, b)
