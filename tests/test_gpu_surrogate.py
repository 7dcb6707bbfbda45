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


def _features(u, lam):
    v = np.minimum(u, 1 - u)
    s = np.sqrt(np.maximum(-2 * np.log(2 * v), 0.0))
    x0 = np.where(u < 0.5, -s, s) / 3.0
    x1 = np.clip(np.log(np.maximum(lam, 1e-30)) / 4.0, -1, 1)
    return np.stack([x0, x1], axis=1)


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
    ref = orc.mlp_forward(_oracle_params(p), _features(u.astype(np.float64), lam.astype(np.float64)))
    err = np.abs(got - ref)
    assert np.all(err <= 0.03 + 0.01 * np.abs(ref)), err.max()
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
    loss, ref = orc.mlp_grad(_oracle_params(p), _features(u.astype(np.float64), lam.astype(np.float64)),
                             tgt.astype(np.float64))
    assert got[4417] / n == pytest.approx(loss, rel=0.05)
    offs = {"W1": (0, 128), "b1": (128, 192), "W2": (192, 4288), "b2": (4288, 4352), "w3": (4352, 4416),
            "b3": (4416, 4417)}
    for name, (a, b) in offs.items():
        gv, rv = got[a:b], ref[name].reshape(-1)
        assert np.linalg.norm(gv - rv) <= 0.05 * np.linalg.norm(rv) + 1e-6, name
        if b - a > 1:
            cos = gv @ rv / (np.linalg.norm(gv) * np.linalg.norm(rv))
            assert cos > 0.995, (name, cos)


@pytest.fixture(scope="module")
def trained(P):
    """Surrogate trained on 2^20 exact targets (the benchmark trains on 2^22)."""
    import torch
    n = 1 << 20
    u = torch.empty(n, device="cuda")
    lam = torch.empty(n, device="cuda")
    p = torch.empty(n, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.ncx2_targets(NU_CFG, n, u, lam, p, st, seed=11, tag=1)
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
    assert rmse_mlp < rmse_gauss / 4, (rmse_mlp, rmse_gauss, reg)
    assert reg[0] < reg[1] / 2, (rmse_mlp, rmse_gauss, reg)


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
    ref = orc.mlp_forward(_oracle_params(p), _features(u[idx].astype(np.float64), lam[idx].astype(np.float64)))
    assert np.all(np.abs(got[idx] - ref) <= 0.03 + 0.01 * np.abs(ref))
