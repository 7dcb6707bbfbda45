"""GPU parity of the sampling kernels against the CPU oracle (through the C ABI).

Tolerances (from the paper's FP32 listing and the method's arithmetic):
  * piecewise constant: bit-exact (a table lookup);
  * piecewise linear: within 2 FP32 ulp of the oracle's FP64 evaluation with
    the same FP32 coefficients (one correctly rounded FMA on the GPU);
  * FP16 output: within 1 FP16 ulp of the FP32 oracle value rounded to FP16;
  * exact Phi^{-1}: within 1e-6 relative (absolute floor 1e-12).
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
def tabs(P):
    tl = P.table_build(P.PWL, 15)
    tc = P.table_build(P.PWC, 1024)
    a, b = tl.coefficients()
    q = tc.coefficients()[0]
    return tl, tc, a.astype(np.float32), b.astype(np.float32), q.astype(np.float32)


def _gpu_sample(P, table, method, n, seed=0, offset=0, u=None, dtype="f32"):
    import torch
    tdt = torch.float32 if dtype == "f32" else torch.float16
    out = torch.full((n,), float("nan"), dtype=tdt, device="cuda")
    uu = None if u is None else torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda()
    P.sample(table, method, out, u=uu, seed=seed, offset=offset, n=n)
    torch.cuda.synchronize()
    return out.float().cpu().numpy().astype(np.float64)


def _ulp32(x):
    return np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)


def _assert_pwl(z, ref):
    both_nan = np.isnan(z) & np.isnan(ref)
    ok = both_nan | (np.abs(z - ref) <= 2 * _ulp32(ref))
    assert ok.all(), (np.flatnonzero(~ok)[:5], z[~ok][:5], ref[~ok][:5])


def _assert_exact(z, ref):
    same_inf = np.isinf(ref) & (z == ref)
    both_nan = np.isnan(z) & np.isnan(ref)
    ok = same_inf | both_nan | (np.abs(z - ref) <= 1e-6 * np.abs(ref) + 1e-12)
    assert ok.all(), (np.flatnonzero(~ok)[:5], z[~ok][:5], ref[~ok][:5])


SIZES = [1, 3, 4, 5, 8, 31, 4097, (1 << 20) + 13]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("offset", [0, 8, 6])
def test_pwl_philox_parity(P, tabs, orc, n, offset):
    tl, _, a, b, _ = tabs
    u = orc.uniforms(seed=7, offset=offset, n=n)
    ref, _ = orc.sample_pwl(a, b, u)
    z = _gpu_sample(P, tl, P.PWL, n, seed=7, offset=offset)
    _assert_pwl(z, ref)
    # one correctly rounded FMA: nearly always bit-equal to the FP32-rounded oracle value
    assert np.mean(z == ref.astype(np.float32).astype(np.float64)) > 0.999


@pytest.mark.parametrize("n", [5, 4099, (1 << 18) + 3])
def test_pwl_pwc_f16(P, tabs, orc, n):
    tl, tc, a, b, q = tabs
    u = orc.uniforms(seed=3, offset=0, n=n)
    ref, _ = orc.sample_pwl(a, b, u)
    h = _gpu_sample(P, tl, P.PWL, n, seed=3, dtype="f16")
    r16 = ref.astype(np.float32).astype(np.float16).astype(np.float64)
    ulp16 = np.spacing(np.abs(r16).astype(np.float16)).astype(np.float64)
    assert np.all(np.abs(h - r16) <= ulp16)
    assert np.mean(h == r16) > 0.999
    refc, _ = orc.sample_pwc(q, u)
    hc = _gpu_sample(P, tc, P.PWC, n, seed=3, dtype="f16")
    assert np.array_equal(hc, refc.astype(np.float32).astype(np.float16).astype(np.float64))


@pytest.mark.parametrize("n", SIZES)
def test_pwc_philox_bit_exact(P, tabs, orc, n):
    _, tc, _, _, q = tabs
    u = orc.uniforms(seed=11, offset=0, n=n)
    ref, _ = orc.sample_pwc(q, u)
    z = _gpu_sample(P, tc, P.PWC, n, seed=11)
    assert np.array_equal(z, ref)


@pytest.mark.parametrize("n", [7, 4096, (1 << 20) + 5])
@pytest.mark.parametrize("method", ["EXACT", "EXACT_LIB"])
def test_exact_philox_parity(P, orc, n, method):
    u = orc.uniforms(seed=1, offset=0, n=n)
    ref = orc.phiinv(u)
    z = _gpu_sample(P, None, getattr(P, method), n, seed=1)
    _assert_exact(z, ref)


def _edge_uniforms():
    tiny = [1e-45, 1e-40, 1.2e-38, 1e-30, 1e-12, 1.7e-8, 2.0 ** -25, 2.0 ** -24, 3e-8, 1e-7]
    specials = [0.0, 1.0, 0.5, np.nan, -0.25, 1.5, -0.0, np.inf,
                np.nextafter(np.float32(0.5), np.float32(0)), np.nextafter(np.float32(0.5), np.float32(1)),
                1.0 - 2.0 ** -24, 0.25, 0.75, 2.0 ** -15, 2.0 ** -16, 2.0 ** -15 * 1.5]
    edges = []
    for k in range(1, 25):
        e = np.float32(2.0 ** -k)
        edges += [e, np.nextafter(e, np.float32(0)), np.nextafter(e, np.float32(1))]
        edges += [np.float32(1) - e]
    rng = np.random.default_rng(9)
    rand = rng.random(5000).astype(np.float32)
    logu = (10.0 ** -rng.uniform(0, 37, 2000)).astype(np.float32)
    return np.concatenate([np.array(tiny + specials, dtype=np.float32), np.array(edges, dtype=np.float32),
                           rand, logu, 1 - logu]).astype(np.float32)


def test_input_mode_edge_cases(P, tabs, orc):
    """Caller-given u: interval edges, subnormals, 0, 1, 1/2, NaN, out-of-range."""
    tl, tc, a, b, q = tabs
    u = _edge_uniforms()
    for n in (u.size, u.size - 3):   # vector path with a ragged tail
        uu = u[:n]
        ref, _ = orc.sample_pwl(a, b, uu)
        z = _gpu_sample(P, tl, P.PWL, n, u=uu)
        _assert_pwl(z, ref)
        # u = 1/2 gives -0 (Algorithm 1 negates the zero row)
        i = int(np.flatnonzero(uu == 0.5)[0])
        assert z[i] == 0.0 and math.copysign(1.0, z[i]) == -1.0
        refc, _ = orc.sample_pwc(q, uu)
        zc = _gpu_sample(P, tc, P.PWC, n, u=uu)
        assert np.array_equal(np.isnan(zc), np.isnan(refc))
        assert np.array_equal(zc[~np.isnan(zc)], refc[~np.isnan(refc)])
        zinv = np.array([orc.phiinv_f64(float(x)) for x in uu])
        for m in ("EXACT", "EXACT_LIB"):
            ze = _gpu_sample(P, None, getattr(P, m), n, u=uu)
            if m == "EXACT":
                _assert_exact(ze, zinv)
            else:  # the library routine is only asked to agree away from u ~ 0
                sel = (uu > 1e-30) & (uu < 1.0) | np.isnan(uu)
                _assert_exact(ze[sel], zinv[sel])


@pytest.mark.parametrize("method", ["PWL", "PWC"])
def test_counters_beyond_32_bits(P, tabs, orc, method):
    """Sample offsets past 2^34 take the 64-bit-index kernel (Philox counter
    word 1 non-zero); offset 2^34 - 4000 straddles the 2^32 block boundary."""
    tl, tc, a, b, q = tabs
    for off in ((1 << 34) + 8, (1 << 34) - 4000):
        n = 8195
        u = orc.uniforms(seed=13, offset=off, n=n)
        if method == "PWL":
            ref, _ = orc.sample_pwl(a, b, u)
            z = _gpu_sample(P, tl, P.PWL, n, seed=13, offset=off)
            _assert_pwl(z, ref)
        else:
            ref, _ = orc.sample_pwc(q, u)
            z = _gpu_sample(P, tc, P.PWC, n, seed=13, offset=off)
            assert np.array_equal(z, ref)


def test_unaligned_pointers_use_scalar_path(P, tabs, orc):
    import torch
    tl, _, a, b, _ = tabs
    n = 1001
    u = orc.uniforms(seed=2, offset=0, n=n + 1)
    ref, _ = orc.sample_pwl(a, b, u[1:])
    buf = torch.full((n + 1,), float("nan"), dtype=torch.float32, device="cuda")
    ubuf = torch.from_numpy(u).cuda()
    P.sample(tl, P.PWL, buf[1:], u=ubuf[1:], n=n)     # 4-byte aligned, not 16
    torch.cuda.synchronize()
    _assert_pwl(buf[1:].cpu().numpy().astype(np.float64), ref)


@pytest.mark.parametrize("pinned", [True, False])
def test_sample_to_host_matches_device(P, tabs, pinned):
    """Pinned host memory: direct kernel stores; pageable: staged chunks with
    overlapped copies (2 MiB staging = two buffers, 8 MiB = four)."""
    import torch
    tl, tc, *_ = tabs
    for sb in (2 << 20, 8 << 20):
        staging = torch.empty(sb, dtype=torch.uint8, device="cuda")
        for table, method, dt, n, off in ((tl, P.PWL, torch.float32, 3 * (1 << 20) + 5, 0),
                                          (tc, P.PWC, torch.float16, (1 << 21) + 77, 12),
                                          (None, P.EXACT, torch.float32, 100003, 4),
                                          (tl, P.PWL, torch.float32, 4099, 6)):
            host = torch.empty(n, dtype=dt)
            if pinned:
                host = host.pin_memory()
            P.sample_to_host(table, method, host, staging, seed=5, offset=off)
            dev = torch.empty(n, dtype=dt, device="cuda")
            P.sample(table, method, dev, seed=5, offset=off)
            torch.cuda.synchronize()
            assert torch.equal(host, dev.cpu())


def test_determinism_and_streams(P, tabs):
    import torch
    tl, *_ = tabs
    n = (1 << 22) + 1
    x = torch.empty(n, device="cuda")
    y = torch.empty(n, device="cuda")
    s = torch.cuda.Stream()
    P.sample(tl, P.PWL, x, seed=123)
    with torch.cuda.stream(s):
        P.sample(tl, P.PWL, y, seed=123)
    torch.cuda.synchronize()
    assert torch.equal(x, y)


def test_statistics_match_table_moments(P, tabs):
    """Mean 0 (antisymmetry) and E[Z~^2] = int D^2 of the table (Section 2.3)."""
    tl, _, a, b, _ = tabs
    n = 1 << 24
    z = _gpu_sample(P, tl, P.PWL, n, seed=99)
    sq = 0.0
    for k in range(1, 16):
        hi = 2.0 ** -k
        lo = 0.0 if k == 15 else hi / 2
        sq += a[k] ** 2 * (hi - lo) + a[k] * b[k] * (hi * hi - lo * lo) + b[k] ** 2 * (hi ** 3 - lo ** 3) / 3
    ez2 = 2 * sq
    assert abs(z.mean()) < 5 * math.sqrt(ez2 / n)
    assert abs((z ** 2).mean() - ez2) < 5 * math.sqrt(2.0 / n)


def test_full_size_sampled_parity(P, tabs, orc):
    """The benchmark workload (2^28 PWL FP32 samples, Philox seed 0) in the
    benchmark's launch configuration, checked on sampled outputs."""
    import torch
    tl, _, a, b, _ = tabs
    n = 1 << 28
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    P.sample(tl, P.PWL, out, seed=0)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([rng.integers(0, n, 20000), np.arange(1000), np.arange(n - 1000, n)]))
    u = np.array([orc.uniforms(0, int(i), 1)[0] for i in idx], dtype=np.float32)
    ref, _ = orc.sample_pwl(a, b, u)
    z = out[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    _assert_pwl(z, ref)
    del out
    # FP16 at the same size
    out16 = torch.empty(n, dtype=torch.float16, device="cuda")
    P.sample(tl, P.PWL, out16, seed=0)
    torch.cuda.synchronize()
    h = out16[torch.from_numpy(idx).cuda()].float().cpu().numpy().astype(np.float64)
    r16 = ref.astype(np.float32).astype(np.float16).astype(np.float64)
    assert np.all(np.abs(h - r16) <= np.spacing(np.abs(r16).astype(np.float16)).astype(np.float64))


@pytest.mark.parametrize("method,offset", [("pwl", 0), ("pwl", 5), ("pwc", 2)])
def test_sweep_maximum_size_sampled_parity(P, tabs, orc, method, offset):
    """The largest size of the benchmark's size sweep, 2^30 FP32 samples
    (4 GiB), at an aligned and two unaligned stream offsets, checked on
    sampled outputs including both ends."""
    import torch
    tl, tc, a, b, q = tabs
    n = 1 << 30
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    if method == "pwl":
        P.sample(tl, P.PWL, out, seed=7, offset=offset)
    else:
        P.sample(tc, P.PWC, out, seed=7, offset=offset)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([rng.integers(0, n, 16000), np.arange(600), np.arange(n - 600, n)]))
    u = np.array([orc.uniforms(7, offset + int(i), 1)[0] for i in idx], dtype=np.float32)
    z = out[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    del out
    if method == "pwl":
        ref, _ = orc.sample_pwl(a, b, u)
        _assert_pwl(z, ref)
    else:
        ref, _ = orc.sample_pwc(q, u)
        assert np.array_equal(z, ref)
