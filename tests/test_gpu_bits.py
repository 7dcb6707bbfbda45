"""GPU parity of truncated-bit sampling (aicdf_sample_bits) against the oracle.

The oracle's B-bit stream (or_uniforms_bits) supplies the uniforms; each
method is then compared with the oracle's sampler at those uniforms, with the
tolerances of the full-precision path: PWC bit-exact, PWL within 2 FP32 ulp,
the cubic within 4 * 2^-24 * sum|c_j| + 2 ulp, the exact inverse within 1e-6
relative.
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


def _gpu(P, table, method, bits, n, seed=0, offset=0, dtype="f32", shift=0):
    """Run aicdf_sample_bits into a buffer starting `shift` elements into an
    allocation (shift != 0 breaks the 32-byte alignment: scalar path)."""
    import torch
    tdt = torch.float32 if dtype == "f32" else torch.float16
    buf = torch.full((n + shift,), float("nan"), dtype=tdt, device="cuda")
    out = buf[shift:]
    P.sample_bits(table, method, bits, out, seed=seed, offset=offset, n=n)
    torch.cuda.synchronize()
    return out.float().cpu().numpy().astype(np.float64)


def _ulp(x):
    return np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)


def _check(P, orc, method, table, z, u):
    if method == P.PWC:
        ref, _ = orc.sample_pwc(table.coefficients()[0].astype(np.float32), u)
        assert np.array_equal(z, ref)
    elif method == P.PWL:
        a, b = (x.astype(np.float32) for x in table.coefficients())
        ref, _ = orc.sample_pwl(a, b, u)
        assert np.all(np.abs(z - ref) <= 2 * _ulp(ref))
    elif method == P.PWP:
        c = table.coefficients()[0].astype(np.float32)
        ref = orc.sample_pwp(c, u)
        ud = u.astype(np.float64)
        v = np.minimum(ud, 1 - ud)
        _, ex = np.frexp(v)
        k = np.where(v >= 0.5, 0, np.minimum(-ex, c.shape[0] - 1))
        bound = 4 * 2.0 ** -24 * np.abs(c.astype(np.float64)).sum(axis=1)[k]
        assert np.all(np.abs(z - ref) <= bound + 2 * _ulp(ref))
    else:
        ref = orc.phiinv(u)
        assert np.all(np.abs(z - ref) <= 1e-6 * np.abs(ref) + 1e-12)


CASES = [("PWL", 15), ("PWC", 1024), ("PWC", 256), ("PWC", 64), ("PWP", 15), ("EXACT", 0)]


def _table(P, name, n):
    if name == "EXACT":
        return None
    if name == "PWP":
        return P.table_build(P.PWP, n, 3)
    return P.table_build(getattr(P, name), n)


@pytest.mark.parametrize("bits", [8, 16])
@pytest.mark.parametrize("name,tn", CASES)
@pytest.mark.parametrize("n,offset,shift", [(1, 0, 0), (37, 0, 0), (4099, 64, 0), ((1 << 20) + 5, 0, 0),
                                            (1000, 3, 0), (999, 0, 1)])
def test_bits_parity(P, orc, bits, name, tn, n, offset, shift):
    method = getattr(P, name)
    t = _table(P, name, tn)
    u = orc.uniforms_bits(seed=11, offset=offset, n=n, bits=bits)
    z = _gpu(P, t, method, bits, n, seed=11, offset=offset, shift=shift)
    _check(P, orc, method, t, z, u)


@pytest.mark.parametrize("bits", [8, 16])
def test_bits_f16_and_large_counters(P, orc, bits):
    t = P.table_build(P.PWL, 15)
    a, b = (x.astype(np.float32) for x in t.coefficients())
    S = 4 * (32 // bits)
    for off in (0, S * ((1 << 32) + 3), S * ((1 << 32) - 40)):
        n = 20011
        u = orc.uniforms_bits(seed=5, offset=off, n=n, bits=bits)
        ref, _ = orc.sample_pwl(a, b, u)
        z = _gpu(P, t, P.PWL, bits, n, seed=5, offset=off, dtype="f16")
        r16 = ref.astype(np.float32).astype(np.float16).astype(np.float64)
        assert np.all(np.abs(z - r16) <= np.spacing(np.abs(r16).astype(np.float16)).astype(np.float64))
        z32 = _gpu(P, t, P.PWL, bits, n, seed=5, offset=off)
        assert np.all(np.abs(z32 - ref) <= 2 * _ulp(ref))


def test_bits_rademacher_and_midpoint_pwc(P, orc):
    """Unit-variance two-point table = Rademacher +-1; the exact inverse at
    8-bit uniforms equals the 256-interval midpoint table (Section 1)."""
    import torch
    t2 = P.table_build(P.PWC, 2, P.Z_V)
    out = torch.empty(1 << 22, dtype=torch.float32, device="cuda")
    P.sample_bits(t2, P.PWC, 8, out, seed=1)
    x = out.double()
    assert set(torch.unique(out).tolist()) == {-1.0, 1.0}
    assert abs(x.mean().item()) < 5 / math.sqrt(x.numel())
    n = 1 << 16
    ze = _gpu(P, None, P.EXACT, 8, n, seed=2)
    tc = P.table_build(P.PWC, 256, P.Z_C)
    zc = _gpu(P, tc, P.PWC, 8, n, seed=2)
    assert np.all(np.abs(ze - zc) <= 1e-6 * np.abs(zc))


def test_bits_full_size_sampled(P, orc):
    """2^28 samples (the benchmark's size) with 16-bit uniforms: sampled
    entries across the whole buffer equal the oracle's."""
    import torch
    t = P.table_build(P.PWL, 15)
    a, b = (x.astype(np.float32) for x in t.coefficients())
    n = 1 << 28
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    P.sample_bits(t, P.PWL, 16, out, seed=9)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([rng.integers(0, n, 3000), [0, 1, 7, 8, n - 1]]))
    got = out[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    for i, g in zip(idx, got):
        u = orc.uniforms_bits(seed=9, offset=int(i), n=1, bits=16)
        ref, _ = orc.sample_pwl(a, b, u)
        assert abs(g - ref[0]) <= 2 * _ulp(ref)[0]
