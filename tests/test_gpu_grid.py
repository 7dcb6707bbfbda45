"""Every point of the library's uniform grid through the caller-uniform path.

The library's own uniforms are the 2^23 cell midpoints u = (2k+1) 2^-24 of
(0, 1) (k < 2^23).  Feeding all of them through aicdf_sample with caller
uniforms exercises the general (capped-index, compare-and-reflect) forms of
Section 3.2 and Algorithm 1 at every interval edge the grid can reach:

* piecewise constant (1024 intervals): bit-equal to the oracle;
* piecewise linear (Algorithm 1) and piecewise cubic: within 2 FP32 ulp of
  the oracle (which evaluates the same FP32 coefficients in FP64), with the
  fraction of bit-equal results reported and required to be near 1;
* FP16 output: the round-to-nearest-even of the kernel's own FP32 result,
  and equal to the FP16 rounding of the oracle's FP32-rounded value wherever
  the two FP32 results agree.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_GRID = 1 << 23


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
def grid():
    k = np.arange(N_GRID, dtype=np.float64)
    u = ((2 * k + 1) * 2.0 ** -24).astype(np.float32)
    assert np.array_equal(u.astype(np.float64), (2 * k + 1) * 2.0 ** -24)   # exact in FP32
    return u


def _run(P, table, method, u, dtype):
    import torch
    ud = torch.from_numpy(u).cuda()
    out = torch.full((u.size,), float("nan"), dtype=dtype, device="cuda")
    P.sample(table, method, out, u=ud)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _ulp_check(z32, ref, what):
    z = z32.astype(np.float64)
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    bad = np.abs(z - ref) > 2 * ulp
    assert not bad.any(), (what, int(bad.sum()), np.flatnonzero(bad)[:5])
    same = np.mean(z32 == ref.astype(np.float32))
    return float(same)


def test_pwc_every_grid_point_bit_exact(P, orc, grid):
    import torch
    t = P.table_build(P.PWC, 1024)
    q32 = t.coefficients()[0].astype(np.float32)
    ref, idx = orc.sample_pwc(q32, grid)
    assert np.array_equal(np.bincount(idx, minlength=1024), np.full(1024, N_GRID // 1024))
    z = _run(P, t, P.PWC, grid, torch.float32)
    assert np.array_equal(z.astype(np.float64), ref)
    z16 = _run(P, t, P.PWC, grid, torch.float16)
    assert np.array_equal(z16, z.astype(np.float16))


def test_pwl_every_grid_point(P, orc, grid):
    import torch
    t = P.table_build(P.PWL, 15)
    a, b = t.coefficients()
    ref, idx = orc.sample_pwl(a.astype(np.float32), b.astype(np.float32), grid)
    assert set(np.unique(idx)) == set(range(1, 16))   # every interval of the table is reached
    z = _run(P, t, P.PWL, grid, torch.float32)
    same = _ulp_check(z, ref, "pwl")
    print(f"piecewise linear: {same:.6f} of the grid bit-equal to the oracle")
    assert same > 0.999, same
    z16 = _run(P, t, P.PWL, grid, torch.float16)
    assert np.array_equal(z16, z.astype(np.float16))
    agree = z == ref.astype(np.float32)
    assert np.array_equal(z16[agree], ref[agree].astype(np.float32).astype(np.float16))


@pytest.mark.parametrize("deg", [1, 3])
def test_pwp_every_grid_point(P, orc, grid, deg):
    import torch
    t = P.table_build(P.PWP, 15, deg)
    c32 = t.coefficients()[0].astype(np.float32)
    ref = orc.sample_pwp(c32, grid)
    z = _run(P, t, P.PWP, grid, torch.float32)
    # the kernels evaluate each row re-expanded in v, d_j = alpha^j sum_{i>=j}
    # C(i, j) beta^(i-j) c_j (s = alpha v + beta), by Horner's rule in FP32:
    # the rounding of the d_j and of each FMA is at most ~3 * 2^-24 of
    # sum_j |d_j| v^j, on top of the 2-ulp band (see test_gpu_pwp.py)
    c = c32.reshape(-1, 4).astype(np.float64)
    K = c.shape[0] - 1
    d = np.zeros_like(c)
    for r in range(K + 1):
        alpha, beta = (2.0 ** K, 0.0) if r == K else (2.0 ** (r + 1), -1.0)
        for j in range(4):
            d[r, j] = alpha ** j * sum(math.comb(i, j) * beta ** (i - j) * c[r, i] for i in range(j, 4))
    v = np.minimum(grid, 1 - grid).astype(np.float64)
    k = np.minimum(np.floor(-np.log2(v)).astype(int), K)
    dk = np.abs(d)[k]
    dv = dk[:, 0] + v * (dk[:, 1] + v * (dk[:, 2] + v * dk[:, 3]))
    bound = (2 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
             + 4 * 2.0 ** -24 * (np.abs(c).sum(axis=1)[k] + dv))
    err = np.abs(z.astype(np.float64) - ref)
    assert np.all(err <= bound), (deg, int((err > bound).sum()))
    same = float(np.mean(z == ref.astype(np.float32)))
    print(f"piecewise polynomial degree {deg}: {same:.4f} of the grid bit-equal to the oracle")
    # the oracle evaluates the s form in FP64, the kernels the v form in FP32:
    # about a third of the grid rounds to the same FP32 value
    assert same > 0.25, same
    z16 = _run(P, t, P.PWP, grid, torch.float16)
    assert np.array_equal(z16, z.astype(np.float16))
