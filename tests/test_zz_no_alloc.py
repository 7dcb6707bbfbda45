"""The MLMC level entry point for callers that cannot allocate device memory
(for example a component inside a host application that owns all GPU memory
through its own pool, or a latency-critical loop that cannot pay for
cudaMalloc).  It must give the same sums as the workspace-taking entry point,
call after call, although its scratch is one array shared by all calls.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone."""
import ctypes as C
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


def test_noalloc_level_matches_workspace_entry_point(P):
    import torch
    L = P.lib()
    tl = P.table_build(P.PWL, 15)
    ws = torch.empty(P.mlmc_level_workspace_bytes(), dtype=torch.uint8, device="cuda")
    ref = torch.zeros(3, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    cases = [
        # (params, level, kind, n_paths, path_offset, seed, tag): two calls in a row
        (P.sde_params(), 5, P.KIND_CORR4, 1_000_003, 17, 7, 11),
        (P.sde_params(model=P.MODEL_CIR, payoff=P.PAYOFF_X, X0=0.04, mu=0.0, sigma=0.3, kappa=0.5,
                      theta=0.04, discount=1.0), 3, P.KIND_APPROX2, 54_321, 0, 8, 12),
    ]
    for prm, level, kind, n, off, seed, tag in cases:
        st = L.aicdf_mlmc_level_noalloc(C.byref(prm), tl.handle, level, kind, n, off, seed, tag,
                                        out.data_ptr(), stream)
        assert st == P.OK, L.aicdf_status_str(st)
        P.mlmc_level(prm, tl, level, kind, n, ref, ws, path_offset=off, seed=seed, tag=tag)
        torch.cuda.synchronize()
        g, r = out.cpu().numpy(), ref.cpu().numpy()
        assert g[2] == n == r[2]
        # the tolerance of the other level-sum tests (same paths, same kernel)
        scale = math.sqrt(n * r[1])
        assert abs(g[0] - r[0]) <= 2e-6 * scale
        assert g[1] == pytest.approx(r[1], rel=2e-6)
    # bad arguments are still refused before anything runs
    assert L.aicdf_mlmc_level_noalloc(C.byref(cases[0][0]), tl.handle, 3, P.KIND_CORR4, 0, 0, 0, 1,
                                      out.data_ptr(), stream) == P.ERR_ARG
