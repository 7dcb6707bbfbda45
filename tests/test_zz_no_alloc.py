"""The MLMC level entry point for callers that cannot allocate device memory
(for example a component inside a host application that owns all GPU memory
through its own pool, or a latency-critical loop that cannot pay for
cudaMalloc).  It must give the same sums as the workspace-taking entry point,
call after call, although its scratch is one array shared by all calls.

Both entry points run the same kernel on the same grid and add the per-block
partials in the same fixed order, so their sums are compared bit for bit.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone."""
import ctypes as C

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


def test_noalloc_level_matches_workspace_entry_point(P):
    import torch
    L = P.lib()
    tl = P.table_build(P.PWL, 15)
    tc = P.table_build(P.PWC, 1024)
    ws = torch.empty(P.mlmc_level_workspace_bytes(), dtype=torch.uint8, device="cuda")
    ref = torch.zeros(P.SUMS, dtype=torch.float64, device="cuda")
    out = torch.zeros(P.SUMS, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    gbm = P.sde_params()
    cir = P.sde_params(model=P.MODEL_CIR, payoff=P.PAYOFF_X, X0=0.04, mu=0.0, sigma=0.3, kappa=0.5,
                       theta=0.04, discount=1.0)
    cases = [
        # (params, table, level, kind, n_paths, path_offset, seed, tag), in this order: a large
        # launch (every slot of the shared array written) right before small ones, so that a
        # slot left over from an earlier call would change the small calls' sums
        (gbm, tl, 5, P.KIND_CORR4, 1_000_003, 17, 7, 11),
        (cir, tl, 3, P.KIND_APPROX2, 54_321, 0, 8, 12),
        (gbm, tl, 0, P.KIND_APPROX2, 4_000_001, 3, 9, 13),   # level 0: four paths per Philox call
        (gbm, tc, 1, P.KIND_CORR4, 777, 5, 10, 14),          # level 1, piecewise constant table
        (gbm, tc, 4, P.KIND_EXACT2, 33, 0, 11, 15),
    ]
    for prm, table, level, kind, n, off, seed, tag in cases:
        for _ in range(2):   # two calls in a row
            out.fill_(-1.0)
            st = L.aicdf_mlmc_level_noalloc(C.byref(prm), table.handle, level, kind, n, off, seed, tag,
                                            out.data_ptr(), stream)
            assert st == P.OK, L.aicdf_status_str(st)
            P.mlmc_level(prm, table, level, kind, n, ref, ws, path_offset=off, seed=seed, tag=tag)
            torch.cuda.synchronize()
            g, r = out.cpu().numpy(), ref.cpu().numpy()
            assert g[4] == n == r[4]
            assert np.array_equal(g, r), (level, kind, n, g, r)
    # bad arguments are still refused before anything runs
    assert L.aicdf_mlmc_level_noalloc(C.byref(gbm), tl.handle, 3, P.KIND_CORR4, 0, 0, 0, 1,
                                      out.data_ptr(), stream) == P.ERR_ARG
