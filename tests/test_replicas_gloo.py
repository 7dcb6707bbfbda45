"""The multi-GPU form of the benchmark is replicas only: one process per GPU,
disjoint Philox streams keyed by rank, no data-path collective, and the job's
time is the slowest rank's (all-reduce MAX).  These host-side pieces run here
as two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank                 # rank 1 is the slower one
        job_ms = bench._max_over_ranks(local_ms, dist, "cpu")
        r, w, lr = bench._env_rank()
        q.put((rank, job_ms, bench._replica_seed(r), w, lr))
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_and_disjoint_streams(orc):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(2))
    assert [o[1] for o in out] == [15.0, 15.0]        # both see the slowest rank's time
    assert [o[3] for o in out] == [2, 2] and [o[4] for o in out] == [0, 1]
    seeds = [o[2] for o in out]
    assert seeds[0] != seeds[1]
    # the replicas' samples come from different Philox keys: no shared values
    u0 = orc.uniforms(seed=seeds[0], offset=0, n=4096)
    u1 = orc.uniforms(seed=seeds[1], offset=0, n=4096)
    assert np.mean(u0 == u1) < 0.01
    import bench
    # whole-job value: all ranks' samples over the slowest time
    assert bench._whole_job_gsamples(2, 1 << 28, 20, 15.0 * 20) == pytest.approx(2 * (1 << 28) / 15e-3 / 1e9)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 3
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
