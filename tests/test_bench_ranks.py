"""The multi-rank benchmark path on CPU: world size 2 over gloo.

Under torchrun each rank runs its own independent job (the method shards by
job; no data-path exchange): each rank's job has its own seed, the timed
region's length is the maximum over ranks (bench.max_over_ranks, the only
collective), and the whole-job rate counts every rank's points
(bench.whole_job_rate). The ranks are spawned processes.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank: int, world: int, port: int, out) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1712_09005_gb300 import inputs
    r, w, local = bench.dist_env()
    slowest = bench.max_over_ranks(10.0 + 5.0 * r)  # rank 1 is the slow one
    seed = inputs.mixture_args(3, job=r, N=1000)["seed"]
    out.put((r, w, local, slowest, seed))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_over_gloo():
    import bench
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 2 and r[2] == r[0] for r in res)
    assert all(r[3] == 15.0 for r in res)  # every rank sees the slowest time
    assert res[0][4] != res[1][4]          # independent jobs
    # whole-job rate: both ranks' points over the slowest rank's seconds
    assert bench.whole_job_rate(2, 1000, 50, 0.015) == pytest.approx(2 * 1000 * 50 / 0.015)
    # a single process needs no group
    assert bench.max_over_ranks(3.5) == 3.5
