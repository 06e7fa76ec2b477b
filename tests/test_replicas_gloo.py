"""The N > 1 path on CPU: two gloo ranks, each running the FP64 oracle on its own shard of
queries (the replica layout the multi-GPU benchmark uses), aggregated as units of all ranks
over the slowest rank's time."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2407_09649_gb300 import replicas, scenes
    ws, r, _ = replicas.rank_env()
    surf = scenes.sphere_plane_frame(0, n_sphere=1500, n_plane=1500)
    queries = scenes.uniform_queries(seed=100 + r, n=200 + 100 * r, lo=(-3, -3, -2), hi=(3, 3, 3))
    S = oracle.Surface(surf, oracle.params())
    res = S.query(queries, want_var=False)
    seconds = 1.0 + r  # rank 1 is the slow one
    rate, slowest = replicas.aggregate(len(queries), seconds, ws)
    q.put((r, rate, slowest, int((res["status"] == 0).sum()), len(queries)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_weak_scaling():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    total = out[0][4] + out[1][4]
    for r, rate, slowest, ok, n in out:
        assert slowest == 2.0
        assert rate == pytest.approx(total / 2.0)
        assert ok == n
