"""The N > 1 path of bench.py on CPU: world_size 2 over gloo.  Every rank
solves its own replica, so the only cross-rank step is the aggregation of
timing (max over ranks) and work (sum over ranks)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.aggregate_ranks(10.0 + 5.0 * rank, 100.0 * (rank + 1))
    q.put((rank, ms, units, bench.dist_setup()))
    dist.destroy_process_group()


def test_rank_aggregation_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, setup in out:
        assert ms == 15.0            # the slowest rank's time
        assert units == 300.0        # all ranks' work
        assert setup == (2, rank, rank)


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.aggregate_ranks(12.5, 7.0) == (12.5, 7.0)
