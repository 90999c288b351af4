"""Multi-rank path of bench.py on CPU (gloo, world size 2): replicas are independent, the timed
region is the maximum over ranks and the work is the sum of every rank's site-steps."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [100.0, 250.0][rank]
    value, total = bench.aggregate(ms, 1000 * (rank + 1), dist)
    q.put((rank, value, total))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, value, total in out:
        assert total == 250.0                         # the slowest rank defines the timed region
        assert abs(value - 3000 / 0.25) < 1e-9        # all ranks' work over that time


def test_single_rank_aggregation():
    import bench
    value, total = bench.aggregate(200.0, 500)
    assert total == 200.0 and abs(value - 2500.0) < 1e-9
