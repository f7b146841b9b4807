"""The benchmark's multi-rank path on CPU (gloo, world size 2): ranks are independent
replicas and the only collective is the max-reduction of the step time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r takes (r + 1) seconds for 100 units: the job takes 2 s for 200 units
        value, t = bench.aggregate_throughput(100.0, float(rank + 1), dist, "cpu")
        out[rank] = (value, t)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    for r in range(2):
        value, t = out[r]
        assert t == 2.0 and value == 100.0


def test_single_rank_needs_no_collective():
    import bench
    assert bench.aggregate_throughput(50.0, 0.5) == (100.0, 0.5)
