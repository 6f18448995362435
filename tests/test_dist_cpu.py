"""The multi-process path of bench.py on CPU: two gloo ranks, barrier, the max
of the ranks' times and the replica throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    from paper_2302_12031_gb300 import dist as D
    r, w = D.init("gloo")
    assert (r, w) == (rank, world)
    D.barrier()
    seconds = 1.0 + rank            # rank 1 is the slowest
    value, t = D.replica_throughput(1000, seconds)
    out.put((rank, value, t, D.max_over_ranks(10.0 * (rank + 1))))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t, mx in res:
        assert t == 2.0                       # the slowest rank's time
        assert value == pytest.approx(2 * 1000 / 2.0)
        assert mx == 20.0


def test_single_process_needs_no_group():
    from paper_2302_12031_gb300 import dist as D
    assert D.max_over_ranks(3.5) == 3.5
    assert D.replica_throughput(10, 2.0) == (5.0, 2.0)
