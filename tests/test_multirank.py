"""The multi-rank path of bench.py on CPU: two gloo ranks each time their own replica; the
job time is the slowest rank's and the value counts the steps of all ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 * (rank + 1)                      # rank 1 is the slow one
        t_max, value = bench.combine_ranks(local_ms, 50, world, "cpu")
        q.put((rank, t_max, value))
    finally:
        dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t_max, value in res:
        assert t_max == 200.0                              # max over ranks
        assert abs(value - 2 * 50 / 0.2) < 1e-9            # all ranks' steps / slowest time


def test_combine_ranks_single():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    t_max, value = bench.combine_ranks(40.0, 10, 1, "cpu")
    assert t_max == 40.0 and abs(value - 250.0) < 1e-9
