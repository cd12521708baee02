"""The multi-rank bench path on CPU: two gloo ranks, each with its own box,
reduce their timed regions and particle counts as bench.py does under
torchrun (no data-path collective; the max over ranks and the sum of
particles are the only exchanges)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: a box of 1000 * (r + 1) particles timed at 10 * (r + 1) ms
        res = bench.reduce_over_ranks(10.0 * (rank + 1), 1000 * (rank + 1), 4, world, torch.device("cpu"))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_bench():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        t_max, n_all, rate = res[r]
        assert t_max == 20.0          # the slowest rank's timed region
        assert n_all == 3000          # particles of both ranks
        assert rate == pytest.approx(3000 * 4 / 0.020)


def test_single_rank_is_local():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(5.0, 100, 2, 1, torch.device("cpu")) == (5.0, 100, 100 * 2 / 0.005)
