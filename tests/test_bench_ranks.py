"""Whole-job timing over ranks (bench.py): the longest rank's time and the
sum of the ranks' units, by all-reduce.  Run here as two gloo ranks on the
CPU; on the GPU path the same helper runs over NCCL."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.ranks_aggregate(10.0 + 5.0 * rank, 100.0 * (rank + 1), world, "cpu")
    q.put((rank, ms, units))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_longest_time_and_all_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert got == [(0, 15.0, 300.0), (1, 15.0, 300.0)]


def test_one_rank_keeps_its_figures():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.ranks_aggregate(12.5, 42.0, 1, "cpu") == (12.5, 42.0)
