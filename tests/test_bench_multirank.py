"""The multi-rank path of bench.py on CPU: two gloo ranks combine their step
times with a max all-reduce (the job's time is its slowest rank), and the
reference arm does no work on ranks other than 0."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.reduce_max(1.5 + rank, dist, "cpu")
    none = bench.reduce_max(3.0, None, "cpu")
    out.put((rank, got, none))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2.5, 3.0), (1, 2.5, 3.0)]


def test_reference_arm_other_ranks_do_nothing():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        warmup = 0
        steps = 1
    assert bench.reference_arm(Args(), rank=1, world=2) is None
