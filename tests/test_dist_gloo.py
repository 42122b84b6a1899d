"""The multi-rank host logic of the benchmark on CPU: two gloo ranks.

bench.py under torchrun times each rank and reports the largest time (the
job's time), and runs its replicas with no exchange on the data path.  Here
two CPU processes stand in for two GPUs: each contributes a different
number and both must read back the maximum.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks(1.5 + rank * 2.25, world, torch.device("cpu"))
    single = bench.max_over_ranks(7.0, 1, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, single))


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 3.75, 7.0), (1, 3.75, 7.0)]
