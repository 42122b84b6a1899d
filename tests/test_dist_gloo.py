"""The multi-rank host logic on CPU: two gloo ranks stand in for two GPUs.

- bench.py under torchrun times each rank and reports the largest time (the
  job's time), and runs its replicas with no exchange on the data path: each
  rank contributes a different number and both must read back the maximum;
- a sharded computation's one exchange (``allreduce_partials``): each rank
  takes the oracle's partials of its own middle-node range, the ranks sum
  them through the binding's all-reduce helper, and both must finalize to
  Algorithm 1's EF;
- the exchange by node range (``reduce_scatter_partials``): each rank gets
  the sums of its own nodes only and finalizes them to Algorithm 1's EF.
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


def _shard_rank(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    import paper_2306_00606_gb300 as ef
    from oracle import shard
    g = synth.disjoint_union([synth.watts_strogatz(150, 6, 0.1, 11), synth.barabasi_albert(120, 3, 12)])
    cuts = shard.node_cuts(g.row_ptr, world)
    p = shard.partials(g, cuts[rank], cuts[rank + 1])
    # the oracle's partials in the binding's five slots (t, and four integer arrays)
    parts = {"t": torch.from_numpy(p["T"].copy()), "q": torch.zeros(g.n, dtype=torch.int64),
             "triangles": torch.zeros(g.n, dtype=torch.int64), "n_clusters": torch.from_numpy(p["N"].copy()),
             "s_open": torch.from_numpy(p["S"].copy())}
    ef.allreduce_partials(parts)
    T, S, N = parts["t"], parts["s_open"], parts["n_clusters"]
    fin = shard.finalize(S.numpy(), T.numpy())
    ref = oracle.alg1(g)
    ok = (np.array_equal(N.numpy(), ref["N"]) and np.array_equal(S.numpy(), ref["S"])
          and np.allclose(fin["EF"], ref["EF"], rtol=1e-12, atol=1e-12)
          and int(np.count_nonzero(p["N"])) < g.n)   # each rank alone holds only part of the clusters
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, bool(ok)))


def test_sharded_partials_allreduce_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, True), (1, True)]


def _rs_rank(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    import paper_2306_00606_gb300 as ef
    from oracle import shard
    g = synth.disjoint_union([synth.watts_strogatz(150, 6, 0.1, 11), synth.barabasi_albert(120, 3, 12)])
    cuts = shard.node_cuts(g.row_ptr, world)
    lo, hi = int(cuts[rank]), int(cuts[rank + 1])
    p = shard.partials(g, lo, hi)
    parts = {"t": torch.from_numpy(p["T"].copy()), "q": torch.zeros(g.n, dtype=torch.int64),
             "triangles": torch.zeros(g.n, dtype=torch.int64), "n_clusters": torch.from_numpy(p["N"].copy()),
             "s_open": torch.from_numpy(p["S"].copy())}
    ranges = ef.shard_ranges((lo, hi))
    ef.reduce_scatter_partials(parts, ranges)
    mine = ef.partials_slice(parts, lo, hi)
    fin = shard.finalize(mine["s_open"].numpy(), mine["t"].numpy())
    ref = oracle.alg1(g)
    ok = (ranges == [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]
          and np.array_equal(mine["n_clusters"].numpy(), ref["N"][lo:hi])
          and np.array_equal(mine["s_open"].numpy(), ref["S"][lo:hi])
          and np.allclose(fin["EF"], ref["EF"][lo:hi], rtol=1e-12, atol=1e-12))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, bool(ok)))


def test_sharded_partials_reduce_scatter_two_gloo_ranks():
    """The exchange by node range: each rank receives the summed partials of
    its own nodes only and finalizes them to Algorithm 1's EF."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rs_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, True), (1, True)]
