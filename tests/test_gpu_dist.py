"""The sharded computation across two processes with the library's own partials.

Two processes share cuda:0 (each would be one GPU's rank; their kernels are
independent and never wait on each other).  Each runs ef_compute_shard for its
rank, copies the five partial arrays to the host and exchanges them over gloo:
- all-reduce (``allreduce_partials``), then ef_finalize_partials of every
  node on the device: N, S and triangles equal Algorithm 1's exactly, EF
  within the precision's bar;
- by node range (``reduce_scatter_partials``), then ef_finalize_partials of
  the rank's own nodes only: the same bars on its range.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    import paper_2306_00606_gb300 as ef
    torch.cuda.set_device(0)
    g = synth.disjoint_union([synth.powerlaw_cm(20000, 2.2, 3, 2000, 51), synth.erdos_renyi(3000, 0.005, 52),
                              synth.complete(30)])
    ref = oracle.alg1(g)
    tri = oracle.triangles(g)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    fails = []
    with ef.Context(0) as ctx:
        for prec, tol in (("fp64", dict(rtol=1e-9, atol=1e-12)), ("fp32c", dict(rtol=0, atol=2e-5))):
            parts = ef.empty_partials(g.n, "cuda")
            frac, (lo, hi) = ef.ef_compute_shard(ctx.handle, rp, ci, rank, world, parts, precision=prec)
            torch.cuda.synchronize()
            own_n = int(np.count_nonzero(parts["n_clusters"].cpu().numpy()))
            # all-reduce over gloo (host copies), finalize every node on the device
            host = {k: v.cpu() for k, v in parts.items()}
            ef.allreduce_partials(host)
            summed = {k: v.cuda() for k, v in host.items()}
            out = {k: torch.empty(g.n, dtype=dt, device="cuda") for k, dt in
                   (("ef", torch.float64), ("n_clusters", torch.int64), ("s", torch.int64),
                    ("triangles", torch.int64))}
            ef.ef_finalize_partials(ctx.handle, summed, frac, precision=prec, **out)
            got = {k: v.cpu().numpy() for k, v in out.items()}
            if not (np.array_equal(got["n_clusters"], ref["N"]) and np.array_equal(got["s"], ref["S"])
                    and np.array_equal(got["triangles"], tri) and 0 < own_n < g.n):
                fails.append(f"{prec} allreduce: integers")
            try:
                np.testing.assert_allclose(got["ef"], ref["EF"], **tol)
            except AssertionError as e:
                fails.append(f"{prec} allreduce: EF {e}")
            # by node range: only this rank's nodes, finalized here
            host = {k: v.cpu() for k, v in parts.items()}
            ranges = ef.shard_ranges((lo, hi))
            ef.reduce_scatter_partials(host, ranges)
            mine = {k: v.cuda() for k, v in ef.partials_slice(host, lo, hi).items()}
            out = {k: torch.empty(hi - lo, dtype=dt, device="cuda") for k, dt in
                   (("ef", torch.float64), ("n_clusters", torch.int64), ("s", torch.int64))}
            if hi > lo:
                ef.ef_finalize_partials(ctx.handle, mine, frac, precision=prec, **out)
            got = {k: v.cpu().numpy() for k, v in out.items()}
            if not (ranges[0][0] == 0 and ranges[-1][1] == g.n and ranges[0][1] == ranges[1][0]
                    and np.array_equal(got["n_clusters"], ref["N"][lo:hi])
                    and np.array_equal(got["s"], ref["S"][lo:hi])):
                fails.append(f"{prec} reduce-scatter: ranges or integers")
            try:
                np.testing.assert_allclose(got["ef"], ref["EF"][lo:hi], **tol)
            except AssertionError as e:
                fails.append(f"{prec} reduce-scatter: EF {e}")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, fails))


def test_two_ranks_exchange_real_shard_partials():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res == [(0, []), (1, [])], res
