"""The sharded computation on the GPU, through the C ABI.

R shards run one after another on one device (each would be one rank of a
multi-GPU job), their partials are summed on the device, and
ef_finalize_partials must then give
- N, S and the triangle counts of the unsharded ef_compute_ex exactly, and
  EF within the precision's bar (1e-9 relative FP64, 2e-5 absolute FP32C);
- Algorithm 1's values (the CPU oracle) on a graph small enough for it.
Per shard: the node ranges are the oracle's cuts (integer work, bit-exact)
and partition the nodes, and on a triangle-free graph each shard's T partial
equals the oracle's partial of the same range node by node, and its closed forms are Algorithm 1's N and S + 8t on its
own nodes.  Edge cases: more shards than nodes (empty ranges), R = 1, an
invalid shard index, a missing array, a fixed-point scale out of range,
asymmetric input.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import shard as oshard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2306_00606_gb300 as ef
    c = ef.Context(0)
    yield c
    c.close()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _shards(ctx, g, R, precision="fp64", wedge_mode=0):
    """Every shard's partials, their device sum (shard order) and the reported ranges."""
    import torch
    import paper_2306_00606_gb300 as ef
    rp, ci = _dev(g.row_ptr), _dev(g.col_idx)
    tot = {k: torch.zeros_like(v) for k, v in ef.empty_partials(g.n, "cuda").items()}
    parts, ranges, fracs = [], [], set()
    for r in range(R):
        p = ef.empty_partials(g.n, "cuda")
        frac, rng = ef.ef_compute_shard(ctx.handle, rp, ci, r, R, p, precision=precision, wedge_mode=wedge_mode)
        for k in tot:
            tot[k] += p[k]
        parts.append(p)
        ranges.append(rng)
        fracs.add(frac)
    assert len(fracs) == 1
    return rp, ci, tot, parts, ranges, fracs.pop()


def _finalize(ctx, tot, frac, precision):
    import torch
    import paper_2306_00606_gb300 as ef
    n = int(tot["t"].shape[0])
    out = dict(ef=torch.empty(n, dtype=torch.float64, device="cuda"),
               n_clusters=torch.empty(n, dtype=torch.int64, device="cuda"),
               s=torch.empty(n, dtype=torch.int64, device="cuda"),
               triangles=torch.empty(n, dtype=torch.int64, device="cuda"),
               flag=torch.empty(n, dtype=torch.uint8, device="cuda"))
    ef.ef_finalize_partials(ctx.handle, tot, frac, precision=precision, **out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _unsharded(ctx, rp, ci, precision):
    out = ctx.compute(rp, ci, precision=precision, outputs=("ef", "n_clusters", "s", "triangles", "flag"))
    return {k: v.cpu().numpy() for k, v in out.items()}


def _check_ranges(g, R, ranges):
    cuts = oshard.node_cuts(g.row_ptr, R)
    assert [r[0] for r in ranges] == cuts[:-1] and [r[1] for r in ranges] == cuts[1:]


def _close(got, ref, precision):
    if precision == "fp64":
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-12)
    else:
        np.testing.assert_allclose(got, ref, rtol=0, atol=2e-5)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
@pytest.mark.parametrize("R", [1, 3, 8])
def test_shards_sum_to_the_unsharded_result(ctx, R, precision):
    g = synth.disjoint_union([synth.powerlaw_cm(40000, 2.1, 2, 8000, 61), synth.watts_strogatz(5000, 10, 0.1, 62),
                              synth.complete(40), synth.star(700), synth.path(3)])
    rp, ci, tot, _, ranges, frac = _shards(ctx, g, R, precision)
    _check_ranges(g, R, ranges)
    got = _finalize(ctx, tot, frac, precision)
    ref = _unsharded(ctx, rp, ci, precision)
    for k in ("n_clusters", "s", "triangles", "flag"):
        np.testing.assert_array_equal(got[k], ref[k])
    _close(got["ef"], ref["ef"], precision)


@pytest.mark.parametrize("wedge_mode", [0, 1])
def test_shards_match_algorithm_1(ctx, wedge_mode):
    g = synth.disjoint_union([synth.barabasi_albert(3000, 6, 63), synth.rmat(11, 8, 64)])
    ref = oracle.alg1(g)
    t = oracle.triangles(g)
    rp, ci, tot, parts, ranges, frac = _shards(ctx, g, 5, "fp64", wedge_mode)
    _check_ranges(g, 5, ranges)
    # each shard's closed forms: Algorithm 1's N and S + 8t on its own nodes, zero elsewhere
    for (lo, hi), p in zip(ranges, parts):
        own = np.zeros(g.n, bool)
        own[lo:hi] = True
        np.testing.assert_array_equal(p["n_clusters"].cpu().numpy(), np.where(own, ref["N"], 0))
        np.testing.assert_array_equal(p["s_open"].cpu().numpy(), np.where(own, ref["S"] + 8 * t, 0))
    got = _finalize(ctx, tot, frac, "fp64")
    np.testing.assert_array_equal(got["n_clusters"], ref["N"])
    np.testing.assert_array_equal(got["s"], ref["S"])
    np.testing.assert_array_equal(got["triangles"], t)
    np.testing.assert_array_equal(got["flag"], ref["flag"])
    np.testing.assert_allclose(got["ef"], ref["EF"], rtol=1e-9, atol=1e-12)


def _bipartite(n, m_edges, seed):
    """Triangle-free: random edges between the two halves, hub-heavy on one side, ids shuffled."""
    rng = np.random.default_rng(seed)
    h = n // 2
    w = 1.0 / np.arange(1, h + 1)
    a = rng.choice(h, size=m_edges, p=w / w.sum())
    b = h + rng.integers(0, n - h, size=m_edges)
    g = synth.from_edges(n, np.stack([a, b], axis=1))
    return synth.relabel(g, rng.permutation(n))


def test_each_shard_matches_the_oracle_partial_on_a_triangle_free_graph(ctx):
    g = _bipartite(3000, 5000, 65)   # degrees up to about 600: small, mid and hub middle nodes
    R = 4
    _, _, _, parts, ranges, _ = _shards(ctx, g, R, "fp64")
    _check_ranges(g, R, ranges)
    for (lo, hi), p in zip(ranges, parts):
        ref = oshard.partials(g, lo, hi)
        assert not p["q"].any().item() and not p["triangles"].any().item()
        np.testing.assert_allclose(p["t"].cpu().numpy(), ref["T"], rtol=1e-12, atol=1e-9)


def test_more_shards_than_nodes(ctx):
    g = synth.disjoint_union([synth.complete(5), synth.cycle(6), synth.star(4)])
    R = g.n + 7
    rp, ci, tot, parts, ranges, frac = _shards(ctx, g, R, "fp64")
    _check_ranges(g, R, ranges)
    assert sum(1 for r in ranges if r[0] == r[1]) >= 7
    got = _finalize(ctx, tot, frac, "fp64")
    ref = oracle.alg1(g)
    np.testing.assert_array_equal(got["s"], ref["S"])
    np.testing.assert_allclose(got["ef"], ref["EF"], rtol=1e-9, atol=1e-12)


def test_errors(ctx):
    import torch
    import paper_2306_00606_gb300 as ef
    g = synth.erdos_renyi(300, 0.05, 66)
    rp, ci = _dev(g.row_ptr), _dev(g.col_idx)
    parts = ef.empty_partials(g.n, "cuda")
    for shard, R in ((2, 2), (-1, 2), (0, 0)):
        with pytest.raises(ef.EfError) as ei:
            ef.ef_compute_shard(ctx.handle, rp, ci, shard, R, parts)
        assert ei.value.code == ef.EF_ERR_ARG
    with pytest.raises(ef.EfError) as ei:   # a missing partial array
        ef.ef_compute_shard(ctx.handle, rp, ci, 0, 1, {k: v for k, v in parts.items() if k != "s_open"})
    assert ei.value.code == ef.EF_ERR_ARG
    frac, _ = ef.ef_compute_shard(ctx.handle, rp, ci, 0, 1, parts)
    for bad in (-1, 53):
        with pytest.raises(ef.EfError) as ei:
            ef.ef_finalize_partials(ctx.handle, parts, bad, ef=torch.empty(g.n, dtype=torch.float64, device="cuda"))
        assert ei.value.code == ef.EF_ERR_ARG
    # an edge stored in one row only: asymmetric, reported by the shard
    rows = [list(g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]) for v in range(g.n)]
    v = next(i for i in range(g.n) if rows[i])
    u = next(x for x in range(g.n) if x != v and x not in rows[v])
    rows[v] = sorted(rows[v] + [u])
    arp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    aci = np.concatenate(rows).astype(np.int32)
    with pytest.raises(ef.EfError) as ei:
        ef.ef_compute_shard(ctx.handle, _dev(arp), _dev(aci), 0, 2, parts)
    assert ei.value.code == ef.EF_ERR_GRAPH


def test_compute_sharded_single_rank(ctx):
    import paper_2306_00606_gb300 as ef
    g = synth.barabasi_albert(20000, 4, 67)
    rp, ci = _dev(g.row_ptr), _dev(g.col_idx)
    got = ef.compute_sharded(ctx.handle, rp, ci, 0, 1, outputs=("ef", "s"))
    ref = _unsharded(ctx, rp, ci, "fp64")
    np.testing.assert_array_equal(got["s"].cpu().numpy(), ref["s"])
    np.testing.assert_allclose(got["ef"].cpu().numpy(), ref["ef"], rtol=1e-9, atol=1e-12)
