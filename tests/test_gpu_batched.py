"""Batched EF, CUDA-graph replay and launch parameters, through the C ABI.

A batch is one CSR over the disjoint union of its graphs.  EF is local:
Algorithm 1 credits a node only for clusters that contain it, and a cluster
lies inside one connected component.  So the batched result must equal each
graph computed alone:
- N, S, t and the flags exactly;
- EF within the same bars as the single-graph parity tests.

The oracle checks the union directly.  Replayed CUDA graphs and every
choice of launch parameters must give the same results as the plain path.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

EF_RTOL64 = 1e-9
EF_ATOL32 = 2e-5
OUTS = ("ef", "n_clusters", "s", "t", "triangles", "flag")


@pytest.fixture(scope="module")
def ctx():
    import paper_2306_00606_gb300 as ef
    c = ef.Context(0)
    yield c
    c.close()


def _alloc(n):
    import torch
    dt = dict(ef=torch.float64, n_clusters=torch.int64, s=torch.int64, t=torch.float64, triangles=torch.int64,
              flag=torch.uint8)
    return {k: torch.full((n,), 7, dtype=dt[k], device="cuda") for k in OUTS}


def _host(res):
    import torch
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in res.items()}


def run_batched(ctx, g, off, precision, **kw):
    import torch
    import paper_2306_00606_gb300 as ef
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    res = _alloc(g.n)
    ef.ef_compute_batched(ctx.handle, rp, ci, off, precision=precision, **res, **kw)
    return _host(res)


def run_one(ctx, rp_h, ci_h, precision, **kw):
    import torch
    import paper_2306_00606_gb300 as ef
    rp = torch.from_numpy(np.ascontiguousarray(rp_h)).cuda()
    ci = torch.from_numpy(np.ascontiguousarray(ci_h)).cuda()
    res = _alloc(len(rp_h) - 1)
    ef.ef_compute_ex(ctx.handle, rp, ci, precision=precision, **res, **kw)
    return _host(res)


def _same(a, b, precision, rtol64=1e-13):
    for k in ("n_clusters", "s", "triangles", "flag"):
        np.testing.assert_array_equal(a[k], b[k])
    if precision == "fp64":
        np.testing.assert_allclose(a["ef"], b["ef"], rtol=rtol64, atol=1e-13)
    else:
        np.testing.assert_allclose(a["ef"], b["ef"], rtol=0, atol=EF_ATOL32)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_batched_equals_graphs_alone(ctx, precision):
    b = synth.ws_batch(40, 30, 700, 4, 12, 0.1, 11)
    off = b.graph_off
    got = run_batched(ctx, b, off, precision)
    for k in range(len(off) - 1):
        lo, hi = int(off[k]), int(off[k + 1])
        e0, e1 = int(b.row_ptr[lo]), int(b.row_ptr[hi])
        rp_k = b.row_ptr[lo:hi + 1] - e0
        ci_k = b.col_idx[e0:e1] - lo
        alone = run_one(ctx, rp_k, ci_k, precision)
        _same({key: v[lo:hi] for key, v in got.items()}, alone, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_batched_against_oracle(ctx, precision):
    parts = [synth.erdos_renyi(300, 0.03, 3), synth.barabasi_albert(500, 4, 4), synth.complete(9), synth.star(30),
             synth.path(3), synth.watts_strogatz(400, 8, 0.1, 5)]
    u = synth.disjoint_union(parts)
    off = np.cumsum([0] + [p.n for p in parts]).astype(np.int64)
    got = run_batched(ctx, u, off, precision)
    ref = oracle.alg1(u)
    np.testing.assert_array_equal(got["n_clusters"], ref["N"])
    np.testing.assert_array_equal(got["s"], ref["S"])
    np.testing.assert_array_equal(got["flag"], ref["flag"])
    np.testing.assert_array_equal(got["triangles"], oracle.triangles(u))
    if precision == "fp64":
        np.testing.assert_allclose(got["ef"], ref["EF"], rtol=EF_RTOL64, atol=1e-12)
    else:
        np.testing.assert_allclose(got["ef"], ref["EF"], rtol=0, atol=EF_ATOL32)


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_full_size_ws_batch_sampled(ctx, precision):
    """The 4096-graph Watts-Strogatz workload at full size, run as the bench
    runs it (one ef_compute_batched call replayed as a CUDA graph): every
    node's N against its closed form, sum N = 4W, and sampled nodes (random,
    the ends of the largest and smallest graphs) against the vertex oracle."""
    import torch
    import paper_2306_00606_gb300 as ef
    g = synth.workload(4)
    off = g.graph_off
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    res = _alloc(g.n)
    for _ in range(2):   # the second call replays the captured graph
        ef.ef_compute_batched(ctx.handle, rp, ci, off, precision=precision, graph=True, **res)
    got = _host(res)
    d = np.diff(g.row_ptr).astype(np.int64)
    sig1 = np.add.reduceat(d[g.col_idx], g.row_ptr[:-1].astype(np.int64), dtype=np.int64)
    np.testing.assert_array_equal(got["n_clusters"], d * (d - 2) + sig1)
    assert int(got["n_clusters"].sum()) == 4 * g.wedges()
    sizes = np.diff(off)
    big, small = int(np.argmax(sizes)), int(np.argmin(sizes))
    rng = np.random.default_rng(4)
    nodes = np.unique(np.concatenate([rng.choice(g.n, 48, replace=False), [off[big], off[big + 1] - 1],
                                      [off[small], off[small + 1] - 1], [int(np.argmax(d))]])).astype(np.int32)
    ref = oracle.vertex(g, nodes)
    for k, r in (("n_clusters", "N"), ("s", "S"), ("triangles", "t"), ("flag", "flag")):
        np.testing.assert_array_equal(got[k][nodes], ref[r])
    if precision == "fp64":
        np.testing.assert_allclose(got["ef"][nodes], ref["EF"], rtol=EF_RTOL64, atol=1e-12)
    else:
        np.testing.assert_allclose(got["ef"][nodes], ref["EF"], rtol=0, atol=EF_ATOL32)


def test_batched_rejects_edge_between_graphs(ctx):
    import paper_2306_00606_gb300 as ef
    parts = [synth.cycle(20), synth.cycle(30)]
    u = synth.disjoint_union(parts)
    # the same union, but cut after node 10 instead of 20: edges now cross
    with pytest.raises(ef.EfError) as ei:
        run_batched(ctx, u, np.array([0, 10, 50], dtype=np.int64), "fp64")
    assert ei.value.code == ef.EF_ERR_GRAPH and "between-graphs" in ef.ef_last_error(ctx.handle)
    run_batched(ctx, u, np.array([0, 20, 50], dtype=np.int64), "fp64")   # the right cut passes


@pytest.mark.parametrize("leaves", [100, 3000])
def test_batched_rejects_edge_between_graphs_at_big_rows(ctx, leaves):
    """The cross-graph check where a warp (degree 101) or a block (degree 3001) walks the row: two
    stars whose centres are joined, cut between the centres, so that the centres' rows hold the
    only entries outside their graph."""
    import paper_2306_00606_gb300 as ef
    c1, c2 = leaves, leaves + 1
    edges = [(i, c1) for i in range(leaves)] + [(c1, c2)] + [(c2, c2 + 1 + i) for i in range(leaves)]
    g = synth.from_edges(2 * leaves + 2, edges)
    with pytest.raises(ef.EfError) as ei:
        run_batched(ctx, g, np.array([0, c2, 2 * leaves + 2], dtype=np.int64), "fp64")
    assert ei.value.code == ef.EF_ERR_GRAPH and "between-graphs" in ef.ef_last_error(ctx.handle)
    run_batched(ctx, g, np.array([0, 2 * leaves + 2], dtype=np.int64), "fp64")


def test_batched_rejects_bad_offsets(ctx):
    import paper_2306_00606_gb300 as ef
    u = synth.cycle(10)
    for off in ([1, 10], [0, 6, 4, 10]):
        with pytest.raises(ef.EfError) as ei:
            run_batched(ctx, u, np.array(off, dtype=np.int64), "fp64")
        assert ei.value.code == ef.EF_ERR_ARG


@pytest.mark.parametrize("trust", [False, True])
def test_graph_replay_matches_plain_path(ctx, trust):
    import torch
    import paper_2306_00606_gb300 as ef
    g = synth.powerlaw_cm(30000, 2.3, 3, 800, 21)
    plain = run_one(ctx, g.row_ptr, g.col_idx, "fp32c")
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    res = _alloc(g.n)
    ctx.stats(reset=True)
    for i in range(3):
        for v in res.values():
            v.fill_(7)
        ef.ef_compute_ex(ctx.handle, rp, ci, precision="fp32c", graph=True, trust_input=trust, **res)
        _same(_host(res), plain, "fp32c")
    assert ctx.stats(reset=True)["graph_replays"] == 2
    # another output buffer is another graph: captured again, still right
    res2 = _alloc(g.n)
    ef.ef_compute_ex(ctx.handle, rp, ci, precision="fp32c", graph=True, trust_input=trust, **res2)
    _same(_host(res2), plain, "fp32c")
    assert ctx.stats(reset=True)["graph_replays"] == 0


TUNINGS = [dict(row_thread_max=8, hub_min=513, tri_variant=0, grid_per_sm=64, layout=0),
           dict(row_thread_max=32, hub_min=129, tri_variant=1, grid_per_sm=16, layout=1),
           dict(row_thread_max=1, hub_min=33, tri_variant=1, grid_per_sm=1, layout=2),
           dict(row_thread_max=16, hub_min=257, tri_variant=0, grid_per_sm=256, layout=1)]


@pytest.mark.parametrize("tuning", TUNINGS)
def test_tunings_on_a_graph_without_rows_above_32(ctx, tuning):
    """No node of degree > 32: the row passes keep node order and the
    orientation's one-thread rows gather eight records at a time; with
    row_thread_max below the degrees, rows go to the warp path instead."""
    import paper_2306_00606_gb300 as ef
    g = synth.disjoint_union([synth.watts_strogatz(6000, 12, 0.1, 23), synth.erdos_renyi(3000, 0.004, 24)])
    assert g.degrees.max() <= 32
    ef.ef_set_tuning(ctx.handle, None)
    base = run_one(ctx, g.row_ptr, g.col_idx, "fp64")
    ref = oracle.alg1(g)
    np.testing.assert_array_equal(base["n_clusters"], ref["N"])
    np.testing.assert_array_equal(base["s"], ref["S"])
    np.testing.assert_array_equal(base["triangles"], oracle.triangles(g))
    np.testing.assert_allclose(base["ef"], ref["EF"], rtol=EF_RTOL64, atol=1e-12)
    ef.ef_set_tuning(ctx.handle, tuning)
    try:
        _same(run_one(ctx, g.row_ptr, g.col_idx, "fp64"), base, "fp64")
    finally:
        ef.ef_set_tuning(ctx.handle, None)


@pytest.mark.parametrize("tuning", TUNINGS)
def test_tunings_give_the_same_results(ctx, tuning):
    import paper_2306_00606_gb300 as ef
    g = synth.powerlaw_cm(20000, 2.1, 2, 3000, 22)
    ef.ef_set_tuning(ctx.handle, None)
    base = run_one(ctx, g.row_ptr, g.col_idx, "fp64")
    ef.ef_set_tuning(ctx.handle, tuning)
    try:
        assert ef.ef_get_tuning(ctx.handle) == tuning
        _same(run_one(ctx, g.row_ptr, g.col_idx, "fp64"), base, "fp64")
    finally:
        ef.ef_set_tuning(ctx.handle, None)


def test_set_tuning_rejects_out_of_range(ctx):
    import paper_2306_00606_gb300 as ef
    before = ef.ef_get_tuning(ctx.handle)
    for bad in (dict(row_thread_max=0), dict(row_thread_max=33), dict(hub_min=32), dict(hub_min=514),
                dict(tri_variant=2), dict(grid_per_sm=0), dict(layout=3), dict(layout=-1)):
        t = dict(before, **bad)
        with pytest.raises(ef.EfError) as ei:
            ef.ef_set_tuning(ctx.handle, t)
        assert ei.value.code == ef.EF_ERR_ARG
    assert ef.ef_get_tuning(ctx.handle) == before


def test_autotune_keeps_a_valid_tuning_and_results(ctx):
    import torch
    import paper_2306_00606_gb300 as ef
    g = synth.barabasi_albert(30000, 5, 23)
    base = run_one(ctx, g.row_ptr, g.col_idx, "fp32c")
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    try:
        best = ef.ef_autotune(ctx.handle, rp, ci, precision="fp32c", reps=2)
        assert ef.ef_get_tuning(ctx.handle) == best
        assert 1 <= best["row_thread_max"] <= 32 and 33 <= best["hub_min"] <= 513
        _same(run_one(ctx, g.row_ptr, g.col_idx, "fp32c"), base, "fp32c")
    finally:
        ef.ef_set_tuning(ctx.handle, None)
