"""GPU parity: libef (through the C ABI) against the CPU oracle.

Bar: cluster counts N_v, degree sums S_v, triangle counts t_v and degenerate
flags bit-exact; EF within 1e-9 relative on the FP64 path and 2e-5 absolute on
the FP32C path; T_v within 1e-10 relative (FP64) / 2e-6 relative (FP32C).
Sizes span several tiles and work items and ragged tails; the full-size
workloads are checked on sampled nodes (vertex-centric oracle) and on
properties that hold at any size.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from badgraphs import BAD_KINDS, bad_graph

pytestmark = pytest.mark.gpu

EF_RTOL64 = 1e-9
EF_ATOL32 = 2e-5


@pytest.fixture(scope="module")
def ctx():
    import paper_2306_00606_gb300 as ef
    c = ef.Context(0)
    yield c
    c.close()


def run(ctx, g, precision, **kw):
    import torch
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    out = ctx.compute(rp, ci, precision=precision,
                      outputs=("ef", "n_clusters", "s", "t", "triangles", "flag"), **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def assert_parity(got, ref, precision, nodes=None):
    sel = (lambda a: a) if nodes is None else (lambda a: a[nodes])
    np.testing.assert_array_equal(sel(got["n_clusters"]), ref["N"])
    np.testing.assert_array_equal(sel(got["s"]), ref["S"])
    np.testing.assert_array_equal(sel(got["flag"]), ref["flag"])
    if "tri" in ref:
        np.testing.assert_array_equal(sel(got["triangles"]), ref["tri"])
    ef, ref_ef = sel(got["ef"]), ref["EF"]
    if precision == "fp64":
        np.testing.assert_allclose(ef, ref_ef, rtol=EF_RTOL64, atol=1e-12)
        np.testing.assert_allclose(sel(got["t"]), ref["T"], rtol=1e-10, atol=1e-9)
    else:
        np.testing.assert_allclose(ef, ref_ef, rtol=0, atol=EF_ATOL32)
        np.testing.assert_allclose(sel(got["t"]), ref["T"], rtol=2e-6, atol=1e-3)


def alg1_ref(g):
    r = oracle.alg1(g)
    r["tri"] = oracle.triangles(g)
    return r


SPECIAL = {
    "K3": lambda: synth.complete(3), "K4": lambda: synth.complete(4), "K9": lambda: synth.complete(9),
    "K40": lambda: synth.complete(40), "K150": lambda: synth.complete(150),
    "star2": lambda: synth.star(2), "star33": lambda: synth.star(33), "star5000": lambda: synth.star(5000),
    "P5": lambda: synth.path(5), "C7": lambda: synth.cycle(7), "petersen": synth.petersen,
    "Q10": lambda: synth.hypercube(10), "K40_40": lambda: synth.complete_bipartite(40, 40),
    "K2+isolated": lambda: synth.from_edges(5, [(1, 3)]),
}


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
@pytest.mark.parametrize("name", list(SPECIAL))
def test_special_graphs(ctx, name, precision):
    g = SPECIAL[name]()
    assert_parity(run(ctx, g, precision), alg1_ref(g), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_er_workload_1(ctx, precision):
    """Erdos-Renyi G(2000, 0.004), the small workload, against literal Algorithm 1."""
    g = synth.workload(1)
    assert_parity(run(ctx, g, precision), alg1_ref(g), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_mixed_union(ctx, precision):
    g = synth.disjoint_union([synth.erdos_renyi(700, 0.02, 3), synth.barabasi_albert(3000, 3, 4),
                              synth.watts_strogatz(900, 8, 0.1, 5), synth.complete(3), synth.path(3),
                              synth.star(70), synth.rmat(9, 8, 6), synth.from_edges(3, [])])
    assert_parity(run(ctx, g, precision), alg1_ref(g), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_ba_many_work_items(ctx, precision):
    """BA n=20000, m=5: hubs with several hundred neighbours -> several CTA work items each."""
    g = synth.barabasi_albert(20000, 5, 11)
    assert g.degrees.max() > 2 * 256
    assert_parity(run(ctx, g, precision), alg1_ref(g), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_dense_triangles(ctx, precision):
    """Dense random graph: many triangles, triangle owners above the warp capacity."""
    g = synth.erdos_renyi(500, 0.5, 12)
    ref = alg1_ref(g)
    assert ref["tri"].max() > 1000
    assert_parity(run(ctx, g, precision), ref, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_powerlaw_hubs_beyond_one_tile(ctx, precision):
    """Power-law configuration model plus a hub joined to 5000 of its nodes: a middle node of
    degree > 4096 (several shared-memory tiles) among power-law neighbours."""
    g0 = synth.powerlaw_cm(20000, 2.3, 3, 1000, 13)
    src = np.repeat(np.arange(g0.n), np.diff(g0.row_ptr))
    e = np.stack([src, g0.col_idx], 1)
    e = e[e[:, 0] < e[:, 1]]
    spokes = np.random.default_rng(13).choice(g0.n, 5000, replace=False)
    hub = np.stack([np.full(5000, g0.n), spokes], 1)
    g = synth.from_edges(g0.n + 1, np.concatenate([e, hub]))
    assert g.degrees.max() > 4096
    ref = oracle.vertex(g)
    ref["tri"] = ref["t"]
    assert_parity(run(ctx, g, precision), ref, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
@pytest.mark.parametrize("r", [300, 3000, 6200])
def test_bipartite_closed_form(ctx, precision, r):
    """K_{r,r}: triangle-free r-regular, so every cluster has d = 3r-4 and EF = ln(2r(r-1)).
    r = 300: warp-level class kernel with every neighbour above its histogram range;
    r = 3000: CTA class kernel, classes in shared memory; r = 6200: classes spill to
    global memory, triangle owners span two shared-memory tiles."""
    g = synth.complete_bipartite(r, r)
    got = run(ctx, g, precision)
    N = 2 * r * (r - 1)
    assert np.all(got["n_clusters"] == N) and np.all(got["s"] == N * (3 * r - 4))
    assert np.all(got["triangles"] == 0) and np.all(got["flag"] == 0)
    tol = dict(rtol=EF_RTOL64, atol=0) if precision == "fp64" else dict(rtol=0, atol=EF_ATOL32)
    np.testing.assert_allclose(got["ef"], math.log(N), **tol)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_complete_closed_form_large(ctx, precision):
    """K_600: every cluster is a triangle of degree 3(n-3), EF = ln(2(n-1)(n-2))."""
    n = 600
    got = run(ctx, synth.complete(n), precision)
    N = 2 * (n - 1) * (n - 2)
    assert np.all(got["n_clusters"] == N) and np.all(got["s"] == N * 3 * (n - 3))
    assert np.all(got["triangles"] == (n - 1) * (n - 2) // 2)
    tol = dict(rtol=EF_RTOL64, atol=0) if precision == "fp64" else dict(rtol=0, atol=EF_ATOL32)
    np.testing.assert_allclose(got["ef"], math.log(N), **tol)


def _closed_counts(g):
    d = g.degrees
    src = np.repeat(np.arange(g.n), d)
    sig1 = np.bincount(src, weights=d[g.col_idx], minlength=g.n).astype(np.int64)
    return d * (d - 2) + sig1


def _sample(g, k_random, k_hub, rng):
    """The 20 largest hubs (degree up to ~1.9e4 on the power-law workloads,
    where FP32C's cancellation is worst), k_hub more spread over degree ranks
    20..419, k_random random nodes, and the smallest-degree node and both ends."""
    d = g.degrees
    order = np.argsort(-d, kind="stable")
    hubs = np.concatenate([order[:20], order[20:420][:: max(1, 400 // max(k_hub, 1))][:k_hub]])
    rnd = rng.choice(g.n, size=k_random, replace=False)
    return np.unique(np.concatenate([hubs, rnd, [order[-1], 0, g.n - 1]])).astype(np.int32)


_FULL_REF = {}


def _full_size_ref(idx):
    """The full-size workload, its sampled nodes and the vertex oracle on them (once per workload)."""
    if idx not in _FULL_REF:
        _FULL_REF.clear()   # one full-size graph held at a time
        g = synth.workload(idx)
        nodes = _sample(g, 48, 6, np.random.default_rng(7 if idx == "3b" else idx))
        ref = oracle.vertex(g, nodes)
        ref["tri"] = ref["t"]
        _FULL_REF[idx] = (g, nodes, ref)
    return _FULL_REF[idx]


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
@pytest.mark.parametrize("idx", [2, 3, "3b", 5])
def test_full_size_workloads_sampled(ctx, idx, precision):
    """BA n=1e6 m=5, the power-law model n=4e6 (minimum degree 3 and 6: 2.1e7
    and 4.4e7 undirected edges) and BA n=1.6e7 m=4 at full size: every node's
    N_v against its closed form, sum N = 4W, and sampled nodes (the 20
    largest hubs included) against the vertex-centric oracle."""
    g, nodes, ref = _full_size_ref(idx)
    got = run(ctx, g, precision)
    np.testing.assert_array_equal(got["n_clusters"], _closed_counts(g))
    assert int(got["n_clusters"].sum()) == 4 * g.wedges()
    assert int(got["triangles"].sum()) % 3 == 0
    assert_parity(got, ref, precision, nodes=nodes)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_direct_and_class_wedge_kernels_agree(ctx, precision):
    """The direct pairwise kernel and the degree-class kernels compute the same credits."""
    g = synth.powerlaw_cm(300000, 2.2, 3, 5000, 41)
    a = run(ctx, g, precision, wedge_mode=0)
    b = run(ctx, g, precision, wedge_mode=1)
    np.testing.assert_array_equal(a["s"], b["s"])
    if precision == "fp64":
        np.testing.assert_allclose(a["t"], b["t"], rtol=1e-12)
        np.testing.assert_allclose(a["ef"], b["ef"], rtol=1e-12)
    else:
        np.testing.assert_allclose(a["ef"], b["ef"], rtol=0, atol=EF_ATOL32)


def test_fp32c_tracks_fp64(ctx):
    g = synth.powerlaw_cm(200000, 2.3, 3, 3000, 21)
    a = run(ctx, g, "fp64")
    b = run(ctx, g, "fp32c")
    np.testing.assert_array_equal(a["s"], b["s"])
    np.testing.assert_allclose(b["ef"], a["ef"], rtol=0, atol=EF_ATOL32)


def test_repeatable_fp64(ctx):
    # integer outputs are exact; the end credits are FP64 sums in L2 whose
    # order varies between runs, so EF may differ by a few ulps
    g = synth.workload(1)
    a, b = run(ctx, g, "fp64"), run(ctx, g, "fp64")
    for k in ("n_clusters", "s", "triangles", "flag"):
        assert np.array_equal(a[k], b[k])
    np.testing.assert_allclose(a["ef"], b["ef"], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("bad", BAD_KINDS)
def test_invalid_graphs_rejected(ctx, bad):
    import torch
    import paper_2306_00606_gb300 as ef
    rp, ci = bad_graph(bad)
    with pytest.raises(ef.EfError) as ei:
        ctx.compute(torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda(), outputs=("ef",))
    assert ei.value.code == ef.EF_ERR_GRAPH


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_rmat_graph(ctx, precision):
    # skewed R-MAT (a, b, c = .57, .19, .19): many hubs and triangles
    g = synth.rmat(12, 8, 31)
    assert_parity(run(ctx, g, precision), alg1_ref(g), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_column_array_not_16_byte_aligned(ctx, precision):
    """col_idx and row_ptr as views that start 4 bytes into their buffers (only 4-byte
    alignment): every read of the caller's arrays is a 4-byte load, so the results are the
    oracle's as for aligned input."""
    import torch
    g = synth.disjoint_union([synth.powerlaw_cm(20000, 2.1, 2, 3000, 71), synth.complete(40), synth.path(3)])
    rbuf = torch.empty(g.n + 2, dtype=torch.int32, device="cuda")
    cbuf = torch.empty(g.nnz + 1, dtype=torch.int32, device="cuda")
    rbuf[1:] = torch.from_numpy(g.row_ptr).cuda()
    cbuf[1:] = torch.from_numpy(g.col_idx).cuda()
    rp, ci = rbuf[1:], cbuf[1:]
    assert rp.data_ptr() % 16 and ci.data_ptr() % 16
    out = ctx.compute(rp, ci, precision=precision, outputs=("ef", "n_clusters", "s", "t", "triangles", "flag"))
    torch.cuda.synchronize()
    assert_parity({k: v.cpu().numpy() for k, v in out.items()}, alg1_ref(g), precision)


def test_empty_graph(ctx):
    import torch
    out = ctx.compute(torch.zeros(1, dtype=torch.int32, device="cuda"),
                      torch.zeros(0, dtype=torch.int32, device="cuda"), outputs=("ef",))
    assert out["ef"].numel() == 0


def test_host_io_matches_device(ctx):
    import paper_2306_00606_gb300 as ef
    g = synth.barabasi_albert(5000, 4, 3)
    dev = run(ctx, g, "fp64")
    host = {k: np.zeros(g.n, dt) for k, dt in (("ef", np.float64), ("s", np.int64), ("n_clusters", np.int64))}
    ef.ef_compute_ex(ctx.handle, g.row_ptr, g.col_idx, precision="fp64", host_io=True, **host)
    assert np.array_equal(host["s"], dev["s"]) and np.array_equal(host["n_clusters"], dev["n_clusters"])
    np.testing.assert_allclose(host["ef"], dev["ef"], rtol=1e-13, atol=1e-13)


def test_async_calls_match_synchronous(ctx):
    """async = 1: device I/O without validation, and host I/O with validation on two contexts whose
    calls alternate (one call's copies beside the other's kernels); every result read after
    ef_sync equals the synchronous call's."""
    import torch
    import paper_2306_00606_gb300 as ef
    g = synth.barabasi_albert(20000, 4, 5)
    ref = run(ctx, g, "fp64")
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    ef.ef_compute_ex(ctx.handle, rp, ci, precision="fp64", trust_input=True, async_=True, ef=out)
    ef.ef_sync(ctx.handle)
    np.testing.assert_allclose(out.cpu().numpy(), ref["ef"], rtol=1e-13, atol=1e-13)
    h_rp = torch.from_numpy(g.row_ptr).pin_memory()
    h_ci = torch.from_numpy(g.col_idx).pin_memory()
    outs = [torch.zeros(g.n, dtype=torch.float64).pin_memory() for _ in range(4)]
    s_out = [torch.zeros(g.n, dtype=torch.int64).pin_memory() for _ in range(4)]
    with ef.Context(0, torch.cuda.Stream()) as ctx2:
        ctxs = (ctx, ctx2)
        for i in range(4):
            ef.ef_compute_ex(ctxs[i % 2].handle, h_rp, h_ci, precision="fp64", host_io=True, async_=True,
                             ef=outs[i], s=s_out[i])
        ef.ef_sync(ctx.handle)
        ef.ef_sync(ctx2.handle)
    for i in range(4):
        assert np.array_equal(s_out[i].numpy(), ref["s"])
        np.testing.assert_allclose(outs[i].numpy(), ref["ef"], rtol=1e-13, atol=1e-13)


def test_plain_ef_compute_entry(ctx):
    import torch
    import paper_2306_00606_gb300 as ef
    g = synth.workload(1)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    ef.ef_compute(rp, ci, out)
    np.testing.assert_allclose(out.cpu().numpy(), oracle.alg1(g)["EF"], rtol=EF_RTOL64, atol=1e-12)


def test_profile_stats(ctx):
    g = synth.barabasi_albert(50000, 5, 1)
    ctx.stats(reset=True)
    run(ctx, g, "fp32c", profile=True)
    st = ctx.stats(reset=True)
    assert st["calls"] == 1 and st["total_ms"] > 0 and st["wedge_big_ms"] > 0 and st["tri_pairs_ms"] > 0


@pytest.mark.parametrize("variant", [1])
def test_pair_test_variants_agree(ctx, variant):
    """The other pair-test kernel variant lists the same triangles: exact per-node
    counts against the oracle and the same N, S and EF as variant 0, on
    graphs whose out-lists run far past a warp step's staged entries (K_600:
    out-degrees up to 599; dense ER; power-law hubs; R-MAT)."""
    import paper_2306_00606_gb300 as ef
    graphs = [synth.complete(600), synth.erdos_renyi(500, 0.5, 12), synth.powerlaw_cm(20000, 2.1, 2, 3000, 22),
              synth.rmat(12, 8, 31)]
    try:
        for g in graphs:
            ef.ef_set_tuning(ctx.handle, None)
            base = run(ctx, g, "fp64")
            ef.ef_set_tuning(ctx.handle, dict(ef.ef_get_tuning(ctx.handle), tri_variant=variant))
            got = run(ctx, g, "fp64")
            np.testing.assert_array_equal(got["triangles"], oracle.triangles(g))
            for k in ("n_clusters", "s", "triangles", "flag"):
                np.testing.assert_array_equal(got[k], base[k])
            np.testing.assert_allclose(got["ef"], base["ef"], rtol=1e-12, atol=1e-12)
    finally:
        ef.ef_set_tuning(ctx.handle, None)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_maximum_degree_star(ctx, precision):
    """The largest degree a validated call accepts, EF_MAX_DEGREE = 2^20: a
    star K_{1,k} with k = 2^20 leaves has S = k(k-1)(k-2) ~ 1.2e18 at its
    centre (its 64-bit sums near the top of their range) and closed forms
    EF = ln(k(k-1)) at the centre and ln(k-1) at every leaf; one more leaf
    is refused with EF_ERR_UNSUPPORTED."""
    import torch
    import paper_2306_00606_gb300 as ef
    k = ef.EF_MAX_DEGREE
    g = synth.star(k)
    got = run(ctx, g, precision)
    assert got["n_clusters"][0] == k * (k - 1) and got["s"][0] == k * (k - 1) * (k - 2)
    assert np.all(got["n_clusters"][1:] == k - 1) and np.all(got["s"][1:] == (k - 1) * (k - 2))
    ref = np.concatenate([[math.log(k * (k - 1))], np.full(k, math.log(k - 1))])
    tol = dict(rtol=EF_RTOL64, atol=0) if precision == "fp64" else dict(rtol=0, atol=EF_ATOL32)
    np.testing.assert_allclose(got["ef"], ref, **tol)
    big = synth.star(k + 1)
    with pytest.raises(ef.EfError) as ei:
        ctx.compute(torch.from_numpy(big.row_ptr).cuda(), torch.from_numpy(big.col_idx).cuda(), outputs=("ef",))
    assert ei.value.code == ef.EF_ERR_UNSUPPORTED and "EF_MAX_DEGREE" in str(ei.value)


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_full_size_relabel_invariance(ctx, precision):
    """Relabelling the nodes of the 4M-node power-law graph by a random
    permutation permutes every output: N, S, triangles and flags exactly, EF
    within the precision's bar.  The relabelled graph moves the hubs to other
    ids, so the out-list layout, the work bins' order and every kernel's
    schedule change, while Algorithm 1's result may not."""
    g, _, _ = _full_size_ref(3)
    perm = np.random.default_rng(99).permutation(g.n)
    h = synth.relabel(g, perm)
    a = run(ctx, g, precision)
    b = run(ctx, h, precision)
    for k in ("n_clusters", "s", "triangles", "flag"):
        np.testing.assert_array_equal(b[k][perm], a[k])
    tol = dict(rtol=2 * EF_RTOL64, atol=1e-12) if precision == "fp64" else dict(rtol=0, atol=2 * EF_ATOL32)
    np.testing.assert_allclose(b["ef"][perm], a["ef"], **tol)


@pytest.mark.parametrize("precision", ["fp32c", "fp64"])
def test_rmat_sweep_graph_sampled(ctx, precision):
    """The densest graph of the R-MAT sweep (2^16 nodes, 32 edges per node,
    a, b, c = .57, .19, .19): sampled nodes, the 20 largest hubs included,
    against the vertex-centric oracle; every node's N in closed form."""
    g = synth.rmat(16, 32, synth.SEED_BASE + 132)
    got = run(ctx, g, precision)
    np.testing.assert_array_equal(got["n_clusters"], _closed_counts(g))
    nodes = _sample(g, 60, 6, np.random.default_rng(5))
    ref = oracle.vertex(g, nodes)
    ref["tri"] = ref["t"]
    assert_parity(got, ref, precision, nodes=nodes)
