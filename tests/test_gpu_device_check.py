"""Validation on the device (ef_options.device_check), through the C ABI.

The row passes validate the graph as before, but no readback follows them: a
one-thread kernel stores the validation bits where every later kernel reads
them first, so on invalid input those kernels do nothing, and the host reads
the bits once the call's work is done.  Then:
- results equal the oracle's (N, S, t and flags exactly, EF within the
  bars of the parity tests), with and without a CUDA graph, for one graph
  and for a batch;
- the whole validated call is one replayed graph (validation included);
- every kind of malformed graph gives EF_ERR_GRAPH and leaves the outputs
  unwritten, and the context stays usable;
- asynchronous calls report a failed validation at the next ef_sync;
- a maximum degree above EF_MAX_DEGREE gives EF_ERR_UNSUPPORTED, and one at
  the limit (the f table at its largest size) is exact.
"""
import math

import numpy as np
import pytest

import synth
from badgraphs import BAD_KINDS, bad_graph
from test_gpu_parity import EF_ATOL32, EF_RTOL64, alg1_ref, assert_parity

pytestmark = pytest.mark.gpu

OUTS = ("ef", "n_clusters", "s", "t", "triangles", "flag")


@pytest.fixture(scope="module")
def ctx():
    import paper_2306_00606_gb300 as ef
    c = ef.Context(0)
    yield c
    c.close()


def _alloc(n, fill=7):
    import torch
    dt = dict(ef=torch.float64, n_clusters=torch.int64, s=torch.int64, t=torch.float64, triangles=torch.int64,
              flag=torch.uint8)
    return {k: torch.full((n,), fill, dtype=dt[k], device="cuda") for k in OUTS}


def _host(res):
    import torch
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in res.items()}


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


GRAPHS = {
    "mixed": lambda: synth.disjoint_union([synth.erdos_renyi(600, 0.01, 1), synth.barabasi_albert(900, 4, 2),
                                           synth.complete(7), synth.star(40), synth.path(3), synth.complete(3)]),
    "powerlaw_hubs": lambda: synth.powerlaw_cm(20000, 2.1, 2, 3000, 22),
    "rmat": lambda: synth.rmat(12, 8, 31),
    "ws_lattice": lambda: synth.watts_strogatz(5000, 10, 0.1, 7),
}


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
@pytest.mark.parametrize("name", list(GRAPHS))
def test_device_check_matches_oracle(ctx, name, precision, graph):
    import paper_2306_00606_gb300 as ef
    g = GRAPHS[name]()
    res = _alloc(g.n)
    ef.ef_compute_ex(ctx.handle, _dev(g.row_ptr), _dev(g.col_idx), precision=precision, device_check=True,
                     graph=graph, **res)
    assert_parity(_host(res), alg1_ref(g), precision)


def test_device_checked_call_is_one_replayed_graph(ctx):
    """With graph = 1 the validated call (validation, gate, part B) is captured once and replayed."""
    import paper_2306_00606_gb300 as ef
    g = synth.powerlaw_cm(30000, 2.3, 3, 800, 21)
    ref = alg1_ref(g)
    rp, ci = _dev(g.row_ptr), _dev(g.col_idx)
    res = _alloc(g.n)
    ctx.stats(reset=True)
    for _ in range(3):
        for v in res.values():
            v.fill_(7)
        ef.ef_compute_ex(ctx.handle, rp, ci, precision="fp32c", graph=True, device_check=True, **res)
        assert_parity(_host(res), ref, "fp32c")
    assert ctx.stats(reset=True)["graph_replays"] == 2


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("bad", BAD_KINDS)
def test_device_check_rejects_invalid_graphs(ctx, bad, graph):
    import paper_2306_00606_gb300 as ef
    rp, ci = bad_graph(bad)
    n = len(rp) - 1
    res = _alloc(n, fill=-7)
    for _ in range(2):   # with graph = 1 the second call replays the captured graph
        with pytest.raises(ef.EfError) as ei:
            ef.ef_compute_ex(ctx.handle, _dev(rp), _dev(ci), precision="fp64", device_check=True, graph=graph,
                             **res)
        assert ei.value.code == ef.EF_ERR_GRAPH
    for k, v in _host(res).items():
        assert np.all(v == np.array(-7).astype(v.dtype)), f"{k} written by a call that failed validation"
    # the context stays usable
    g = synth.erdos_renyi(300, 0.05, 2)
    ok = _alloc(g.n)
    ef.ef_compute_ex(ctx.handle, _dev(g.row_ptr), _dev(g.col_idx), precision="fp64", device_check=True,
                     graph=graph, **ok)
    assert_parity(_host(ok), alg1_ref(g), "fp64")


def test_device_check_async_reports_at_sync(ctx):
    """async = 1: a failed validation comes back from the next ef_sync (once), and a valid call
    queued after it on the same context is still right."""
    import paper_2306_00606_gb300 as ef
    rp, ci = bad_graph("asym")
    bad_out = _alloc(len(rp) - 1, fill=-7)
    ef.ef_compute_ex(ctx.handle, _dev(rp), _dev(ci), precision="fp64", device_check=True, async_=True, **bad_out)
    g = synth.barabasi_albert(20000, 4, 5)
    res = _alloc(g.n)
    ef.ef_compute_ex(ctx.handle, _dev(g.row_ptr), _dev(g.col_idx), precision="fp64", device_check=True,
                     async_=True, **res)
    with pytest.raises(ef.EfError) as ei:
        ef.ef_sync(ctx.handle)
    assert ei.value.code == ef.EF_ERR_GRAPH and "asymmetric" in ef.ef_last_error(ctx.handle)
    assert_parity(_host(res), alg1_ref(g), "fp64")
    assert np.all(_host(bad_out)["ef"] == -7.0)
    ef.ef_sync(ctx.handle)   # reported once: nothing pending now
    ok = _alloc(g.n)
    ef.ef_compute_ex(ctx.handle, _dev(g.row_ptr), _dev(g.col_idx), precision="fp32c", device_check=True,
                     async_=True, graph=True, **ok)
    ef.ef_sync(ctx.handle)
    assert_parity(_host(ok), alg1_ref(g), "fp32c")


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_device_check_degree_limit(ctx, precision):
    """A star with EF_MAX_DEGREE leaves (the f table at its largest, 3 * 2^20 + 1 entries, sized
    without a readback) is exact; one more leaf gives EF_ERR_UNSUPPORTED."""
    import paper_2306_00606_gb300 as ef
    k = ef.EF_MAX_DEGREE
    g = synth.star(k)
    res = _alloc(g.n)
    ef.ef_compute_ex(ctx.handle, _dev(g.row_ptr), _dev(g.col_idx), precision=precision, device_check=True, **res)
    got = _host(res)
    assert got["n_clusters"][0] == k * (k - 1) and got["s"][0] == k * (k - 1) * (k - 2)
    ref = np.concatenate([[math.log(k * (k - 1))], np.full(k, math.log(k - 1))])
    tol = dict(rtol=EF_RTOL64, atol=0) if precision == "fp64" else dict(rtol=0, atol=EF_ATOL32)
    np.testing.assert_allclose(got["ef"], ref, **tol)
    big = synth.star(k + 1)
    out = _alloc(big.n, fill=-7)
    with pytest.raises(ef.EfError) as ei:
        ef.ef_compute_ex(ctx.handle, _dev(big.row_ptr), _dev(big.col_idx), precision=precision,
                         device_check=True, **out)
    assert ei.value.code == ef.EF_ERR_UNSUPPORTED and "EF_MAX_DEGREE" in str(ei.value)
    assert np.all(_host(out)["ef"] == -7.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_device_check_batched(ctx, precision):
    """A batch in one replayed graph with validation on the device: equal to the oracle on the union;
    a cut that puts edges between graphs is refused."""
    import paper_2306_00606_gb300 as ef
    parts = [synth.watts_strogatz(800 + 150 * i, 4 + 2 * (i % 5), 0.1, 40 + i) for i in range(12)]
    parts += [synth.barabasi_albert(3000, 5, 60), synth.complete(30), synth.star(700)]
    u = synth.disjoint_union(parts)
    off = np.concatenate([[0], np.cumsum([p.n for p in parts])]).astype(np.int64)
    rp, ci = _dev(u.row_ptr), _dev(u.col_idx)
    for _ in range(2):
        res = _alloc(u.n)
        ef.ef_compute_batched(ctx.handle, rp, ci, off, precision=precision, graph=True, device_check=True, **res)
        assert_parity(_host(res), alg1_ref(u), precision)
    cyc = synth.disjoint_union([synth.cycle(20), synth.cycle(30)])
    res = _alloc(cyc.n, fill=-7)
    with pytest.raises(ef.EfError) as ei:
        ef.ef_compute_batched(ctx.handle, _dev(cyc.row_ptr), _dev(cyc.col_idx), np.array([0, 10, 50], np.int64),
                              precision=precision, graph=True, device_check=True, **res)
    assert ei.value.code == ef.EF_ERR_GRAPH and "between-graphs" in ef.ef_last_error(ctx.handle)
    assert np.all(_host(res)["ef"] == -7.0)


def test_device_check_host_buffers_two_contexts_in_flight(ctx):
    """The end-to-end form of the benchmark: host buffers, validation on the device, one replayed
    graph per call, asynchronous calls alternating between two contexts on two streams (one call's
    copies beside the other's kernels); every result read after ef_sync is Algorithm 1's."""
    import torch
    import paper_2306_00606_gb300 as ef
    g = synth.barabasi_albert(20000, 4, 5)
    ref = alg1_ref(g)
    h_rp = torch.from_numpy(g.row_ptr).pin_memory()
    h_ci = torch.from_numpy(g.col_idx).pin_memory()
    outs = [torch.zeros(g.n, dtype=torch.float64).pin_memory() for _ in range(6)]
    s_out = [torch.zeros(g.n, dtype=torch.int64).pin_memory() for _ in range(6)]
    with ef.Context(0, torch.cuda.Stream()) as ctx2:
        ctxs = (ctx, ctx2)
        for i in range(6):
            ef.ef_compute_ex(ctxs[i % 2].handle, h_rp, h_ci, precision="fp64", host_io=True, async_=True,
                             device_check=True, graph=True, ef=outs[i], s=s_out[i])
        ef.ef_sync(ctx.handle)
        ef.ef_sync(ctx2.handle)
    for i in range(6):
        np.testing.assert_array_equal(s_out[i].numpy(), ref["S"])
        np.testing.assert_allclose(outs[i].numpy(), ref["EF"], rtol=EF_RTOL64, atol=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_device_check_direct_kernel_and_profile(ctx, precision):
    """The direct pairwise wedge kernel (wedge_mode 1, its item counts and reduction gated too) and a
    profiled call (per-pass events, the gate kernel counted) with validation on the device: results
    are Algorithm 1's, and a malformed graph is still refused with the outputs left as they were."""
    import paper_2306_00606_gb300 as ef
    g = synth.powerlaw_cm(20000, 2.1, 2, 3000, 22)
    ref = alg1_ref(g)
    for kw in (dict(wedge_mode=1), dict(profile=True)):
        ctx.stats(reset=True)
        res = _alloc(g.n)
        ef.ef_compute_ex(ctx.handle, _dev(g.row_ptr), _dev(g.col_idx), precision=precision, device_check=True,
                         **kw, **res)
        assert_parity(_host(res), ref, precision)
        if kw.get("profile"):
            st = ctx.stats(reset=True)
            assert st["calls"] == 1 and st["prep_ms"] > 0 and st["tri_pairs_ms"] > 0
        rp, ci = bad_graph("range")
        out = _alloc(len(rp) - 1, fill=-7)
        with pytest.raises(ef.EfError) as ei:
            ef.ef_compute_ex(ctx.handle, _dev(rp), _dev(ci), precision=precision, device_check=True, **kw, **out)
        assert ei.value.code == ef.EF_ERR_GRAPH
        assert np.all(_host(out)["ef"] == -7.0)
