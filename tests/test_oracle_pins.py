"""Pins for the CPU oracle, checked against what the paper and the mathematics fix.

None of these compares the oracle with itself: closed forms for graph families
(tests/golden/closed_forms.txt), closed-form cluster counts and degree sums,
an edge-by-edge brute force over ordered transmission sequences (exhaustive on
all labelled graphs with up to 5 nodes, random graphs up to 10 nodes),
agreement of Algorithm 1 with the vertex-centric formulation and invariances
(relabelling, disjoint union, locality).
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")


def _family(name, p):
    if name == "complete":
        return synth.complete(p), dict(n=p)
    if name == "star":
        return synth.star(p), dict(k=p)
    if name == "cycle":
        return synth.cycle(p), dict(n=p, r=2)
    if name == "bipartite":
        return synth.complete_bipartite(p, p), dict(r=p)
    if name == "hypercube":
        return synth.hypercube(p), dict(r=p)
    if name == "petersen":
        return synth.petersen(), dict(r=3)
    if name == "path5":
        return synth.path(5), dict()
    raise ValueError(name)


def _nodes(name, role, g):
    if role == "any":
        return list(range(g.n))
    if name == "star":
        return [0] if role == "centre" else list(range(1, g.n))
    if name == "path5":
        return {"end": [0, 4], "second": [1, 3], "middle": [2]}[role]
    raise ValueError(role)


def _golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            fam, p, role, ef, N, S = line.split()
            rows.append((fam, int(p), role, ef, N, S))
    return rows


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: f"{r[0]}{r[1]}-{r[2]}")
def test_closed_forms(row):
    fam, p, role, ef_expr, n_expr, s_expr = row
    g, env = _family(fam, p)
    env = dict(env, log=math.log)
    o = oracle.alg1(g)
    v = oracle.vertex(g)
    for node in _nodes(fam, role, g):
        assert o["N"][node] == int(eval(n_expr, {}, env))
        assert o["S"][node] == int(eval(s_expr, {}, env))
        assert o["EF"][node] == pytest.approx(eval(ef_expr, {}, env), rel=1e-13, abs=1e-13)
        assert v["EF"][node] == pytest.approx(eval(ef_expr, {}, env), rel=1e-13, abs=1e-13)
        assert o["flag"][node] == 0


def test_complete_graph_single_cluster_degree():
    # Every cluster of K_n is a triangle: one histogram bin at d = 3(n-3).
    for n in (4, 5, 7):
        g = synth.complete(n)
        for s in range(n):
            assert oracle.alg1_hist(g, s) == {3 * (n - 3): 2 * (n - 1) * (n - 2)}


def test_degenerate_cases():
    # K3: all 4 credited clusters have degree 0 -> S = 0 -> degenerate.
    o = oracle.alg1(synth.complete(3))
    assert list(o["N"]) == [4, 4, 4] and list(o["S"]) == [0, 0, 0]
    assert list(o["flag"]) == [1, 1, 1] and list(o["EF"]) == [0, 0, 0]
    # P3 (= star K_{1,2}): the one cluster has degree 0.
    o = oracle.alg1(synth.path(3))
    assert list(o["N"]) == [1, 2, 1] and list(o["S"]) == [0, 0, 0] and list(o["flag"]) == [1, 1, 1]
    # K2 and isolated nodes: no clusters at all.
    g = synth.from_edges(4, [(0, 1)])
    o = oracle.alg1(g)
    assert list(o["N"]) == [0, 0, 0, 0] and list(o["flag"]) == [1, 1, 1, 1]
    # empty graph
    g = synth.from_edges(0, [])
    o = oracle.alg1(g)
    assert o["EF"].shape == (0,)


def _closed_counts(g):
    d = g.degrees
    src = np.repeat(np.arange(g.n), d)
    sig1 = np.bincount(src, weights=d[g.col_idx], minlength=g.n).astype(np.int64)
    t = oracle.triangles(g)
    N = d * (d - 2) + sig1
    nb = (d[g.col_idx] - 1) * (d[g.col_idx] + d[src] - 4) + sig1[g.col_idx] - d[src]
    S = d * (d - 1) * (d - 4) + 2 * (d - 1) * sig1 + np.bincount(src, weights=nb, minlength=g.n).astype(np.int64) - 8 * t
    return N, S, t


@pytest.mark.parametrize("make", [
    lambda: synth.erdos_renyi(300, 0.03, 1),
    lambda: synth.barabasi_albert(400, 3, 2),
    lambda: synth.powerlaw_cm(500, 2.3, 2, 60, 3),
    lambda: synth.watts_strogatz(300, 6, 0.2, 4),
    lambda: synth.complete(12),
])
def test_closed_form_counts_and_degree_sums(make):
    """N_v = D(D-2) + sigma1(v);  S_v from degrees, sigma1 and triangle counts."""
    g = make()
    N, S, t = _closed_counts(g)
    o = oracle.alg1(g)
    assert np.array_equal(o["N"], N)
    assert np.array_equal(o["S"], S)
    assert int(o["N"].sum()) == 4 * g.wedges()
    v = oracle.vertex(g)
    assert np.array_equal(v["t"], t)


def _all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield [pairs[i] for i in range(len(pairs)) if mask >> i & 1]


def _check_against_brute(n, edges):
    g = synth.from_edges(n, edges)
    adj = brute.adjacency(n, edges)
    o = oracle.alg1(g)
    for s in range(n):
        ef, N, S, T, fl = brute.expected_force(adj, s)
        assert o["N"][s] == N and o["S"][s] == S and o["flag"][s] == fl
        assert o["T"][s] == pytest.approx(T, rel=1e-12, abs=1e-12)
        assert o["EF"][s] == pytest.approx(ef, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_brute_force_exhaustive(n):
    for edges in _all_graphs(n):
        _check_against_brute(n, edges)


def test_brute_force_random_up_to_10():
    rng = np.random.default_rng(7)
    for it in range(400):
        n = int(rng.integers(3, 11))
        p = float(rng.uniform(0.15, 0.9))
        edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
        _check_against_brute(n, edges)


def test_histograms_three_ways():
    """H_s from Algorithm 1, from the vertex-centric walk and from brute force agree."""
    rng = np.random.default_rng(11)
    for it in range(60):
        n = int(rng.integers(4, 11))
        edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.45]
        g = synth.from_edges(n, edges)
        adj = brute.adjacency(n, edges)
        for s in range(n):
            hb = brute.histogram(adj, s)
            assert oracle.alg1_hist(g, s) == hb
            assert oracle.vertex_hist(g, s) == hb


@pytest.mark.parametrize("make", [
    lambda: synth.workload(1),
    lambda: synth.barabasi_albert(3000, 5, 5),
    lambda: synth.powerlaw_cm(4000, 2.3, 3, 400, 6),
    lambda: synth.rmat(10, 8, 7),
])
def test_vertex_centric_equals_alg1(make):
    g = make()
    a = oracle.alg1(g)
    v = oracle.vertex(g, threads=2)
    assert np.array_equal(a["N"], v["N"]) and np.array_equal(a["S"], v["S"])
    assert np.array_equal(a["flag"], v["flag"])
    np.testing.assert_allclose(v["T"], a["T"], rtol=1e-13)
    np.testing.assert_allclose(v["EF"], a["EF"], rtol=1e-12, atol=1e-13)


def test_relabelling_invariance():
    g = synth.barabasi_albert(500, 4, 9)
    perm = np.random.default_rng(3).permutation(g.n)
    h = synth.relabel(g, perm)
    a, b = oracle.alg1(g), oracle.alg1(h)
    assert np.array_equal(a["N"], b["N"][perm]) and np.array_equal(a["S"], b["S"][perm])
    np.testing.assert_allclose(a["EF"], b["EF"][perm], rtol=1e-12, atol=1e-13)


def test_disjoint_union_invariance():
    parts = [synth.erdos_renyi(200, 0.05, 1), synth.star(9), synth.complete(3), synth.cycle(7),
             synth.barabasi_albert(150, 3, 2)]
    u = synth.disjoint_union(parts)
    ou = oracle.alg1(u)
    for i, g in enumerate(parts):
        lo, hi = u.graph_off[i], u.graph_off[i + 1]
        og = oracle.alg1(g)
        assert np.array_equal(og["N"], ou["N"][lo:hi]) and np.array_equal(og["S"], ou["S"][lo:hi])
        np.testing.assert_allclose(og["EF"], ou["EF"][lo:hi], rtol=1e-12, atol=1e-13)


def _bfs_dist(g, s):
    dist = np.full(g.n, -1)
    dist[s] = 0
    frontier = [s]
    while frontier:
        nxt = []
        for v in frontier:
            for u in g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]:
                if dist[u] < 0:
                    dist[u] = dist[v] + 1
                    nxt.append(int(u))
        frontier = nxt
    return dist


def test_locality():
    """An edge whose ends are both at distance >= 3 from v leaves EF(v) unchanged,
    while one touching distance 2 changes it (d depends on degrees at distance 2)."""
    g = synth.watts_strogatz(200, 4, 0.05, 12)
    v = 0
    dist = _bfs_dist(g, v)
    base = oracle.alg1(g)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    edges = [(int(a), int(b)) for a, b in zip(src, g.col_idx) if a < b]
    far = [int(x) for x in np.where((dist >= 3) | (dist < 0))[0]]
    adj = set(edges)
    a, b = next((x, y) for x in far for y in far if x < y and (x, y) not in adj)
    o = oracle.alg1(synth.from_edges(g.n, edges + [(a, b)]))
    assert o["EF"][v] == base["EF"][v] and o["N"][v] == base["N"][v]
    two = [int(x) for x in np.where(dist == 2)[0]]
    c = next(y for y in far if (min(two[0], y), max(two[0], y)) not in adj)
    o2 = oracle.alg1(synth.from_edges(g.n, edges + [(two[0], c)]))
    assert o2["S"][v] != base["S"][v]


def test_invalid_csr_rejected():
    rp = np.array([0, 1, 2], np.int32)
    with pytest.raises(RuntimeError):
        oracle.alg1(rp, np.array([0, 0], np.int32))       # self-loop
    with pytest.raises(RuntimeError):
        oracle.alg1(rp, np.array([1, 5], np.int32))       # out of range
    with pytest.raises(RuntimeError):
        oracle.alg1(np.array([0, 2, 2], np.int32), np.array([1, 1], np.int32))  # duplicate
