"""TEST INFRASTRUCTURE ONLY: brute-force EF_2 for tiny graphs, pure Python.

Independent of Algorithm 1's degree formula.  For a seed s it enumerates the
ordered two-step transmission sequences (Section 3.3: a cluster is one
possible infection state after j = 2 transmission events from s): s infects a
neighbour a, then either s or a infects a node b outside {s, a}.  The cluster
is the node set {s, a, b}; its out-degree is counted edge by edge as the
number of edges with exactly one end in the cluster.  EF(s) is Eq. 1 over
these clusters, natural logarithm; a seed whose degrees sum to 0 is
degenerate (EF = 0, flag = 1).
"""
from __future__ import annotations

import math


def adjacency(n, edges):
    adj = [set() for _ in range(n)]
    for u, v in edges:
        if u != v:
            adj[u].add(v)
            adj[v].add(u)
    return adj


def adjacency_from_csr(row_ptr, col_idx):
    n = len(row_ptr) - 1
    return [set(int(x) for x in col_idx[row_ptr[v]:row_ptr[v + 1]]) for v in range(n)]


def out_degree(adj, cluster) -> int:
    """Number of edges joining a node of `cluster` to a node outside it."""
    return sum(1 for x in cluster for y in adj[x] if y not in cluster)


def histogram(adj, s) -> dict:
    h = {}
    for a in adj[s]:
        for infector in (s, a):
            for b in adj[infector]:
                if b == s or b == a:
                    continue
                d = out_degree(adj, {s, a, b})
                h[d] = h.get(d, 0) + 1
    return h


def expected_force(adj, s):
    """(EF, N, S, T, flag) of seed s."""
    h = histogram(adj, s)
    N = sum(h.values())
    S = sum(c * d for d, c in h.items())
    T = sum(c * d * math.log(d) for d, c in sorted(h.items()) if d > 0)
    if S == 0:
        return 0.0, N, S, T, 1
    ef = 0.0
    for d, c in sorted(h.items()):
        if d > 0:
            p = d / S
            ef -= c * p * math.log(p)
    return ef, N, S, T, 0
