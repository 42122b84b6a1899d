"""TEST INFRASTRUCTURE ONLY: the sharded form of Algorithm 1, in plain Python.

Only ``tests/`` may import this module.  It shares no code with the CUDA
library.

Algorithm 1 visits every cluster (i, v, j) once, at its middle node v, and
credits its degree d to i once, to j once and to v twice (Section 4).
Restricting that loop to the middle nodes of a range [lo, hi) gives a shard's
partials: for every node x, the credited cluster count N, the credited degree
sum S and the credited sum of d ln d, T, over the clusters whose middle node
is in the range.  Every cluster has exactly one middle node, so the
element-wise sums of the partials over any partition of the nodes into
ranges are Algorithm 1's N, S and T, and Eq. 1 in the form
EF = ln S - T / S finalizes them.

The cluster degree follows Section 3.3: D_i + D_v + D_j - 4 edges leave the
cluster, 2 fewer when i and j are adjacent (the edge i-j is then inside).

Pure-Python loops: small graphs only.
"""
from __future__ import annotations

import math

import numpy as np


def partials(g, lo: int, hi: int) -> dict:
    """N, S (int64) and T (float64) of every node from the clusters whose middle node is in [lo, hi)."""
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    ci = np.asarray(g.col_idx, dtype=np.int64)
    n = rp.shape[0] - 1
    deg = np.diff(rp)
    rows = [set(ci[rp[v]:rp[v + 1]].tolist()) for v in range(n)]
    N = np.zeros(n, np.int64)
    S = np.zeros(n, np.int64)
    T = np.zeros(n, np.float64)
    for v in range(max(lo, 0), min(hi, n)):
        nb = ci[rp[v]:rp[v + 1]].tolist()
        for a in range(len(nb)):
            for b in range(a + 1, len(nb)):
                i, j = nb[a], nb[b]
                d = int(deg[i] + deg[v] + deg[j] - 4 - (2 if j in rows[i] else 0))
                f = d * math.log(d) if d > 1 else 0.0
                for x, w in ((i, 1), (j, 1), (v, 2)):
                    N[x] += w
                    S[x] += w * d
                    T[x] += w * f
    return dict(N=N, S=S, T=T)


def finalize(S, T) -> dict:
    """Eq. 1 from summed partials: EF = ln S - T/S; EF = 0 with flag 1 where S = 0."""
    S = np.asarray(S, dtype=np.int64)
    T = np.asarray(T, dtype=np.float64)
    ef = np.zeros(S.shape[0], np.float64)
    flag = (S == 0).astype(np.uint8)
    pos = S > 0
    ef[pos] = np.log(S[pos].astype(np.float64)) - T[pos] / S[pos]
    return dict(EF=ef, flag=flag)


def node_cuts(row_ptr, num_shards: int) -> list:
    """Shard boundaries: shard r takes the nodes [cut[r], cut[r+1]), cut at the
    first row that starts at or after adjacency entry r m / R."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    n, m = rp.shape[0] - 1, int(rp[-1])
    cuts = [0]
    for r in range(1, num_shards):
        cuts.append(int(np.searchsorted(rp, m * r // num_shards, side="left")))
    cuts.append(n)
    return cuts
