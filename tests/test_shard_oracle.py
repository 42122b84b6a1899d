"""Pins for the sharded form of Algorithm 1 in the oracle (oracle/shard.py).

- summed over any partition of the middle nodes, the partials are the
  literal C implementation of Algorithm 1's N, S and T, and Eq. 1 finalizes
  them to its EF (the decomposition every shard of the library relies on);
- a star's clusters all sit at its centre: closed forms for the centre's
  shard, zeros for the leaves';
- the shard cuts split the adjacency entries evenly.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import shard


def _graphs():
    return [
        synth.erdos_renyi(90, 0.12, 5),
        synth.barabasi_albert(150, 3, 6),
        synth.watts_strogatz(120, 6, 0.1, 7),   # many triangles
        synth.disjoint_union([synth.complete(7), synth.star(12), synth.path(5), synth.petersen()]),
    ]


def _sum_over(g, cuts):
    tot = {k: np.zeros(g.n, dt) for k, dt in (("N", np.int64), ("S", np.int64), ("T", np.float64))}
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        p = shard.partials(g, lo, hi)
        for k in tot:
            tot[k] += p[k]
    return tot


@pytest.mark.parametrize("gi", range(4))
def test_partials_sum_to_algorithm_1_over_any_partition(gi):
    g = _graphs()[gi]
    ref = oracle.alg1(g)
    rng = np.random.default_rng(gi)
    partitions = [[0, g.n], shard.node_cuts(g.row_ptr, 3), shard.node_cuts(g.row_ptr, g.n + 4),
                  [0] + sorted(rng.choice(np.arange(1, g.n), size=5, replace=False).tolist()) + [g.n]]
    for cuts in partitions:
        tot = _sum_over(g, cuts)
        np.testing.assert_array_equal(tot["N"], ref["N"])
        np.testing.assert_array_equal(tot["S"], ref["S"])
        np.testing.assert_allclose(tot["T"], ref["T"], rtol=1e-12, atol=1e-9)
        fin = shard.finalize(tot["S"], tot["T"])
        np.testing.assert_allclose(fin["EF"], ref["EF"], rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(fin["flag"], ref["flag"])


def test_star_clusters_sit_at_the_centre():
    k = 11
    g = synth.star(k)   # centre 0, leaves 1..k; every cluster is (leaf, 0, leaf) of degree k - 2
    centre = shard.partials(g, 0, 1)
    leaves = shard.partials(g, 1, g.n)
    d = k - 2
    assert centre["N"][0] == k * (k - 1) and centre["S"][0] == k * (k - 1) * d
    assert math.isclose(centre["T"][0], k * (k - 1) * d * math.log(d), rel_tol=1e-14)
    assert np.all(centre["N"][1:] == k - 1) and np.all(centre["S"][1:] == (k - 1) * d)
    for key in ("N", "S", "T"):
        assert not np.any(leaves[key])


def test_node_cuts_split_the_adjacency_evenly():
    g = synth.barabasi_albert(400, 4, 8)
    deg = np.diff(g.row_ptr)
    m = int(g.row_ptr[-1])
    for R in (1, 2, 5, 13, 1000):
        cuts = shard.node_cuts(g.row_ptr, R)
        assert cuts[0] == 0 and cuts[-1] == g.n and all(a <= b for a, b in zip(cuts[:-1], cuts[1:]))
        for r in range(R):
            nnz = int(g.row_ptr[cuts[r + 1]] - g.row_ptr[cuts[r]])
            assert abs(nnz - m / R) <= deg.max() + 1
