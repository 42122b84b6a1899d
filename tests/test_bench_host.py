"""Host-side figures of bench.py that feed the bench line (CPU only): the
cluster count W, the f evaluations of the wedge kernels behind the ALU
roofline, and the per-pass algorithmic bytes.  Each is checked against a
plain count on small graphs: W against Algorithm 1's credited clusters from
the oracle (every cluster credits 4), the class-kernel evaluations against a
loop over the middle nodes that forms the classes as the kernels do."""
import numpy as np

import bench
import oracle
import synth


def _graphs():
    hub = synth.from_edges(1400, [(0, j) for j in range(1, 700)] + [(1, j) for j in range(700, 1400)] +
                           [(2, j) for j in range(3, 60)] + [(j, j + 1) for j in range(3, 1399)])
    return [synth.erdos_renyi(300, 0.05, 3), synth.barabasi_albert(3000, 6, 4), synth.powerlaw_cm(4000, 2.1, 2, 900, 5),
            hub, synth.complete(70)]


def test_cluster_count_is_algorithm_1s():
    for g in _graphs():
        st = bench.graph_stats(g)
        assert int(oracle.alg1(g)["N"].sum()) == 4 * st["W"]
        d = g.degrees.astype(np.int64)
        assert st["small_evals"] + st["big_evals"] == int((d * (d - 1)).sum())


def test_class_evaluations_by_a_plain_loop():
    for g in _graphs():
        d = g.degrees.astype(np.int64)
        want = 0
        for u in range(g.n):
            if d[u] <= 32:
                continue
            limit = 256 if d[u] < 513 else 2048   # dense histogram of the warp / CTA kernel
            nb = d[g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]]
            K = len(set(int(x) for x in nb if x < limit)) + int((nb >= limit).sum())
            want += K * (K + 1)
        assert bench.class_evals(g) == want


def test_pair_test_bytes_formula():
    g = synth.barabasi_albert(3000, 6, 4)
    alg = bench.algorithmic_bytes(g, bench.graph_stats(g))
    n, m = g.n, g.nnz
    assert alg["tri_pairs_ms"] == 4 * (n + 1) + 10 * m + 16 * n
    assert alg["finalize_ms"] == 68 * n
    assert all(v > 0 for v in alg.values())
