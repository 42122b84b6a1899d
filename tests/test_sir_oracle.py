"""Pins for the SIR oracle (oracle/sir.py), none of them the oracle against itself.

- Philox4x32-10 against the published known-answer vectors of its authors;
- beta = gamma = 1 makes the epidemic a breadth-first search: final size,
  length, peak and the infection tree against SciPy's shortest paths and
  connected components;
- gamma = 1 on the complete graph is the Reed-Frost chain binomial: the
  final-size distribution of many simulations against its exact law;
- beta = 0: the epidemic length is geometric (mean 1 / gamma);
- spreading power on a path in closed form; an immune node cuts a path;
- a simulation's result depends on its id and the seed only, not on the
  batch around it.
"""
import math

import numpy as np
import pytest

import synth
from oracle import sir


@pytest.mark.parametrize("ctr,key,out", [
    ((0, 0, 0, 0), 0, (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, 0xFFFFFFFFFFFFFFFF, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), 0x299F31D0A4093822,
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
])
def test_philox_known_answers(ctr, key, out):
    got = sir.philox4x32_10(*[np.array([c]) for c in ctr], key)
    assert tuple(int(w[0]) for w in got) == out


def test_thresholds():
    assert sir.threshold(0.0) == 0 and sir.threshold(1.0) == 2 ** 32 and sir.threshold(0.5) == 2 ** 31
    with pytest.raises(ValueError):
        sir.threshold(1.5)


def _levels(g, src):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path
    A = csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    d = shortest_path(A, unweighted=True, indices=src)
    return np.where(np.isinf(d), -1, d).astype(np.int64)


@pytest.mark.parametrize("gi", range(3))
def test_certain_infection_and_recovery_is_breadth_first_search(gi):
    g = [synth.erdos_renyi(300, 0.008, 1), synth.barabasi_albert(400, 2, 2),
         synth.disjoint_union([synth.path(30), synth.cycle(9)])][gi]
    rng = np.random.default_rng(gi)
    idx = rng.choice(g.n, 6, replace=False)
    r = sir.simulate(g, idx, 1.0, 1.0, seed=7)
    for b, s in enumerate(idx):
        lv = _levels(g, s)
        reach = lv >= 0
        assert r["final_size"][b] == reach.sum()
        assert r["length"][b] == lv.max() + 1
        sizes = np.bincount(lv[reach])
        assert r["peak_infected"][b] == sizes.max() and r["peak_step"][b] == int(np.argmax(sizes))
        par = r["parent"][b]
        assert par[s] == s and np.all(par[~reach] == -1)
        for x in np.nonzero(reach)[0]:
            if x == s:
                continue
            nb = g.col_idx[g.row_ptr[x]:g.row_ptr[x + 1]]
            assert par[x] == nb[lv[nb] == lv[x] - 1].min()


def test_one_step_infectiousness_on_a_complete_graph_is_reed_frost():
    scipy_stats = pytest.importorskip("scipy.stats")
    n, beta, sims = 12, 0.12, 4000
    g = synth.complete(n)
    r = sir.simulate(g, np.zeros(sims, np.int64), beta, 1.0, seed=11)
    exact = sir.reed_frost_final_size(n, beta)
    assert math.isclose(exact.sum(), 1.0, rel_tol=1e-12)
    obs = np.bincount(r["final_size"], minlength=n + 1)
    # pool the sizes with few expected counts into one cell
    keep = exact * sims >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exact[keep], exact[~keep].sum()) * sims
    if e[-1] == 0:
        o, e = o[:-1], e[:-1]
    p = scipy_stats.chisquare(o, e).pvalue
    assert p > 1e-3, (p, obs, exact * sims)


def test_no_infection_gives_geometric_lengths():
    g = synth.star(6)
    sims = 4000
    r = sir.simulate(g, np.zeros(sims, np.int64), 0.0, 0.5, seed=3)
    assert np.all(r["final_size"] == 1) and np.all(r["peak_infected"] == 1)
    L = r["length"]
    assert L.min() >= 1 and abs(L.mean() - 2.0) < 5 * math.sqrt(2.0) / math.sqrt(sims)
    assert abs((L == 1).mean() - 0.5) < 5 * 0.5 / math.sqrt(sims)


def test_spreading_power_on_a_path():
    n, depth = 12, 4
    g = synth.path(n)
    r = sir.simulate(g, [0], 1.0, 1.0, seed=1, depth=depth)
    for k in range(1, depth + 1):
        assert list(r["spread"][0, k - 1]) == [min(k, n - 1 - v) for v in range(n)]


def test_an_immune_node_cuts_a_path():
    g = synth.path(10)
    imm = np.zeros((1, 10), np.uint8)
    imm[0, 5] = 1
    r = sir.simulate(g, [0, 9], 1.0, 1.0, seed=1, immune=imm, immune_set=[0, -1])
    assert list(r["final_size"]) == [5, 10]
    assert np.all(r["parent"][0, 5:] == -1)
    with pytest.raises(ValueError):
        sir.simulate(g, [5], 1.0, 1.0, seed=1, immune=imm, immune_set=[0])


def test_result_depends_on_simulation_id_not_on_batch():
    g = synth.barabasi_albert(500, 3, 4)
    idx = np.array([3, 17, 17, 250, 99])
    full = sir.simulate(g, idx, 0.3, 0.4, seed=5, sim_base=100)
    one = sir.simulate(g, idx[3:4], 0.3, 0.4, seed=5, sim_base=103)
    for k in ("final_size", "length", "peak_infected", "peak_step"):
        assert full[k][3] == one[k][0]
    assert np.array_equal(full["parent"][3], one["parent"][0])
    # the two simulations from node 17 draw different numbers
    assert not np.array_equal(full["parent"][1], full["parent"][2]) or full["final_size"][1] == 1
