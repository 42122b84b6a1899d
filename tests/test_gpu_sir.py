"""The SIR simulation on the GPU, through the C ABI, against the CPU oracle.

Both sides draw the same Philox4x32-10 numbers from the same counters, so
every simulation must agree exactly: final size, length, peak and its step,
truncation, the whole infection tree (parent of every node), and the
spreading-power sums of orders 1-4 (over all simulations, and over the
global outbreaks only).  Cases: the ER 2000 graph and heavy-tailed graphs
(BA, power-law, R-MAT) at the paper's calibration (gamma = 1/3,
beta = 1.3 / (3 <k>)) and at a higher beta that gives large outbreaks;
immune sets per simulation; batches split across calls (sim_base); a step
cap; a 200 000-node graph; invalid arguments.
"""
import numpy as np
import pytest

import synth
from oracle import sir as osir

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


ALL = ("final_size", "length", "peak_infected", "peak_step", "truncated", "parent", "spread", "spread_sims")


def _gpu(ctx, g, idx, min_size=0, **kw):
    out = ctx.sir(_dev(g.row_ptr), _dev(g.col_idx), _dev(np.asarray(idx, np.int32)), outputs=ALL,
                  spread_min_size=min_size, **kw)
    return {k: v.cpu().numpy() for k, v in out.items()}


def _compare(got, ref, min_size=0):
    for k in ("final_size", "length", "peak_infected", "peak_step"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    np.testing.assert_array_equal(got["truncated"].astype(bool), ref["truncated"])
    np.testing.assert_array_equal(got["parent"], ref["parent"])
    sel = ref["final_size"] >= min_size
    np.testing.assert_array_equal(got["spread"], ref["spread"][sel].sum(axis=0))
    np.testing.assert_array_equal(got["spread_sims"], (ref["parent"][sel] >= 0).sum(axis=0))


def _graphs():
    return {
        "er2000": synth.workload(1),
        "ba3000": synth.barabasi_albert(3000, 4, 71),
        "plcm5000": synth.powerlaw_cm(5000, 2.3, 3, 400, 72),
        "rmat12": synth.rmat(12, 8, 73),
    }


@pytest.mark.parametrize("name", ["er2000", "ba3000", "plcm5000", "rmat12"])
@pytest.mark.parametrize("r0", [1.3, 4.0])
def test_simulations_match_oracle(ctx, name, r0):
    g = _graphs()[name]
    k = g.nnz / g.n
    beta, gamma = r0 / (3 * k), 1 / 3
    rng = np.random.default_rng(5)
    idx = rng.integers(0, g.n, 48)
    idx[:3] = idx[0]   # repeated index cases draw different numbers
    min_size = int(0.25 * g.n)
    ref = osir.simulate(g, idx, beta, gamma, seed=1234, sim_base=17)
    got = _gpu(ctx, g, idx, min_size=min_size, beta=beta, gamma=gamma, seed=1234, sim_base=17)
    _compare(got, ref, min_size)
    got_all = _gpu(ctx, g, idx, beta=beta, gamma=gamma, seed=1234, sim_base=17)
    _compare(got_all, ref, 0)
    if r0 > 2:
        assert (ref["final_size"] >= min_size).any()   # the high-beta case has global outbreaks


def test_immune_sets(ctx):
    g = synth.barabasi_albert(4000, 3, 74)
    rng = np.random.default_rng(6)
    deg = np.diff(g.row_ptr)
    imm = np.zeros((2, g.n), np.uint8)
    imm[0, rng.choice(g.n, g.n // 20, replace=False)] = 1   # 5% at random
    imm[1, np.argsort(-deg)[:g.n // 20]] = 1                 # the 5% of highest degree
    idx = rng.choice(np.nonzero(imm.sum(axis=0) == 0)[0], 30)
    sets = np.array([-1, 0, 1] * 10, np.int32)
    beta, gamma = 3.0 / (3 * g.nnz / g.n), 1 / 3
    ref = osir.simulate(g, idx, beta, gamma, seed=9, immune=imm, immune_set=sets)
    got = _gpu(ctx, g, idx, beta=beta, gamma=gamma, seed=9, immune=_dev(imm), immune_set=_dev(sets))
    _compare(got, ref)
    for s in range(30):
        if sets[s] >= 0:
            assert np.all(got["parent"][s][imm[sets[s]] == 1] == -1)


def test_batches_split_by_sim_base(ctx):
    g = synth.barabasi_albert(3000, 4, 75)
    idx = np.random.default_rng(7).integers(0, g.n, 40)
    kw = dict(beta=0.08, gamma=0.3, seed=77)
    whole = _gpu(ctx, g, idx, sim_base=1000, **kw)
    a = _gpu(ctx, g, idx[:13], sim_base=1000, **kw)
    b = _gpu(ctx, g, idx[13:], sim_base=1013, **kw)
    for k in ("final_size", "length", "peak_infected", "peak_step", "parent"):
        np.testing.assert_array_equal(whole[k], np.concatenate([a[k], b[k]]))
    np.testing.assert_array_equal(whole["spread"], a["spread"] + b["spread"])


def test_step_cap(ctx):
    g = synth.barabasi_albert(2000, 4, 76)
    idx = np.arange(20)
    ref = osir.simulate(g, idx, 0.2, 0.1, seed=3, max_steps=3)
    got = _gpu(ctx, g, idx, beta=0.2, gamma=0.1, seed=3, max_steps=3)
    assert ref["truncated"].any()
    _compare(got, ref)


def test_large_graph(ctx):
    g = synth.barabasi_albert(200000, 4, 77)
    idx = np.random.default_rng(8).integers(0, g.n, 16)
    beta, gamma = 3.0 / (3 * g.nnz / g.n), 1 / 3
    ref = osir.simulate(g, idx, beta, gamma, seed=5)
    got = _gpu(ctx, g, idx, min_size=int(0.25 * g.n), beta=beta, gamma=gamma, seed=5)
    _compare(got, ref, int(0.25 * g.n))


def test_errors(ctx):
    import paper_2306_00606_gb300 as ef
    g = synth.erdos_renyi(200, 0.05, 78)
    rp, ci = _dev(g.row_ptr), _dev(g.col_idx)
    imm = np.zeros((1, g.n), np.uint8)
    imm[0, 7] = 1
    cases = [
        dict(index_cases=_dev(np.array([0, g.n], np.int32))),
        dict(index_cases=_dev(np.array([-1], np.int32))),
        dict(index_cases=_dev(np.array([7], np.int32)), immune=_dev(imm), immune_set=_dev(np.array([0], np.int32))),
        dict(index_cases=_dev(np.array([3], np.int32)), immune=_dev(imm), immune_set=_dev(np.array([1], np.int32))),
        dict(index_cases=_dev(np.array([3], np.int32)), beta=1.5),
        dict(index_cases=_dev(np.array([3], np.int32)), depth=5),
        dict(index_cases=_dev(np.array([3], np.int32)), max_steps=0),
    ]
    for c in cases:
        kw = dict(beta=0.1, gamma=0.3, seed=1)
        kw.update(c)
        with pytest.raises(ef.EfError) as ei:
            ef.ef_sir_run(ctx.handle, rp, ci, kw.pop("index_cases"), **kw)
        assert ei.value.code == ef.EF_ERR_ARG, c
