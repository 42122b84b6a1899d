"""The learned ranking path on the GPU, through the C ABI, against the CPU oracle.

- features: every one of the 16 against oracle/surrogate.py (FP32 logs,
  so 1e-5 relative);
- exact EF of chosen nodes: N, S and t exactly, EF within the parity bars,
  against the vertex-centric oracle;
- the network: forward pass and gradients (BF16 operands, FP32
  accumulation), element by element:
  * on a network and inputs of few-bit dyadic values, where every operand is
    a BF16 number and every sum is exact in FP32, the GPU must equal the
    FP64 oracle exactly (any transposed, misplaced or dropped term shows);
  * on realistic features, against the oracle with the same BF16 operand
    rounding: each gradient element within 2^-6 of the absolute sum of its
    own terms (one BF16 step on every operand, and the FP32 sums), rows
    whose ReLU masks FP32 sums could decide differently allowed their full
    terms; each prediction within 2^-7 of the absolute sum it is made of;
    and against the unrounded FP64 oracle block by block;
- training lowers the loss, and save/load round-trips;
- ranking: the trained network's top set reaches 0.95 recall of the exact
  top 1% while computing exact EF for a few percent of the nodes, and it
  beats the same network untrained and the ranking by degree.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import surrogate as sg
from netcases import dyadic_network

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


def _features(ctx, g, mode):
    import torch
    import paper_2306_00606_gb300 as ef
    x = torch.empty((g.n, 16), dtype=torch.float32, device="cuda")
    ef.ef_features(ctx.handle, _dev(g.row_ptr), _dev(g.col_idx), x, mode=mode)
    torch.cuda.synchronize()
    return x


def _exact_all(ctx, g, precision="fp32c"):
    import torch
    out = ctx.compute(_dev(g.row_ptr), _dev(g.col_idx), precision=precision, outputs=("ef",))
    torch.cuda.synchronize()
    return out["ef"].cpu().numpy()


@pytest.mark.parametrize("mode", [0, 1])
def test_features_match_oracle(ctx, mode):
    # hubs (degree > 32) next to isolated nodes: the row passes then walk the
    # work lists and clear the isolated rows separately
    g = synth.disjoint_union([synth.barabasi_albert(3000, 4, 41), synth.powerlaw_cm(4000, 2.2, 2, 900, 42),
                              synth.complete(12), synth.star(50), synth.path(2), synth.from_edges(4, [])])
    assert (g.degrees == 0).sum() >= 4 and g.degrees.max() > 32
    got = _features(ctx, g, mode).cpu().numpy()
    ref = sg.features(g, triangles=oracle.triangles(g) if mode == 1 else None)
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=2e-5)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_nodes_exact_matches_oracle(ctx, precision):
    import torch
    import paper_2306_00606_gb300 as ef
    g = synth.powerlaw_cm(30000, 2.1, 2, 6000, 43)
    deg = np.diff(g.row_ptr)
    rng = np.random.default_rng(1)
    nodes = np.concatenate([np.argsort(-deg)[:40], rng.choice(g.n, 300, replace=False), [0, 0]]).astype(np.int32)
    out = {k: torch.empty(len(nodes), dtype=dt, device="cuda") for k, dt in
           (("ef", torch.float64), ("n_clusters", torch.int64), ("s", torch.int64), ("triangles", torch.int64))}
    ef.ef_compute_nodes(ctx.handle, _dev(g.row_ptr), _dev(g.col_idx), _dev(nodes), precision=precision, **out)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    ref = oracle.vertex(g, nodes)
    np.testing.assert_array_equal(got["n_clusters"], ref["N"])
    np.testing.assert_array_equal(got["s"], ref["S"])
    np.testing.assert_array_equal(got["triangles"], ref["t"])
    if precision == "fp64":
        np.testing.assert_allclose(got["ef"], ref["EF"], rtol=1e-9, atol=1e-12)
    else:
        np.testing.assert_allclose(got["ef"], ref["EF"], rtol=0, atol=2e-5)
    with pytest.raises(ef.EfError) as ei:
        ef.ef_compute_nodes(ctx.handle, _dev(g.row_ptr), _dev(g.col_idx), _dev(np.array([5, g.n], np.int32)),
                            ef=torch.empty(2, dtype=torch.float64, device="cuda"))
    assert ei.value.code == ef.EF_ERR_ARG


def _random_model(ctx, seed, X):
    import paper_2306_00606_gb300 as ef
    rng = np.random.default_rng(seed)
    p = sg.init_params(seed, mean=X.mean(axis=0), std=X.std(axis=0) + 0.5)
    p["b1"] = rng.normal(size=64) * 0.2
    p["b2"] = rng.normal(size=64) * 0.2
    p["b3"] = 0.4
    m = ef.Model(ctx.handle)
    m.set(np.concatenate([sg.flatten(p), p["mean"], p["std"]]).astype(np.float32))
    # the oracle takes the parameters the device holds (rounded to float32)
    flat = m.get().astype(np.float64)
    return m, sg.unflatten(flat[:sg.N_PARAMS], flat[sg.N_PARAMS:sg.N_PARAMS + 16], flat[sg.N_PARAMS + 16:])


def test_network_forward_matches_oracle(ctx):
    import torch
    g = synth.barabasi_albert(5000, 5, 44)
    x = _features(ctx, g, 0)
    X = x.cpu().numpy().astype(np.float64)
    m, p = _random_model(ctx, 3, X)
    out = torch.empty(g.n, dtype=torch.float32, device="cuda")
    m.forward(x, out)
    got = out.cpu().numpy()
    ref, _ = sg.forward(p, X)
    scale = np.abs(ref).mean() + np.abs(ref).std()
    assert np.abs(got - ref).max() <= 2e-2 * scale, (np.abs(got - ref).max(), scale)
    # element by element against the oracle with the same BF16 operands: a
    # rounding that FP32 sums decide the other way moves one operand by one
    # BF16 step (at most 2^-7 of it), so a prediction stays within 2^-7 of
    # the absolute sum it is made of
    ref16, a = sg.forward(p, X, operands="bf16")
    err = np.abs(got - ref16)
    tol = 2.0 ** -7 * _abs_forward(p, a)
    assert np.all(err <= tol), (int(np.argmax(err / tol)), float(np.max(err / tol)))


def test_network_exact_on_dyadic_values(ctx):
    import torch
    import paper_2306_00606_gb300 as ef
    rows = 64   # four 16-row tiles; 1/batch is a power of two
    p, X, y = dyadic_network(7, rows)
    m = ef.Model(ctx.handle)
    m.set(np.concatenate([sg.flatten(p), p["mean"], p["std"]]).astype(np.float32))
    assert np.array_equal(m.get().astype(np.float64), np.concatenate([sg.flatten(p), p["mean"], p["std"]]))
    x = _dev(X.astype(np.float32))
    out = torch.empty(rows, dtype=torch.float32, device="cuda")
    m.forward(x, out)
    ref, _ = sg.forward(p, X)
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.float64), ref)
    loss, grad = m.grad(x, _dev(y.astype(np.float32)))
    ref_loss, ref_g = sg.loss_and_grads(p, X, y)
    assert loss == ref_loss
    gf = sg.flatten(ref_g)
    o = 0
    for k in sg.TRAINED:
        size = int(np.prod(sg.SHAPES[k]))
        a, b = grad[o:o + size].astype(np.float64), gf[o:o + size]
        assert np.count_nonzero(b) > size // 4, k   # the check covers mostly non-zero elements
        np.testing.assert_array_equal(a, b, err_msg=k)
        o += size


def _abs_forward(p, a):
    """Per row, the absolute sum the prediction is made of, propagated through both layers."""
    z = sg.bf16(a["Z"])
    h1 = np.abs(z) @ np.abs(sg.bf16(p["W1"])) + np.abs(p["b1"])
    h2 = h1 @ np.abs(sg.bf16(p["W2"])) + np.abs(p["b2"])
    return h2 @ np.abs(p["w3"]) + abs(p["b3"])


def _near_midpoint(v, window):
    """Values within `window` of a BF16 rounding midpoint (the FP32 value the
    GPU rounds may lie on the other side of it)."""
    v = np.asarray(v, dtype=np.float64)
    r = sg.bf16(v)
    _, e = np.frexp(r)
    step = np.ldexp(1.0, e - 8)   # BF16 spacing above |r| (8 significant bits)
    d = np.minimum(np.abs(np.abs(v) - (np.abs(r) + step / 2)), np.abs(np.abs(v) - (np.abs(r) - step / 4)))
    d = np.minimum(d, np.abs(np.abs(v) - (np.abs(r) - step / 2)))
    return (d <= window) & (v != 0)


def _mask_unsure_rows(p, a):
    """Rows with a ReLU pre-activation closer to 0 than the GPU's FP32 sums
    and its BF16 roundings could move it: 2^-18 of the pre-activation's
    absolute sum, plus one BF16 step (2^-7) of every operand whose rounding
    could go either way."""
    z, w1, w2 = a["Z"], sg.bf16(p["W1"]), sg.bf16(p["W2"])
    zb = sg.bf16(z)
    s1 = np.abs(zb) @ np.abs(w1) + np.abs(p["b1"])
    zc = _near_midpoint(z, 2.0 ** -20 * np.abs(z))
    d1 = 2.0 ** -7 * (np.abs(zb) * zc) @ np.abs(w1) + 2.0 ** -18 * s1
    h1 = a["H1"]
    h1b = sg.bf16(h1)
    s2 = np.abs(h1b) @ np.abs(w2) + np.abs(p["b2"])
    hc = _near_midpoint(h1, d1)
    d2 = 2.0 ** -7 * (np.abs(h1b) * hc) @ np.abs(w2) + d1 @ np.abs(w2) + 2.0 ** -18 * s2
    return np.any(np.abs(a["A1"]) <= d1, axis=1) | np.any(np.abs(a["A2"]) <= d2, axis=1)


def test_network_gradients_match_oracle(ctx):
    g = synth.barabasi_albert(3000, 5, 45)
    x = _features(ctx, g, 0)
    X = x.cpu().numpy().astype(np.float64)
    y = oracle.alg1(g)["EF"]
    m, p = _random_model(ctx, 4, X)
    loss, grad = m.grad(x, _dev(y.astype(np.float32)))
    ref_loss, ref_g = sg.loss_and_grads(p, X, y)
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss
    gf = sg.flatten(ref_g)
    o = 0
    for k in sg.TRAINED:
        size = int(np.prod(sg.SHAPES[k]))
        a, b = grad[o:o + size].astype(np.float64), gf[o:o + size]
        err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
        assert err <= 3e-2, (k, err)
        o += size
    # element by element against the oracle with the same BF16 operands: each
    # element within 2^-6 of the absolute sum of its own terms (every term's
    # operands one BF16 step away, and the FP32 sums); rows whose ReLU masks
    # the GPU could decide differently may change their terms completely
    _, g16 = sg.loss_and_grads(p, X, y, operands="bf16")
    out, a = sg.forward(p, X, operands="bf16")
    unsure = _mask_unsure_rows(p, a)
    assert unsure.sum() <= 0.05 * len(y), unsure.sum()
    sums, _ = sg.grad_term_sums(p, X, y, operands="bf16")
    au = {k: v[unsure] for k, v in a.items()}
    d_abs = np.abs(2.0 * (out - y) / len(y))[unsure]
    open_sums = _open_term_sums(p, au, d_abs * 1.01)
    o = 0
    for k in sg.TRAINED:
        size = int(np.prod(sg.SHAPES[k]))
        a_k = grad[o:o + size].astype(np.float64)
        b_k = np.ravel(g16[k])
        tol = 2.0 ** -6 * np.ravel(sums[k]) + 2.0 * np.ravel(open_sums[k]) + 1e-12
        ratio = np.abs(a_k - b_k) / tol
        assert np.all(ratio <= 1.0), (k, int(np.sum(ratio > 1)), float(ratio.max()))
        o += size


def _open_term_sums(p, a, d_abs):
    """Absolute term sums of the rows in `a`, with every ReLU mask open and
    |dL/dprediction| = d_abs: a bound on what those rows add to each
    gradient element, whichever way their masks go."""
    z = np.abs(sg.bf16(a["Z"]))
    h1 = np.abs(sg.bf16(a["H1"]))
    h2 = np.abs(a["H2"])
    e2 = np.outer(d_abs, np.abs(p["w3"]))
    e1 = np.abs(sg.bf16(e2)) @ np.abs(sg.bf16(p["W2"])).T
    return {"W1": z.T @ np.abs(sg.bf16(e1)), "b1": e1.sum(axis=0), "W2": h1.T @ np.abs(sg.bf16(e2)),
            "b2": e2.sum(axis=0), "w3": h2.T @ d_abs, "b3": float(d_abs.sum())}


def _training_set(ctx):
    """Exact EF on graphs shaped like the small workloads (ER 2000, BA), as labels."""
    import torch
    gs = [synth.workload(1), synth.barabasi_albert(60000, 5, 46), synth.barabasi_albert(30000, 4, 47)]
    xs, ys = [], []
    for g in gs:
        xs.append(_features(ctx, g, 0))
        ys.append(_dev(_exact_all(ctx, g).astype(np.float32)))
    return torch.cat(xs), torch.cat(ys)


@pytest.fixture(scope="module")
def trained(ctx):
    import paper_2306_00606_gb300 as ef
    x, y = _training_set(ctx)
    m = ef.Model(ctx.handle, seed=5)
    st = m.train(x, y, steps=1500, batch=4096, lr=2e-3, seed=9)
    return m, st, x, y


def test_training_lowers_the_loss(trained):
    m, st, x, y = trained
    assert st["last_loss"] < 0.05 * st["first_loss"], st


def test_model_save_load_roundtrip(ctx, trained, tmp_path):
    import torch
    import paper_2306_00606_gb300 as ef
    m, _, x, _ = trained
    path = tmp_path / "model.bin"
    m.save(str(path))
    m2 = ef.Model.load(ctx.handle, str(path))
    a = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    m.forward(x, a)
    m2.forward(x, b)
    assert torch.equal(a, b) and np.array_equal(m.get(), m2.get())


def _rank(ctx, model, g, cand_frac):
    import torch
    kt = math.ceil(0.01 * g.n)
    idx = torch.empty(kt, dtype=torch.int32, device="cuda")
    efv = torch.empty(kt, dtype=torch.float64, device="cuda")
    score = torch.empty(g.n, dtype=torch.float32, device="cuda")
    st = model.rank(_dev(g.row_ptr), _dev(g.col_idx), idx, efv, top_frac=0.01, cand_frac=cand_frac,
                    audit_frac=0.01, seed=3, out_score=score)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), efv.cpu().numpy(), score.cpu().numpy(), st


def test_rank_scores_equal_network_on_fp32_features(ctx, trained):
    """The ranking path writes its features standardised and rounded to BF16 (the network's first
    operand) and runs the network on those rows; every prediction equals the network's on the FP32
    rows of ef_features, bit for bit."""
    import torch
    import paper_2306_00606_gb300 as ef
    model = trained[0]
    g = synth.barabasi_albert(50000, 4, 61)
    _, _, score, _ = _rank(ctx, model, g, cand_frac=0.02)
    x = _features(ctx, g, ef.ef_model_feature_mode(model.handle))
    ref = torch.empty(g.n, dtype=torch.float32, device="cuda")
    model.forward(x, ref)
    torch.cuda.synchronize()
    assert np.array_equal(score, ref.cpu().numpy())


def test_ranking_recall_and_what_the_network_gains(ctx, trained):
    import paper_2306_00606_gb300 as ef
    model = trained[0]
    g = synth.barabasi_albert(200000, 4, 48)   # not seen in training
    exact = _exact_all(ctx, g)
    truth = set(sg.top_set(exact, 0.01).tolist())
    idx, efv, score, st = _rank(ctx, model, g, cand_frac=0.03)
    # the reported EF values are the exact ones, and the set is the top of the candidates
    np.testing.assert_allclose(efv, exact[idx], rtol=0, atol=2e-5)
    recall = len(truth & set(idx.tolist())) / len(truth)
    assert recall >= 0.95, (recall, st)
    assert st["n_candidates"] == math.ceil(0.03 * g.n) and st["spearman_audit"] > 0.9
    # without the trained network: the same network untrained, and ranking by degree
    raw = ef.Model(ctx.handle, seed=5)
    raw.set(np.concatenate([sg.flatten(sg.init_params(5)), model.get()[sg.N_PARAMS:]]).astype(np.float32))
    idx_raw, _, _, _ = _rank(ctx, raw, g, cand_frac=0.03)
    recall_raw = len(truth & set(idx_raw.tolist())) / len(truth)
    deg = np.diff(g.row_ptr).astype(np.float64)
    cand_deg = sg.top_set(deg, 0.03)
    top_deg = cand_deg[np.lexsort((cand_deg, -exact[cand_deg]))][:len(truth)]
    recall_deg = len(truth & set(top_deg.tolist())) / len(truth)
    print(f"top-1% recall: trained {recall:.4f}, untrained {recall_raw:.4f}, degree {recall_deg:.4f}")
    assert recall > recall_raw and recall > recall_deg, (recall, recall_raw, recall_deg)


def test_full_size_ranking_ba16m(ctx, trained):
    """BA n=1.6e7, m=4 at full size, as the bench ranks it: the reported EF of
    every returned node equals exact-all's, top-1% recall >= 0.95, and
    returned nodes below the top hubs against the vertex oracle."""
    model = trained[0]
    g = synth.workload(5)
    exact = _exact_all(ctx, g)
    idx, efv, score, st = _rank(ctx, model, g, cand_frac=0.02)
    np.testing.assert_allclose(efv, exact[idx], rtol=0, atol=2e-5)
    truth = set(sg.top_set(exact, 0.01).tolist())
    assert len(truth & set(idx.tolist())) / len(truth) >= 0.95
    deg = np.diff(g.row_ptr)
    cand = idx[deg[idx] < 4000]
    sample = cand[np.linspace(0, len(cand) - 1, 8).astype(int)]
    ref = oracle.vertex(g, sample)
    pos = {int(v): i for i, v in enumerate(idx)}
    np.testing.assert_allclose(efv[[pos[int(v)] for v in sample]], ref["EF"], rtol=0, atol=2e-5)
