"""Pins for the CPU oracle of the learned ranking path (oracle/surrogate.py).

None of these compares the oracle with itself:
- features on graph families whose degree sums are known in closed form;
- the cluster-count and degree-sum features against Algorithm 1's literal
  C oracle;
- gradients against central finite differences;
- the forward pass in its linear regime against one composed affine map;
- Adam's first step against its closed form;
- Spearman's rho against SciPy;
- recall on hand-made cases;
- BF16 rounding against PyTorch's float32 -> bfloat16 conversion and hand
  ties; the BF16-operand network against the FP64 one on a network whose
  operands are all BF16 numbers with exact sums (they must agree exactly);
- the gradient term sums against |gradient| where every term is >= 0.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import surrogate as sg
from netcases import dyadic_network


def test_feature_count_and_names():
    assert len(sg.FEATURE_NAMES) == sg.NF == 16 and sg.N_PARAMS == 16 * 64 + 64 + 64 * 64 + 64 + 64 + 1


def test_features_star_closed_form():
    k = 9
    g = synth.star(k)   # centre 0, leaves 1..k
    X = sg.features(g, triangles=np.zeros(g.n))
    L = np.log1p
    c = X[0]
    # centre: D = k, neighbours all of degree 1; omega = k * sigma1(leaf) = k * k
    assert np.allclose(c[[0, 1, 2, 3, 6, 7]], [L(k), L(k), L(k), L(k * k), L(1), L(1)])
    assert np.isclose(c[8], L(k * (k - 2) + k))            # N = k(k-1)
    leaf = X[1]
    # leaf: D = 1, its neighbour has degree k; omega = sigma1(centre) = k
    assert np.allclose(leaf[[0, 1, 2, 3, 4, 5]], [L(1), L(k), L(k * k), L(k), L(k), 0.0])
    assert np.isclose(leaf[8], L(k - 1))


def test_features_complete_graph_closed_form():
    n = 7
    g = synth.complete(n)
    t = np.full(n, math.comb(n - 1, 2))
    X = sg.features(g, triangles=t)
    d = n - 1
    L = np.log1p
    assert np.allclose(X[:, 0], L(d)) and np.allclose(X[:, 1], L(d * d)) and np.allclose(X[:, 2], L(d ** 3))
    assert np.allclose(X[:, 3], L(d * d * d)) and np.allclose(X[:, 12], 1.0)
    # every cluster is a triangle of degree 3(n-3): S = N * 3(n-3)
    N = 2 * (n - 1) * (n - 2)
    assert np.allclose(X[:, 8], L(N)) and np.allclose(X[:, 13], L(N * 3 * (n - 3)))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_count_and_degree_sum_features_match_algorithm_1(seed):
    g = synth.erdos_renyi(120, 0.08, seed)
    ref = oracle.alg1(g)
    t = oracle.triangles(g)
    X = sg.features(g, triangles=t)
    np.testing.assert_allclose(np.expm1(X[:, 8]), ref["N"], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(np.expm1(X[:, 13]), ref["S"], rtol=1e-12, atol=1e-9)
    # without triangles the degree-sum feature is the open-degree sum S + 8t
    X0 = sg.features(g)
    np.testing.assert_allclose(np.expm1(X0[:, 9]), ref["S"] + 8 * t, rtol=1e-12, atol=1e-9)


def _data(seed, B=37):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, 16)) * 2 + 1
    y = rng.normal(size=B)
    p = sg.init_params(seed, mean=rng.normal(size=16) * 0.1, std=rng.uniform(0.5, 2, size=16))
    for k in ("b1", "b2"):
        p[k] = rng.normal(size=p[k].shape) * 0.1
    p["b3"] = 0.3
    return p, X, y


@pytest.mark.parametrize("seed", [0, 1])
def test_gradients_match_finite_differences(seed):
    p, X, y = _data(seed)
    L, g = sg.loss_and_grads(p, X, y)
    flat = sg.flatten(p)
    gflat = sg.flatten(g)
    rng = np.random.default_rng(seed + 100)
    idx = rng.choice(flat.size, size=120, replace=False)
    h = 1e-6
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        Lp = sg.loss_and_grads(sg.unflatten(fp, p["mean"], p["std"]), X, y)[0]
        Lm = sg.loss_and_grads(sg.unflatten(fm, p["mean"], p["std"]), X, y)[0]
        num = (Lp - Lm) / (2 * h)
        assert abs(num - gflat[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, gflat[i])


def test_forward_linear_regime_is_one_affine_map():
    rng = np.random.default_rng(5)
    p = sg.init_params(5)
    p["W1"] = np.abs(p["W1"])
    p["W2"] = np.abs(p["W2"])
    p["b1"] = np.full(64, 0.5)
    p["b2"] = np.full(64, 0.5)
    X = np.abs(rng.normal(size=(20, 16)))   # all pre-activations positive: ReLU is the identity
    out, _ = sg.forward(p, X)
    M = p["W1"] @ p["W2"] @ p["w3"]
    c = (p["b1"] @ p["W2"] + p["b2"]) @ p["w3"] + p["b3"]
    np.testing.assert_allclose(out, X @ M + c, rtol=1e-12)


def test_adam_first_step_closed_form():
    p, X, y = _data(3)
    _, g = sg.loss_and_grads(p, X, y)
    m = {k: np.zeros_like(np.asarray(p[k], dtype=float)) for k in sg.TRAINED}
    v = {k: np.zeros_like(np.asarray(p[k], dtype=float)) for k in sg.TRAINED}
    before = sg.flatten(p)
    sg.adam(p, g, m, v, 1, lr=0.01, eps=1e-8)
    gf = sg.flatten(g)
    # after one step from zero moments the update is lr * g / (|g| + eps)
    np.testing.assert_allclose(sg.flatten(p), before - 0.01 * gf / (np.abs(gf) + 1e-8), rtol=1e-12, atol=1e-15)


def test_spearman_matches_scipy():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(7)
    a = rng.integers(0, 20, size=300).astype(float)   # many ties
    b = a + rng.normal(size=300) * 3
    assert math.isclose(sg.spearman(a, b), stats.spearmanr(a, b).correlation, rel_tol=1e-12)


def test_topk_recall_hand_cases():
    exact = np.array([5.0, 4.0, 3.0, 2.0, 1.0, 0.0, -1.0, -2.0, -3.0, -4.0])
    assert sg.topk_recall(exact, exact, 0.2) == 1.0
    assert sg.topk_recall(-exact, exact, 0.2) == 0.0
    pred = exact.copy()
    pred[1] = -10   # the second-best node is predicted worst
    assert sg.topk_recall(pred, exact, 0.2) == 0.5
    assert list(sg.top_set(np.zeros(5), 0.4)) == [0, 1]   # ties go to the smaller index


def test_bf16_rounding_matches_torch_and_hand_ties():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-6, 6, size=20000),
                        [1.0, -1.0, 0.0, 3.0, 1e-3]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(sg.bf16(x.astype(np.float64)), ref)
    # 8 significant bits: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 (ties to
    # the even 1); 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6
    # (ties to the even 1 + 2^-6); anything above a midpoint rounds up; 96.5
    # has 8 significant bits, 96.25 and 96.75 are ties (to 96 and 97)
    hand = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -30, -(1 + 2.0 ** -7), 96.5,
                     96.25, 96.75])
    np.testing.assert_array_equal(sg.bf16(hand), [1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -(1 + 2.0 ** -7), 96.5,
                                                  96.0, 97.0])


@pytest.mark.parametrize("seed", [7, 8])
def test_bf16_network_equals_fp64_when_operands_are_bf16_exact(seed):
    p, X, y = dyadic_network(seed, 64)
    for k in ("W1", "W2"):
        assert np.array_equal(sg.bf16(p[k]), p[k])
    out64, a64 = sg.forward(p, X)
    out16, a16 = sg.forward(p, X, operands="bf16")
    np.testing.assert_array_equal(out16, out64)
    L64, g64 = sg.loss_and_grads(p, X, y)
    L16, g16 = sg.loss_and_grads(p, X, y, operands="bf16")
    assert L16 == L64
    np.testing.assert_array_equal(sg.flatten(g16), sg.flatten(g64))
    # and the bf16 mode does round: on generic values it differs from FP64
    q, Xq, yq = _data(seed)
    assert not np.array_equal(sg.forward(q, Xq, operands="bf16")[0], sg.forward(q, Xq)[0])


def test_grad_term_sums_equal_gradient_when_terms_are_nonnegative():
    rng = np.random.default_rng(12)
    p = sg.init_params(12)
    for k in ("W1", "W2", "w3"):
        p[k] = np.abs(p[k])
    p["b1"] = np.full(64, 0.1)
    p["b2"] = np.full(64, 0.1)
    X = np.abs(rng.normal(size=(30, 16)))     # mean 0, std 1: every activation > 0
    out, _ = sg.forward(p, X)
    y = out - rng.uniform(0.5, 1.0, size=30)   # every error > 0: every term >= 0
    _, g = sg.loss_and_grads(p, X, y)
    sums, maxima = sg.grad_term_sums(p, X, y)
    for k in sg.TRAINED:
        np.testing.assert_allclose(np.ravel(sums[k]), np.ravel(np.abs(g[k])), rtol=1e-12)
        assert np.all(np.ravel(maxima[k]) <= np.ravel(sums[k]) * (1 + 1e-12))
    # with mixed signs the sums bound the gradient
    q, Xq, yq = _data(2)
    _, gq = sg.loss_and_grads(q, Xq, yq)
    sq, _ = sg.grad_term_sums(q, Xq, yq)
    for k in sg.TRAINED:
        assert np.all(np.abs(np.ravel(gq[k])) <= np.ravel(sq[k]) * (1 + 1e-12))
