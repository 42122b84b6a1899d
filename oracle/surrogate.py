"""TEST INFRASTRUCTURE ONLY: CPU oracle of the learned ranking path, in FP64.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU legs may
import this module.  It shares no code with the CUDA library.

The learned path ranks nodes by a small regression network on cheap local
features, then recomputes exact EF on the top candidates and on a random
audit sample.  The paper has no learned part; this follows the build's own
definition:

* ``features``   -- 16 per-node features from degrees, neighbour-degree
  moments, 2-hop sums, the closed forms of the cluster count N and degree
  sum S (Algorithm 1's credits), and triangles;
* ``forward`` / ``loss_and_grads`` -- the network 16-64-64-1 with ReLU on
  standardised features and a mean-squared-error loss, written out as plain
  matrix products;
* ``adam``       -- one Adam step (Kingma and Ba, "Adam: a method for
  stochastic optimization", Algorithm 1);
* ``bf16`` and ``operands="bf16"`` of ``forward`` / ``loss_and_grads`` --
  the same network with the operands of every matrix product rounded to
  BF16 (the network's stated precision: BF16 operands, sums kept wide),
  and ``grad_term_sums``, the size of the terms each gradient element sums;
* ``spearman`` and ``topk_recall`` -- the quality measures.

Parameters are a dict of float64 arrays: W1 (16, 64), b1 (64), W2 (64, 64),
b2 (64), w3 (64), b3 (scalar), and the standardisation mean (16) and std
(16).  ``flatten`` gives the trained ones in the library's order: W1
row-major, b1, W2 row-major (W2[i, j] joins hidden unit i of layer 1 to unit
j of layer 2), b2, w3, b3.
"""
from __future__ import annotations

import math

import numpy as np

NF, H = 16, 64
TRAINED = ("W1", "b1", "W2", "b2", "w3", "b3")
SHAPES = {"W1": (NF, H), "b1": (H,), "W2": (H, H), "b2": (H,), "w3": (H,), "b3": ()}
N_PARAMS = sum(int(np.prod(SHAPES[k])) for k in TRAINED)   # 5377

FEATURE_NAMES = (
    "ln(1+D)", "ln(1+sigma1)", "ln(1+sigma2)", "ln(1+omega)", "ln(1+mean nbr deg)", "ln(1+sd nbr deg)",
    "ln(1+min nbr deg)", "ln(1+max nbr deg)", "ln(1+N)", "ln(1+S_open)", "ln(1+S_open)-ln(1+N)", "ln(1+t)",
    "clustering", "ln(1+S)", "ln(1+sigma2)-ln(1+sigma1)", "ln(1+omega)-ln(1+sigma1)")


def features(g, triangles=None) -> np.ndarray:
    """The 16 features of every node, float64 [n, 16].

    D = degree; sigma1, sigma2 = sum of neighbour degrees and of their
    squares; omega = sum over neighbours of their sigma1; min / max neighbour
    degree; N = D(D-2) + sigma1 (clusters credited to the node, Algorithm 1's
    weights 2/1/1); S_open = the credited degree sum with every cluster at
    its open degree D_i + D_u + D_j - 4; S = S_open - 8 t, t = triangles at
    the node (pass t = None for the features without triangles: t = 0).
    """
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    ci = np.asarray(g.col_idx, dtype=np.int64)
    n = rp.shape[0] - 1
    D = np.diff(rp).astype(np.float64)
    src = np.repeat(np.arange(n), np.diff(rp))
    Dn = D[ci]
    s1 = np.bincount(src, weights=Dn, minlength=n)
    s2 = np.bincount(src, weights=Dn * Dn, minlength=n)
    om = np.bincount(src, weights=s1[ci], minlength=n)
    dmin = np.zeros(n)
    dmax = np.zeros(n)
    for v in range(n):   # plain per-row loop
        if rp[v + 1] > rp[v]:
            row = Dn[rp[v]:rp[v + 1]]
            dmin[v] = row.min()
            dmax[v] = row.max()
    t = np.zeros(n) if triangles is None else np.asarray(triangles, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        mean = np.where(D > 0, s1 / np.where(D > 0, D, 1), 0.0)
        var = np.where(D > 0, s2 / np.where(D > 0, D, 1) - mean * mean, 0.0)
    sd = np.sqrt(np.maximum(var, 0.0))
    N = D * (D - 2) + s1
    S_open = D * (D - 1) * (D - 4) + 2 * (D - 1) * s1 + s2 - s1 + (D - 4) * (s1 - D) + om - D * D
    S = S_open - 8 * t
    pairs = D * (D - 1) / 2
    clus = np.where(pairs > 0, t / np.where(pairs > 0, pairs, 1), 0.0)
    L = np.log1p
    X = np.stack([L(D), L(s1), L(s2), L(om), L(mean), L(sd), L(dmin), L(dmax), L(N), L(S_open),
                  L(S_open) - L(N), L(t), clus, L(S), L(s2) - L(s1), L(om) - L(s1)], axis=1)
    return X


def init_params(seed: int, mean=None, std=None) -> dict:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for k in TRAINED:
        shp = SHAPES[k]
        if k.startswith("b"):
            p[k] = np.zeros(shp)
        else:
            fan_in = shp[0]
            p[k] = rng.uniform(-1, 1, size=shp) / math.sqrt(fan_in)
    p["mean"] = np.zeros(NF) if mean is None else np.asarray(mean, dtype=np.float64)
    p["std"] = np.ones(NF) if std is None else np.asarray(std, dtype=np.float64)
    return p


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.atleast_1d(np.asarray(p[k], dtype=np.float64)).ravel() for k in TRAINED])


def unflatten(flat, mean=None, std=None) -> dict:
    flat = np.asarray(flat, dtype=np.float64)
    p, o = {}, 0
    for k in TRAINED:
        size = int(np.prod(SHAPES[k]))
        p[k] = flat[o:o + size].reshape(SHAPES[k]) if SHAPES[k] else flat[o]
        o += size
    p["mean"] = np.zeros(NF) if mean is None else np.asarray(mean, dtype=np.float64)
    p["std"] = np.ones(NF) if std is None else np.asarray(std, dtype=np.float64)
    return p


def standardize(p: dict, X) -> np.ndarray:
    return (np.asarray(X, dtype=np.float64) - p["mean"]) / p["std"]


def bf16(a) -> np.ndarray:
    """Round to the nearest BF16 value, ties to even, returned as float64.

    BF16 keeps the sign, the 8-bit exponent and the 7 leading stored
    significand bits of an IEEE binary32 number.  In binary64 that is the
    top 8 bits of the 53-bit significand, so the rounding drops the low 45
    stored bits (normal values; the network's values stay far from BF16's
    range limits).
    """
    a = np.ascontiguousarray(a, dtype=np.float64)
    u = a.view(np.uint64)
    low = np.uint64((1 << 45) - 1)
    odd = (u >> np.uint64(45)) & np.uint64(1)
    r = (u + (low >> np.uint64(1)) + odd) & ~low
    return r.view(np.float64)


def _op(a, operands):
    return bf16(a) if operands == "bf16" else a


def forward(p: dict, X, operands: str = "fp64") -> tuple[np.ndarray, dict]:
    """Prediction for each row of X (raw features) and the activations.

    operands="bf16" rounds both operands of the two hidden-layer matrix
    products to BF16 (standardised features, hidden activations, weights);
    sums, biases, ReLU and the output layer stay in FP64.
    """
    Z = standardize(p, X)
    A1 = _op(Z, operands) @ _op(p["W1"], operands) + p["b1"]
    H1 = np.maximum(A1, 0.0)
    A2 = _op(H1, operands) @ _op(p["W2"], operands) + p["b2"]
    H2 = np.maximum(A2, 0.0)
    out = H2 @ p["w3"] + p["b3"]
    return out, dict(Z=Z, A1=A1, H1=H1, A2=A2, H2=H2)


def loss_and_grads(p: dict, X, y, operands: str = "fp64") -> tuple[float, dict]:
    """L = mean over rows of (prediction - y)^2 and its gradient (chain rule).

    operands="bf16" also rounds to BF16 the operands of the backward matrix
    products: the layer-2 errors and W2 for the layer-1 errors, and the
    activations and errors whose products form the weight gradients of W1
    and W2.  Bias gradients and the output layer's stay in FP64.
    """
    y = np.asarray(y, dtype=np.float64)
    out, a = forward(p, X, operands)
    B = out.shape[0]
    r = out - y
    L = float(np.mean(r * r))
    d_out = 2.0 * r / B
    g = {"b3": float(d_out.sum()), "w3": a["H2"].T @ d_out}
    d_A2 = np.outer(d_out, p["w3"]) * (a["A2"] > 0)
    g["W2"] = _op(a["H1"], operands).T @ _op(d_A2, operands)
    g["b2"] = d_A2.sum(axis=0)
    d_A1 = (_op(d_A2, operands) @ _op(p["W2"], operands).T) * (a["A1"] > 0)
    g["W1"] = _op(a["Z"], operands).T @ _op(d_A1, operands)
    g["b1"] = d_A1.sum(axis=0)
    return L, g


def grad_term_sums(p: dict, X, y, operands: str = "fp64") -> tuple[dict, dict]:
    """For every gradient element, the sum and the largest of the absolute
    values of the per-row terms it adds up (same products as
    ``loss_and_grads``): the scale against which rounding in those terms is
    measured.  Returns (sums, maxima), keyed like the gradient."""
    y = np.asarray(y, dtype=np.float64)
    out, a = forward(p, X, operands)
    B = out.shape[0]
    d_out = 2.0 * (out - y) / B
    d_A2 = np.outer(d_out, p["w3"]) * (a["A2"] > 0)
    d_A1 = (_op(d_A2, operands) @ _op(p["W2"], operands).T) * (a["A1"] > 0)
    pairs = {"w3": (a["H2"], d_out[:, None]), "b3": (np.ones((B, 1)), d_out[:, None]),
             "W2": (_op(a["H1"], operands), _op(d_A2, operands)), "b2": (np.ones((B, 1)), d_A2),
             "W1": (_op(a["Z"], operands), _op(d_A1, operands)), "b1": (np.ones((B, 1)), d_A1)}
    sums, maxima = {}, {}
    for k, (u, v) in pairs.items():
        au, av = np.abs(u), np.abs(v)
        s = au.T @ av
        mx = np.max(au[:, :, None] * av[:, None, :], axis=0)
        if k in ("w3",):
            s, mx = s[:, 0], mx[:, 0]
        elif k in ("b3",):
            s, mx = float(s[0, 0]), float(mx[0, 0])
        elif k in ("b1", "b2"):
            s, mx = s[0], mx[0]
        sums[k], maxima[k] = s, mx
    return sums, maxima


def adam(p: dict, g: dict, m: dict, v: dict, step: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8) -> None:
    """One Adam update in place; `step` counts from 1."""
    for k in TRAINED:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = m[k] / (1 - b1 ** step)
        vh = v[k] / (1 - b2 ** step)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def ranks(a) -> np.ndarray:
    """Ranks 1..n with ties given their average rank."""
    a = np.asarray(a)
    order = np.argsort(a, kind="mergesort")
    r = np.empty(len(a), dtype=np.float64)
    sa = a[order]
    i = 0
    while i < len(a):
        j = i
        while j + 1 < len(a) and sa[j + 1] == sa[i]:
            j += 1
        r[order[i:j + 1]] = (i + j) / 2.0 + 1.0
        i = j + 1
    return r


def spearman(a, b) -> float:
    """Spearman's rank correlation: Pearson correlation of the ranks."""
    ra, rb = ranks(a), ranks(b)
    ra -= ra.mean()
    rb -= rb.mean()
    den = math.sqrt(float((ra * ra).sum() * (rb * rb).sum()))
    return float((ra * rb).sum() / den) if den > 0 else 0.0


def top_set(a, frac: float) -> np.ndarray:
    """Indices of the ceil(frac n) largest values (ties to the smaller index)."""
    a = np.asarray(a)
    k = int(math.ceil(frac * len(a)))
    order = np.lexsort((np.arange(len(a)), -a))
    return order[:k]


def topk_recall(pred, exact, frac: float) -> float:
    """Fraction of the exact top ceil(frac n) that the predicted top set holds."""
    t = top_set(exact, frac)
    s = top_set(pred, frac)
    return len(np.intersect1d(t, s)) / max(len(t), 1)
