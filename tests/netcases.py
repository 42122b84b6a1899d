"""Inputs for the surrogate network's tests (no arithmetic of the method here)."""
import numpy as np

from oracle import surrogate as sg


def dyadic_network(seed, rows):
    """A network and inputs of few-bit dyadic values: features in {-1, 0, 1}
    (standardisation mean 0, std 1), W1 in {0, +-1/4}, W2 in {0, +-1/8}
    with four non-zeros per row and per column, w3 = +-1/2, dyadic biases,
    and labels 1 or 2 away from the prediction.  Every product operand is
    then a BF16 number and every sum is exact in FP32 and FP64, so BF16
    operands with FP32 sums give exactly the FP64 result."""
    rng = np.random.default_rng(seed)
    X = rng.integers(-1, 2, size=(rows, 16)).astype(np.float64)
    p = {"W1": rng.integers(-1, 2, size=(16, 64)) / 4.0, "b1": rng.integers(-2, 3, size=64) / 4.0,
         "b2": rng.integers(-4, 5, size=64) / 32.0, "w3": rng.choice([-0.5, 0.5], size=64), "b3": 0.5,
         "mean": np.zeros(16), "std": np.ones(16)}
    W2 = np.zeros((64, 64))
    for _ in range(4):   # four signed permutation matrices
        W2[np.arange(64), rng.permutation(64)] = rng.choice([-0.125, 0.125], size=64)
    p["W2"] = W2
    out, _ = sg.forward(p, X)
    y = out - rng.choice([-2.0, -1.0, 1.0, 2.0], size=rows)
    return p, X, y
