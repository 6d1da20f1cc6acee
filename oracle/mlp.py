"""Learned threshold predictor: features and MLP -- TEST INFRASTRUCTURE ONLY.

The predictor maps a relation's degree distribution to thresholds
(log Delta1, log Delta2).  Its features are two 64-bin log-degree histograms
(x degrees and y degrees): bin(d) = min(63, floor(4 * log2 d)) =
min(63, floor(log2 d^4)), computed exactly here with Python integers, and
each bin's count c enters as log2(1 + c) / 32, which keeps the relation's
scale (a relation twice as large moves every populated bin up by about 1/32;
fractions of the domain would hide it, while the best thresholds grow with N,
Lemma 3).  The network is a plain MLP
128 -> 256 -> 256 -> 2 with ReLU, weights rounded to bfloat16 and all
arithmetic in float64.  The backward pass is the chain rule of that forward
pass written out; it is pinned against finite differences in the tests.
"""
from __future__ import annotations

import numpy as np

NBIN = 64
DIMS = (128, 256, 256, 2)


def log_degree_bin(d: int) -> int:
    """floor(4 log2 d) for d >= 1, capped at 63 (exact: bit length of d^4 minus 1)."""
    if d < 1:
        raise ValueError("degree must be >= 1")
    return min(NBIN - 1, (int(d) ** 4).bit_length() - 1)


def histogram(degrees) -> np.ndarray:
    """64-bin log-degree histogram: the number of values with degree >= 1 per bin."""
    h = np.zeros(NBIN, np.float64)
    for d in degrees:
        if int(d) >= 1:
            h[log_degree_bin(int(d))] += 1
    return h


def bin_feature(counts) -> np.ndarray:
    """The network input of a bin holding c values: log2(1 + c) / 32."""
    return np.log2(1.0 + np.asarray(counts, np.float64)) / 32.0


def features(degx, degy) -> np.ndarray:
    return np.concatenate([bin_feature(histogram(degx)), bin_feature(histogram(degy))])


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed: int = 0):
    """He-style initial weights (float64) for the 128-256-256-2 network."""
    rng = np.random.default_rng(seed)
    params = []
    for i in range(3):
        fan_in, fan_out = DIMS[i], DIMS[i + 1]
        W = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=(fan_in, fan_out))
        b = np.zeros(fan_out)
        params += [W, b]
    return params


def forward(params, X):
    """Returns (Y, cache).  X: (B, 128)."""
    W1, b1, W2, b2, W3, b3 = params
    Z1 = X @ W1 + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2 + b2
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ W3 + b3
    return Y, (X, Z1, H1, Z2, H2)


def mse(Y, T) -> float:
    return float(np.mean(np.sum((Y - T) ** 2, axis=1)))


def backward(params, cache, Y, T):
    """Gradients of mse(Y, T) = mean over the batch of ||Y - T||^2."""
    W1, b1, W2, b2, W3, b3 = params
    X, Z1, H1, Z2, H2 = cache
    B = X.shape[0]
    dY = 2.0 * (Y - T) / B
    dW3 = H2.T @ dY
    db3 = dY.sum(axis=0)
    dH2 = dY @ W3.T
    dZ2 = dH2 * (Z2 > 0)
    dW2 = H1.T @ dZ2
    db2 = dZ2.sum(axis=0)
    dH1 = dZ2 @ W2.T
    dZ1 = dH1 * (Z1 > 0)
    dW1 = X.T @ dZ1
    db1 = dZ1.sum(axis=0)
    return [dW1, db1, dW2, db2, dW3, db3]


def adam_update(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (bias-corrected), returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for p, g, mi, vi in zip(params, grads, m, v):
        mi = beta1 * mi + (1 - beta1) * g
        vi = beta2 * vi + (1 - beta2) * g * g
        mh = mi / (1 - beta1 ** step)
        vh = vi / (1 - beta2 ** step)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mi)
        out_v.append(vi)
    return out_p, out_m, out_v
