"""Pins of the learned-predictor oracle (features and MLP gradients)."""
import math

import numpy as np
import pytest

from oracle import mlp as M


def test_log_degree_bins_match_the_definition():
    # floor(4 log2 d): exact powers and quarter-octave boundaries
    assert M.log_degree_bin(1) == 0
    assert M.log_degree_bin(2) == 4
    assert M.log_degree_bin(3) == 6            # 4 * 1.585 = 6.34
    assert M.log_degree_bin(16) == 16
    assert M.log_degree_bin(65536) == 63       # 4 * 16 = 64, capped
    for d in list(range(1, 5000)) + [2 ** 20 - 1, 2 ** 20, 10 ** 7]:
        f = 4.0 * math.log2(d)
        b = min(63, math.floor(f))
        if abs(f - round(f)) > 1e-9:            # away from ties the float agrees
            assert M.log_degree_bin(d) == b
        # the exact definition: 2^bin <= d^4 < 2^(bin+1) below the cap
        k = M.log_degree_bin(d)
        if k < 63:
            assert 2 ** k <= d ** 4 < 2 ** (k + 1)


def test_histogram_counts_and_bin_feature_scale():
    rng = np.random.default_rng(0)
    d = rng.integers(1, 10 ** 6, 1000)
    h = M.histogram(d)
    assert h.shape == (64,) and h.sum() == 1000 and (h >= 0).all()
    assert M.histogram([0, 0]).sum() == 0.0
    # log2(1 + c) / 32: empty bins give 0, one value 1/32, 2^32 - 1 values 1
    assert M.bin_feature([0, 1, 3, 2 ** 32 - 1]).tolist() == [0.0, 1 / 32, 2 / 32, 1.0]
    # doubling a bin's population (c -> 2c + 1) raises its feature by exactly 1/32
    c = rng.integers(0, 10 ** 9, 100).astype(np.float64)
    assert np.allclose(M.bin_feature(2 * c + 1) - M.bin_feature(c), 1 / 32, atol=1e-15)
    # a relation with every degree count doubled sees every populated bin move up
    f1 = M.features(d, d)
    f2 = M.features(np.repeat(d, 2), np.repeat(d, 2))
    pop = M.histogram(d) > 0
    assert (f2[:64][pop] > f1[:64][pop]).all() and (f2[:64][~pop] == 0).all()


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 3.14159, -2.5e-3, 65504.0])
    r = M.bf16_round(x)
    assert r[0] == 1.0 and r[2] == 1.0 + 2 ** -7
    assert r[1] == 1.0                          # tie rounds to even
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    params = M.init_params(3)
    X = rng.random((5, 128))
    T = rng.normal(size=(5, 2))
    Y, cache = M.forward(params, X)
    grads = M.backward(params, cache, Y, T)
    h = 1e-6
    for pi, g in zip(range(6), grads):
        P = params[pi]
        for idx in [tuple(rng.integers(0, s) for s in P.shape) for _ in range(6)]:
            old = P[idx]
            P[idx] = old + h
            lp = M.mse(M.forward(params, X)[0], T)
            P[idx] = old - h
            lm = M.mse(M.forward(params, X)[0], T)
            P[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[idx]) <= 1e-5 * max(1.0, abs(fd)), (pi, idx, fd, g[idx])


def test_adam_first_step_moves_by_lr():
    p = [np.array([1.0, -2.0])]
    g = [np.array([0.5, -3.0])]
    m = [np.zeros(2)]
    v = [np.zeros(2)]
    q, _, _ = M.adam_update(p, g, m, v, 1, 0.01)
    # bias-corrected first step is lr * sign(g) (up to eps)
    assert np.allclose(q[0], p[0] - 0.01 * np.sign(g[0]), atol=1e-8)
