"""Pins of the threshold formulas (Section 3.1, Section 3.2, Section 5, Algorithm 3)."""
import math

import numpy as np
import pytest

from oracle import cost_model as CM


def _grid_min(N, OUT):
    best = (math.inf, None)
    for e1 in np.linspace(0, math.log(N), 400):
        for e2 in np.linspace(0, math.log(N), 400):
            d1, d2 = math.exp(e1), math.exp(e2)
            f = CM.f_two_path(N, OUT, d1, d2)
            if f < best[0]:
                best = (f, (d1, d2))
    return best


@pytest.mark.parametrize("N,OUT", [(1e6, 1e3), (1e6, 1e5), (1e6, 1e6), (1e6, 1e8), (2e4, 7.3e5)])
def test_closed_form_is_the_grid_minimum(N, OUT):
    fmin, _ = _grid_min(N, OUT)
    d1, d2 = CM.closed_form(N, OUT)
    assert 1.0 <= d1 <= N and 1.0 <= d2 <= N
    f = CM.f_two_path(N, OUT, d1, d2)
    assert f <= fmin * (1 + 1e-6)
    assert f >= fmin * (1 - 0.02)        # the grid is fine enough to get within 2 %


def test_case1_critical_point():
    N, OUT = 1e6, 1e4                    # OUT <= N
    d1, d2 = CM.closed_form(N, OUT)
    # partial derivatives of N*d1 + OUT*d2 + N^2/(d1*d2) vanish there
    assert abs(N - N * N / (d2 * d1 * d1)) < 1e-6 * N
    assert abs(OUT - N * N / (d1 * d2 * d2)) < 1e-6 * OUT
    assert d1 <= d2


def test_case2_derivative_zero():
    N, OUT = 1e6, 1e9                    # OUT > N: border D1 = D2 = D
    d, d_ = CM.closed_form(N, OUT)
    assert d == d_
    assert abs(d ** 3 - 2 * N * N / (N + OUT)) < 1e-9 * d ** 3
    g = lambda t: (N + OUT) * t + N * N / (t * t)
    h = 1e-4 * d
    assert abs((g(d + h) - g(d - h)) / (2 * h)) < 1e-4 * (N + OUT)


@pytest.mark.parametrize("N,OUT", [(1e6, 1e3), (1e6, 1e6), (1e6, 1e9)])
def test_lemma3_time_matches_cost_order(N, OUT):
    d1, d2 = CM.closed_form(N, OUT)
    ratio = CM.f_two_path(N, OUT, d1, d2) / CM.lemma3_time(N, OUT)
    assert 0.5 < ratio < 5.0


def test_star_k3_worked_example_balances_terms():
    # Section 3.2 example: k = 3, OUT = N^(3/2), D2 = N^(6/16), D1 = N^(7/16)
    # makes all three cost terms N^(15/8)
    for N in (1e6, 1e8, 1e10):
        OUT = N ** 1.5
        terms = CM.star_cost_terms(N, OUT, N ** (7 / 16), N ** (6 / 16), 3)
        for t in terms:
            assert abs(math.log(t) - 15 / 8 * math.log(N)) < 1e-9
        # and the combinatorial bound of Lemma 2 (N * OUT^(2/3) = N^2) is worse
        assert sum(terms) < N * OUT ** (2 / 3)


def test_out_estimate_lies_between_bounds(oracle_mod):
    rng = np.random.default_rng(0)
    for _ in range(10):
        n = int(rng.integers(50, 2000))
        x = rng.integers(0, int(rng.integers(5, 300)), n)
        y = rng.integers(0, int(rng.integers(2, 100)), n)
        ux, uy = oracle_mod.normalise(x, y)
        N = len(ux)
        degy = np.unique(uy, return_counts=True)[1].astype(np.float64)
        oj = float((degy * degy).sum())
        domx = len(np.unique(ux))
        est = CM.out_estimate(domx, oj, N)
        out = len(oracle_mod.two_path(ux, uy)[0])
        lo = max(domx, (oj / N) ** 2)
        hi = min(domx * domx, oj)
        assert lo <= est * (1 + 1e-12) and est <= hi * (1 + 1e-12)
        assert domx <= out <= hi                       # the bounds themselves
        assert oj <= N * math.sqrt(out) * (1 + 1e-12)  # OUT_join <= N sqrt(OUT)


def test_degree_index_against_loops():
    rng = np.random.default_rng(1)
    x = rng.integers(0, 40, 300)
    y = rng.integers(0, 25, 300)
    key = np.unique(x * 1000 + y)
    x, y = key // 1000, key % 1000
    ux, degx = np.unique(x, return_counts=True)
    uy, degy = np.unique(y, return_counts=True)
    dy = dict(zip(uy.tolist(), degy.tolist()))
    dx = dict(zip(ux.tolist(), degx.tolist()))
    cand = {a: sum(dy[b] for b in y[x == a]) for a in ux.tolist()}
    idx = CM.DegreeIndex(degx, degy, [cand[a] for a in ux.tolist()])
    for delta in (0, 1, 2, 5, 9, 13, 100):
        assert idx.sum_y(delta) == sum(d * d for d in degy if d <= delta)
        assert idx.cdfx(delta) == sum(d for d in degy if d <= delta)
        assert idx.sum_x(delta) == sum(cand[a] for a in dx if dx[a] <= delta)
        assert idx.heavy_x(delta) == sum(1 for a in dx if dx[a] > delta)
        assert idx.heavy_y(delta) == sum(1 for d in degy if d > delta)


def _idx_from(x, y):
    ux, degx = np.unique(x, return_counts=True)
    uy, degy = np.unique(y, return_counts=True)
    dy = dict(zip(uy.tolist(), degy.tolist()))
    cand = [sum(dy[b] for b in y[x == a]) for a in ux.tolist()]
    return CM.DegreeIndex(degx, degy, cand)


def test_algorithm3_wcoj_switch_and_descent():
    rng = np.random.default_rng(2)
    x = rng.integers(0, 200, 4000)
    y = rng.integers(0, 40, 4000)
    key = np.unique(x * 1000 + y)
    x, y = key // 1000, key % 1000
    N = len(x)
    idx = _idx_from(x, y)
    degy = np.unique(y, return_counts=True)[1].astype(np.float64)
    oj = float((degy * degy).sum())
    # a full join of at most 20 N means plain worst-case optimal join
    assert CM.algorithm3(idx, N, 1e5, 1, 0, 0, lambda u, v, w: 0, out_join=19 * N)[2] == "wcoj"
    # a prohibitively expensive product keeps everything light
    d1, d2, _ = CM.algorithm3(idx, N, 3e4, 1e-9, 0, 0, lambda u, v, w: 1e30, out_join=oj)
    assert idx.heavy_x(d2) == 0 or idx.heavy_y(d1) == 0
    # a free product with expensive light work descends until heavy parts exist
    d1, d2, _ = CM.algorithm3(idx, N, 3e4, 1.0, 0, 0, lambda u, v, w: 0.0, out_join=oj)
    assert idx.heavy_x(d2) > 0 and idx.heavy_y(d1) > 0
    assert 1 <= d1 <= N and 1 <= d2 <= N


def test_star_grid_minimum_reaches_the_worked_example_exponent():
    # Section 3.2 example (k = 3, OUT = N^(3/2)): the paper's thresholds give
    # running time N^(15/8); the grid minimum of the same cost can only be
    # lower, and is of the same order
    for N in (1e6, 1e8, 1e10):
        OUT = N ** 1.5
        d1, d2 = CM.star_grid_thresholds(int(N), OUT, 3)
        best = CM.star_cost(N, OUT, d1, d2, 3)
        paper = CM.star_cost(N, OUT, N ** (7 / 16), N ** (6 / 16), 3)
        assert best <= paper * (1 + 1e-12)
        assert 0.5 * N ** (15 / 8) <= best
