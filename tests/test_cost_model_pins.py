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
    idx = CM.DegreeIndex(degx, [cand[a] for a in ux.tolist()], degy)
    for delta in (0, 1, 2, 5, 9, 13, 100):
        assert idx.sum_y(delta) == sum(d * d for d in degy if d <= delta)
        assert idx.cdfx(delta) == sum(d for d in degy if d <= delta)
        assert idx.sum_x(delta) == sum(cand[a] for a in dx if dx[a] <= delta)
        assert idx.heavy_x(delta) == sum(1 for a in dx if dx[a] > delta)
        assert idx.heavy_y(delta) == sum(1 for d in degy if d > delta)
        assert idx.heavy_z(delta) == idx.heavy_x(delta)


def test_index_of_relations_r_ne_s_against_loops():
    """R != S: R's dangling tuples dropped, y degree max(deg_R, deg_S), products deg_R deg_S."""
    rng = np.random.default_rng(3)
    rx = rng.integers(-30, 30, 400)
    ry = rng.integers(-12, 20, 400)          # y in [12, 20) never occurs in S: dangling
    sz = rng.integers(-50, 10, 500)
    sy = rng.integers(-15, 12, 500)          # y in [-15, -12) only in S
    R = sorted(set(zip(rx.tolist(), ry.tolist())))
    S = sorted(set(zip(sz.tolist(), sy.tolist())))
    ys = {b for _, b in S}
    R = [(a, b) for a, b in R if b in ys]
    degr, degs, degx, degz = {}, {}, {}, {}
    for a, b in R:
        degr[b] = degr.get(b, 0) + 1
        degx[a] = degx.get(a, 0) + 1
    for c, b in S:
        degs[b] = degs.get(b, 0) + 1
        degz[c] = degz.get(c, 0) + 1
    cand = {a: sum(degs[b] for x_, b in R if x_ == a) for a in degx}
    idx, info = CM.index_of_relations(rx, ry, sz, sy)
    assert info["n_r"] == len(R) and info["n_s"] == len(S)
    assert info["N"] == max(len(R), len(S))
    assert info["dom_x"] == len(degx) and info["dom_y"] == len(ys) and info["dom_z"] == len(degz)
    assert info["out_join"] == sum(degr.get(b, 0) * degs[b] for b in ys)
    assert info["out_join"] == sum(1 for a, b in R for c, b2 in S if b == b2)
    ymax = {b: max(degr.get(b, 0), degs[b]) for b in ys}
    for delta in (0, 1, 2, 3, 5, 8, 13, 40):
        assert idx.sum_y(delta) == sum(degr.get(b, 0) * degs[b] for b in ys if ymax[b] <= delta)
        assert idx.cdfx(delta) == sum(degr.get(b, 0) for b in ys if ymax[b] <= delta)
        assert idx.sum_x(delta) == sum(cand[a] for a in degx if degx[a] <= delta)
        assert idx.heavy_x(delta) == sum(1 for a in degx if degx[a] > delta)
        assert idx.heavy_y(delta) == sum(1 for b in ys if ymax[b] > delta)
        assert idx.heavy_z(delta) == sum(1 for c in degz if degz[c] > delta)


def _idx_from(x, y):
    return CM.index_of_relations(x, y)[0]


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


# A six-value degree index on which Algorithm 3 is worked out by hand.
#   x degrees 1, 2, 4, 8, 16, 32 with cand = 10 * degree: 10, 20, 40, 80, 160, 320
#   y degrees (deg_R = deg_S) 1, 2, 4, 8, 16, 32: deg_R * deg_S = 1, 4, 16, 64, 256, 1024
#   so, for delta = 64, 32, 16, 8, 4, 2, 1:
#     sum_y  = 1365, 1365, 341, 85, 21, 5, 1       cdfx = 63, 63, 31, 15, 7, 3, 1
#     sum_x  = 630,  630,  310, 150, 70, 30, 10    heavy_x = heavy_y = 0, 0, 1, 2, 3, 4, 5
_DEG = [1, 2, 4, 8, 16, 32]


def _hand_index(degz=None):
    return CM.DegreeIndex(_DEG, [10 * d for d in _DEG], _DEG, _DEG, degz)


# Run A: N = OUT = 64 (so Delta2 = Delta1), eps = 0.5 (Delta1 halves), T_I = 1,
# T_s = T_m = 0, mhat = 20 u v w.
#   D1=64: light 1365 + 630 = 1995, u = 0: no product           -> 1995
#   D1=32: the same degrees are light                            -> 1995 (not larger: go on)
#   D1=16: light 341 + 310 = 651, u = v = w = 1: 20              -> 671
#   D1=8:  light 85 + 150 = 235, u = v = w = 2: 160              -> 395
#   D1=4:  light 21 + 70 = 91,   u = v = w = 3: 540              -> 631 > 395: stop at (8, 8)
_RUN_A = [(64.0, 64.0, 1995.0), (32.0, 32.0, 1995.0), (16.0, 16.0, 671.0), (8.0, 8.0, 395.0),
          (4.0, 4.0, 631.0)]
# Run B: N = 64, OUT = 128 (Delta2 = Delta1 / 2), eps = 0.5, T_I = 1, T_m = 0.5,
# T_s = 0.25 (|dom x| = 6: T_m |dom x| = 3, T_s cdfx |dom x| = 1.5 cdfx),
# mhat = 4 u v w, heavy cost mhat + 0.5 (u v + u w), w = u:
#   D=(64,32): 1365 + 630 + 3 + 94.5 = 2092.5, u = 0               -> 2092.5
#   D=(32,16): 1365 + 310 + 3 + 94.5 = 1772.5, u = 1 but v = 0       -> 1772.5
#   D=(16,8):  341 + 150 + 3 + 46.5 = 540.5; u=2 v=1 w=2: 16 + 3 = 19 -> 559.5
#   D=(8,4):   85 + 70 + 3 + 22.5 = 180.5;   u=3 v=2 w=3: 72 + 7.5   -> 260
#   D=(4,2):   21 + 30 + 3 + 10.5 = 64.5;    u=4 v=3 w=4: 192 + 14   -> 270.5 > 260: stop at (8, 4)
_RUN_B = [(64.0, 32.0, 2092.5), (32.0, 16.0, 1772.5), (16.0, 8.0, 559.5), (8.0, 4.0, 260.0),
          (4.0, 2.0, 270.5)]
# Run C: run A's constants with z degrees 1, 1, 64, 64, 64, 64 (R != S: w = 4
# heavy z at every threshold below 64, u stays as in run A):
#   D1=16: 651 + 20 * 1 * 1 * 4 = 731;  D1=8: 235 + 20 * 2 * 2 * 4 = 555;
#   D1=4:  91 + 20 * 3 * 3 * 4 = 811 > 555: stop at (8, 8)
_RUN_C = [(64.0, 64.0, 1995.0), (32.0, 32.0, 1995.0), (16.0, 16.0, 731.0), (8.0, 8.0, 555.0),
          (4.0, 4.0, 811.0)]
_DEGZ_C = [1, 1, 64, 64, 64, 64]


def _run(idx, which, eps=0.5, T_I=1.0):
    tr = []
    if which == "A" or which == "C":
        res = CM.algorithm3(idx, 64, 64.0, T_I, 0.0, 0.0, lambda u, v, w: 20.0 * u * v * w,
                            eps=eps, out_join=10_000, trace=tr)
    else:
        res = CM.algorithm3(idx, 64, 128.0, T_I, 0.25, 0.5, lambda u, v, w: 4.0 * u * v * w,
                            eps=eps, out_join=10_000, trace=tr)
    return res, tr


def test_algorithm3_hand_worked_runs():
    res, tr = _run(_hand_index(), "A")
    assert res == (8, 8, "mm") and tr == _RUN_A
    res, tr = _run(_hand_index(), "B")
    assert res == (8, 4, "mm") and tr == _RUN_B
    res, tr = _run(_hand_index(_DEGZ_C), "C")
    assert res == (8, 8, "mm") and tr == _RUN_C
    # the switch to the plain join: OUT_join <= 20 N
    assert CM.algorithm3(_hand_index(), 64, 64.0, 1.0, 0, 0, lambda u, v, w: 0.0,
                         out_join=20 * 64) == (64, 64, "wcoj")


class _NoSumX(CM.DegreeIndex):
    def sum_x(self, delta):
        return 0.0


class _WIsU(CM.DegreeIndex):
    def heavy_z(self, delta):
        return self.heavy_x(delta)


class _DegSquared(CM.DegreeIndex):
    """y weighed by max degree squared instead of deg_R * deg_S."""

    def __init__(self, degx, cand, r, s, degz=None):
        super().__init__(degx, cand, r, s, degz)
        d = np.maximum(np.asarray(r, np.int64), np.asarray(s, np.int64))
        self.sy2 = np.concatenate([[0.0], np.cumsum(np.sort(d).astype(np.float64) ** 2)])


def test_algorithm3_pins_catch_planted_mistakes():
    """Plausible mistakes, planted in CPU copies of the oracle, each fail a pin."""
    # a wrong step (eps 0.45 instead of 0.5)
    assert _run(_hand_index(), "A", eps=0.45)[1] != _RUN_A
    # a perturbed T_I
    assert _run(_hand_index(), "A", T_I=1.01)[1] != _RUN_A
    # the x term of the light cost dropped
    idx = _NoSumX(_DEG, [10 * d for d in _DEG], _DEG, _DEG)
    assert _run(idx, "A")[1] != _RUN_A and _run(idx, "B")[1] != _RUN_B
    # w taken as u (the self-join shortcut) on R != S
    idx = _WIsU(_DEG, [10 * d for d in _DEG], _DEG, _DEG, _DEGZ_C)
    assert _run(idx, "C")[1] != _RUN_C
    # y weighed by its squared degree when deg_R != deg_S
    r = [1, 2, 4, 8, 16, 32]
    s = [1, 1, 2, 2, 32, 32]
    good = _run(CM.DegreeIndex(_DEG, [10 * d for d in _DEG], r, s), "A")[1]
    bad = _run(_DegSquared(_DEG, [10 * d for d in _DEG], r, s), "A")[1]
    assert good != bad


def test_closed_form_roots_to_rounding():
    # OUT <= N: D1^3 = OUT and D2 * D1^2 = N, to the rounding of a cube root
    for N, OUT in ((1e8, 1e6), (1e8, 12345.0), (5e6, 5e6)):
        d1, d2 = CM.closed_form(N, OUT)
        assert abs(d1 ** 3 - OUT) <= 4e-16 * 3 * OUT
        assert abs(d2 * d1 * d1 - N) <= 1e-15 * 4 * N
    # OUT > N: D^3 (N + OUT) = 2 N^2
    for N, OUT in ((19683.0, 19683.0 * 2 - 19683.0 + 1.0), (1e7, 3.9e9)):
        d, d_ = CM.closed_form(N, OUT)
        assert d == d_
        assert abs(d ** 3 * (N + OUT) - 2 * N * N) <= 1e-15 * 4 * 2 * N * N
