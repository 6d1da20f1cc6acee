"""Threshold formulas of the paper, in fp64 -- TEST INFRASTRUCTURE ONLY.

* ``f_two_path``: the omega = 2, N_R = N_S = N cost of Section 3.1,
  f(D1, D2) = N + N*D1 + OUT*D2 + N^2 / (D2 * min(D1, D2)).
* ``closed_form``: its minimiser (Section 3.1, the two cases before Lemma 3):
  OUT <= N gives D1 = OUT^(1/3), D2 = N / OUT^(2/3); OUT > N gives
  D1 = D2 = (2 N^2 / (N + OUT))^(1/3).
* ``lemma3_time``: the resulting running time of Lemma 3.
* ``star_cost``: the Section 3.2 star cost
  N*D1^(k-1) + OUT*D2 + M((N/D2)^ceil(k/2), N/D1, (N/D2)^floor(k/2)) with
  M(U,V,W) = UVW * beta^(omega-3) (Lemma 1).
* ``out_estimate``: the Section 5 estimate of |OUT|, the geometric mean of
  max(|dom x|, (OUT_join / N)^2) and min(|dom x|^2, OUT_join).
* ``algorithm3``: the cost-based optimizer (Algorithm 3) on degree indexes.

Integer thresholds: D >= 1 (Section 3.1); real values are floored and clamped
to [1, N].
"""
from __future__ import annotations

import math

import numpy as np


def f_two_path(N: float, OUT: float, d1: float, d2: float) -> float:
    return N + N * d1 + OUT * d2 + N * N / (d2 * min(d1, d2))


def closed_form(N: float, OUT: float):
    """Real-valued minimiser (D1, D2) of ``f_two_path``."""
    if OUT <= N:
        return OUT ** (1.0 / 3.0), N / OUT ** (2.0 / 3.0)
    d = (2.0 * N * N / (N + OUT)) ** (1.0 / 3.0)
    return d, d


def to_int_threshold(d: float, N: int) -> int:
    return int(min(max(math.floor(d), 1), max(N, 1)))


def lemma3_time(N: float, OUT: float) -> float:
    return N + N ** (2.0 / 3.0) * OUT ** (1.0 / 3.0) * max(N, OUT) ** (1.0 / 3.0)


def mm_cost(U: float, V: float, W: float, omega: float = 2.0) -> float:
    beta = min(U, V, W)
    return U * V * W * beta ** (omega - 3.0)


def star_cost_terms(N: float, OUT: float, d1: float, d2: float, k: int, omega: float = 2.0):
    kv, kw = (k + 1) // 2, k // 2
    return (N * d1 ** (k - 1), OUT * d2,
            mm_cost((N / d2) ** kv, N / d1, (N / d2) ** kw, omega))


def star_cost(N, OUT, d1, d2, k, omega=2.0):
    return sum(star_cost_terms(N, OUT, d1, d2, k, omega))


def out_estimate(dom_x: float, out_join: float, N: float) -> float:
    lo = max(dom_x, (out_join / N) ** 2)
    hi = min(dom_x * dom_x, out_join)
    return math.sqrt(lo * hi)


class DegreeIndex:
    """Sorted-degree indexes of Section 5 for a self-join relation.

    ``degx[a]`` = |R[a]|, ``degy[b]`` = |R[b]| (y side), ``cand[a]`` =
    sum_{b in R[a]} |R[b]| (the deduplication effort of x = a).  Queries
    answer, for a threshold delta:
      sum_y(delta)   = sum over y with deg <= delta of deg^2
      sum_x(delta)   = sum over x with deg <= delta of cand
      cdfx(delta)    = sum over y with deg <= delta of deg
      count_x(delta) = number of x with deg > delta (heavy x), same for y.
    """

    def __init__(self, degx, degy, cand):
        ox = np.argsort(degx, kind="stable")
        self.dx = np.asarray(degx, np.int64)[ox]
        self.cx = np.concatenate([[0.0], np.cumsum(np.asarray(cand, np.float64)[ox])])
        oy = np.argsort(degy, kind="stable")
        self.dy = np.asarray(degy, np.int64)[oy]
        dyf = self.dy.astype(np.float64)
        self.sy2 = np.concatenate([[0.0], np.cumsum(dyf * dyf)])
        self.sy1 = np.concatenate([[0.0], np.cumsum(dyf)])

    def _nle(self, arr, delta):
        return int(np.searchsorted(arr, math.floor(delta), side="right"))

    def sum_y(self, delta):
        return float(self.sy2[self._nle(self.dy, delta)])

    def sum_x(self, delta):
        return float(self.cx[self._nle(self.dx, delta)])

    def cdfx(self, delta):
        return float(self.sy1[self._nle(self.dy, delta)])

    def heavy_x(self, delta):
        return len(self.dx) - self._nle(self.dx, delta)

    def heavy_y(self, delta):
        return len(self.dy) - self._nle(self.dy, delta)


def algorithm3(idx: DegreeIndex, N: int, OUT: float, T_I: float, T_s: float, T_m: float,
               mhat, eps: float = 0.05, wcoj_factor: float = 20.0, out_join=None):
    """Algorithm 3: geometric descent on Delta1 with Delta2 = N * Delta1 / OUT.

    Readings (Section 5, Algorithm 3 is garbled in places):
    * the step is Delta1 <- (1 - eps) * Delta1 with eps = 0.05 (the footnote's
      0.95 is read as the multiplier);
    * the light cost is T_I * sum(y_D1) + T_I * sum(x_D2) + T_m * |dom x|
      + T_s * cdfx(y_D1) * |dom x| (as printed; the stray ``+ .`` before the
      second T_I is dropped);
    * the first cost is the all-light one at Delta1 = N (the printed start
      value of t_light is a join size, not a time);
    * the heavy cost is mhat(u, v, w) + T_m * (u*v + u*w), with u, w the
      heavy x (= z, self-join) counts and v the heavy y count;
    * the loop stops at the first step whose total cost is larger than the
      previous one (the Section 5 text says "larger"; the algorithm box's
      ``<=`` would stop on the all-light plateau right after Delta1 = N,
      before any degree falls above the thresholds) and returns the previous
      thresholds.
    Returns (delta1, delta2, mode) with mode "wcoj" when the full join is at
    most wcoj_factor * N (all light).
    """
    if out_join is not None and out_join <= wcoj_factor * N:
        return N, N, "wcoj"
    dom_x = len(idx.dx)
    d1 = float(N)
    d2 = max(N * d1 / OUT, 1.0)
    prev_cost = math.inf
    prev = (d1, d2)
    while True:
        light = (T_I * idx.sum_y(d1) + T_I * idx.sum_x(d2) + T_m * dom_x
                 + T_s * idx.cdfx(d1) * dom_x)
        u = idx.heavy_x(d2)
        v = idx.heavy_y(d1)
        heavy = (mhat(u, v, u) + T_m * (u * v + u * u)) if (u and v) else 0.0
        cost = light + heavy
        if cost > prev_cost:
            return to_int_threshold(prev[0], N), to_int_threshold(prev[1], N), "mm"
        prev_cost, prev = cost, (d1, d2)
        if d1 <= 1.0:
            return to_int_threshold(d1, N), to_int_threshold(d2, N), "mm"
        d1 = max(d1 * (1.0 - eps), 1.0)
        d2 = max(N * d1 / OUT, 1.0)


def star_grid_thresholds(N: int, OUT: float, k: int = 3, steps: int = 96):
    """Integer (Delta1, Delta2) minimising the Section 3.2 star cost (omega = 2)
    over a log-spaced grid of [1, N] with ``steps`` intervals per axis: the
    Section 3.2 cost has no closed form for general k and OUT."""
    lnN = math.log(max(N, 1))
    grid = [max(1, math.floor(math.exp(lnN * i / steps))) for i in range(steps + 1)]
    best, arg = math.inf, (1, 1)
    for t1 in grid:
        for t2 in grid:
            c = star_cost(float(N), float(OUT), float(t1), float(t2), k)
            if c < best:
                best, arg = c, (t1, t2)
    return arg
