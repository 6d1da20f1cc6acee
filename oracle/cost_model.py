"""Threshold formulas of the paper, in fp64 -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` may use this
module; the product library shares no code with it.

* ``f_two_path``: the omega = 2, N_R = N_S = N cost of Section 3.1,
  f(D1, D2) = N + N*D1 + OUT*D2 + N^2 / (D2 * min(D1, D2)).
* ``closed_form``: its minimiser (Section 3.1, the two cases before Lemma 3):
  OUT <= N gives D1 = OUT^(1/3), D2 = N / OUT^(2/3); OUT > N gives
  D1 = D2 = (2 N^2 / (N + OUT))^(1/3).  Cube roots are taken with
  ``math.cbrt`` and OUT^(2/3) as the square of the cube root.
* ``lemma3_time``: the resulting running time of Lemma 3.
* ``star_cost``: the Section 3.2 star cost
  N*D1^(k-1) + OUT*D2 + M((N/D2)^ceil(k/2), N/D1, (N/D2)^floor(k/2)) with
  M(U,V,W) = UVW * beta^(omega-3) (Lemma 1).
* ``out_estimate``: the Section 5 estimate of |OUT|, the geometric mean of
  max(|dom x|, (OUT_join / N)^2) and min(|dom x|^2, OUT_join).
* ``DegreeIndex`` / ``index_of_relations``: the Section 5 degree indexes of
  R and S (R != S allowed; the y degree is max(deg_R, deg_S), the partition
  rule that reproduces the Section 3.1 worked example).
* ``algorithm3``: the cost-based optimizer (Algorithm 3) on degree indexes.

Integer thresholds: D >= 1 (Section 3.1); real values are floored and clamped
to [1, N].  For R != S, N is max(|R|, |S|) after R's dangling tuples (y not in
S) are removed (Section 3.1 assumes |R| = |S| = N).
"""
from __future__ import annotations

import math

import numpy as np


def f_two_path(N: float, OUT: float, d1: float, d2: float) -> float:
    return N + N * d1 + OUT * d2 + N * N / (d2 * min(d1, d2))


def closed_form(N: float, OUT: float):
    """Real-valued minimiser (D1, D2) of ``f_two_path``."""
    if OUT <= N:
        c = math.cbrt(OUT)
        return c, N / (c * c)
    d = math.cbrt(2.0 * N * N / (N + OUT))
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
    """Sorted-degree indexes of Section 5 ("Indexing relations").

    Inputs, one entry per value:
      ``degx[a]`` = |R[a]| and ``cand[a]`` = sum_{b in R[a]} |S[b]| (the
      deduplication effort of x = a);
      ``degy_r[b]`` = |R[b]|, ``degy_s[b]`` = |S[b]| for every y of S;
      ``degz[c]`` = |S[c]| for every z of S (None: the self-join, z = x).
    A y value is light at delta iff max(deg_R(y), deg_S(y)) <= delta.
    Queries, for a threshold delta:
      sum_y(delta)   = sum over light y of deg_R(y) * deg_S(y)  (light join size)
      sum_x(delta)   = sum over x with deg <= delta of cand
      cdfx(delta)    = sum over light y of deg_R(y)
      heavy_x(delta) = number of x with deg > delta; heavy_y, heavy_z likewise.
    """

    def __init__(self, degx, cand, degy_r, degy_s=None, degz=None):
        degx = np.asarray(degx, np.int64)
        ox = np.argsort(degx, kind="stable")
        self.dx = degx[ox]
        self.cx = np.concatenate([[0.0], np.cumsum(np.asarray(cand, np.float64)[ox])])
        r = np.asarray(degy_r, np.int64)
        s = r if degy_s is None else np.asarray(degy_s, np.int64)
        dy = np.maximum(r, s)
        oy = np.argsort(dy, kind="stable")
        self.dy = dy[oy]
        self.sy2 = np.concatenate([[0.0], np.cumsum((r * s).astype(np.float64)[oy])])
        self.sy1 = np.concatenate([[0.0], np.cumsum(r.astype(np.float64)[oy])])
        self.dz = self.dx if degz is None else np.sort(np.asarray(degz, np.int64))

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

    def heavy_z(self, delta):
        return len(self.dz) - self._nle(self.dz, delta)


def index_of_relations(rx, ry, sz=None, sy=None):
    """Degree indexes and sizes of R and S (S = R when ``sz`` is None).

    R's tuples whose y has no S tuple are dropped first (dangling tuples,
    Section 3.1).  Returns ``(idx, info)`` with ``info`` holding ``N`` =
    max(|R|, |S|), ``n_r``, ``n_s``, ``dom_x``, ``dom_y``, ``dom_z`` and
    ``out_join`` = sum_y deg_R(y) deg_S(y) (an exact Python integer).
    """
    self_join = sz is None
    rx = np.asarray(rx, np.int64)
    ry = np.asarray(ry, np.int64)
    key = np.unique((rx << 32) | (ry & 0xFFFFFFFF))
    rx = key >> 32
    ry = (key & 0xFFFFFFFF).astype(np.uint32).astype(np.int32).astype(np.int64)
    if self_join:
        sz, sy = rx, ry
    else:
        sz = np.asarray(sz, np.int64)
        sy = np.asarray(sy, np.int64)
        k2 = np.unique((sz << 32) | (sy & 0xFFFFFFFF))
        sz = k2 >> 32
        sy = (k2 & 0xFFFFFFFF).astype(np.uint32).astype(np.int32).astype(np.int64)
        keep = np.isin(ry, sy)
        rx, ry = rx[keep], ry[keep]
    ys, degy_s = np.unique(sy, return_counts=True)
    degy_r = np.zeros(len(ys), np.int64)
    yr, cr = np.unique(ry, return_counts=True)
    degy_r[np.searchsorted(ys, yr)] = cr
    xs, xinv = np.unique(rx, return_inverse=True)
    degx = np.bincount(xinv, minlength=len(xs)).astype(np.int64)
    cand = np.bincount(xinv, weights=degy_s[np.searchsorted(ys, ry)].astype(np.float64),
                       minlength=len(xs))
    zs, degz = np.unique(sz, return_counts=True)
    idx = DegreeIndex(degx, cand, degy_r, degy_s, None if self_join else degz)
    out_join = sum(int(a) * int(b) for a, b in zip(degy_r.tolist(), degy_s.tolist()))
    info = dict(N=max(len(rx), len(sz)), n_r=len(rx), n_s=len(sz), dom_x=len(xs),
                dom_y=len(ys), dom_z=len(zs), out_join=out_join)
    return idx, info


def algorithm3(idx: DegreeIndex, N: int, OUT: float, T_I: float, T_s: float, T_m: float,
               mhat, eps: float = 0.05, wcoj_factor: float = 20.0, out_join=None, trace=None):
    """Algorithm 3: geometric descent on Delta1 with Delta2 = N * Delta1 / OUT.

    Readings (Section 5, Algorithm 3 is garbled in places):
    * the step is Delta1 <- (1 - eps) * Delta1 with eps = 0.05 (the footnote's
      0.95 is read as the multiplier);
    * the light cost is T_I * sum(y_D1) + T_I * sum(x_D2) + T_m * |dom x|
      + T_s * cdfx(y_D1) * |dom x| (as printed; the stray ``+ .`` before the
      second T_I is dropped);
    * the first cost is the all-light one at Delta1 = N (the printed start
      value of t_light is a join size, not a time);
    * the heavy cost is mhat(u, v, w) + T_m * (u*v + u*w), with u the heavy
      x, v the heavy y and w the heavy z counts, and 0 when one of them is 0
      (no product);
    * the loop stops at the first step whose total cost is larger than the
      previous one (the Section 5 text says "larger"; the algorithm box's
      ``<=`` would stop on the all-light plateau right after Delta1 = N,
      before any degree falls above the thresholds) and returns the previous
      thresholds.
    Returns (delta1, delta2, mode) with mode "wcoj" when the full join is at
    most wcoj_factor * N (all light).  ``trace``, a list, receives
    (delta1, delta2, cost) for every step evaluated.
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
        w = idx.heavy_z(d2)
        heavy = (mhat(u, v, w) + T_m * (u * v + u * w)) if (u and v and w) else 0.0
        cost = light + heavy
        if trace is not None:
            trace.append((d1, d2, cost))
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
