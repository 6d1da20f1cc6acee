"""Seeded synthetic relations for the join-project path.

This module only draws inputs. It holds none of the method's arithmetic (no
join, projection, degree threshold or deduplication), so both the CPU oracle
and the CUDA path may use it.

The paper evaluates on real bipartite datasets (Section 7.1, Table 1) that are
not available here. These generators stand in for them:

* ``uniform_relation``: pairs drawn uniformly from a box, kept until ``n``
  distinct pairs exist (the small two-path workload, N = 20,000).
* ``powerlaw_relation``: a bipartite relation whose x and y degree
  distributions follow a discrete power law ``P(d) ~ d^-gamma`` on
  ``[1, d_max]``, with ``d_max`` chosen so that the mean degree equals
  ``n / |dom|``.  Target degrees are drawn per value, then tuples are drawn by
  Chung-Lu endpoint sampling (x with probability ~ its target degree, y
  likewise), deduplicated and topped up until exactly ``n`` distinct tuples
  exist (the 10M-tuple two-path workload).
* ``star_relations``: k relations over one shared y domain that reuse the same
  power-law y target-degree sequence on the same y ids, with x uniform over
  its own domain (the k = 3 star workload, 3 x 2M tuples).

Every function is deterministic in its seed (numpy ``default_rng``).  Tuples
are returned as two int32 numpy arrays in draw order of first appearance.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "uniform_relation",
    "powerlaw_relation",
    "star_relations",
    "powerlaw_pmf",
    "solve_dmax",
    "random_small_relation",
    "WORKLOADS",
]


def _first_distinct(keys: np.ndarray, n: int) -> np.ndarray:
    """First ``n`` distinct int64 keys of ``keys`` in order of first appearance."""
    _, first = np.unique(keys, return_index=True)
    first.sort()
    return keys[first[:n]]


def _split(keys: np.ndarray):
    x = (keys >> 32).astype(np.int64) - (1 << 31)
    y = (keys & 0xFFFFFFFF).astype(np.int64) - (1 << 31)
    return x.astype(np.int32), y.astype(np.int32)


def _pack(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    return ((x.astype(np.int64) + (1 << 31)) << 32) | (y.astype(np.int64) + (1 << 31))


def _draw_until(n: int, draw, rng, max_rounds: int = 64):
    """Call ``draw(rng, m)`` (returns packed keys) until ``n`` distinct exist."""
    keys = np.empty(0, dtype=np.int64)
    have = 0
    m = n
    for _ in range(max_rounds):
        keys = np.concatenate([keys, draw(rng, m)])
        keys = _first_distinct(keys, len(keys))
        have = len(keys)
        if have >= n:
            return keys[:n]
        # draw a little more than the deficit; duplicates are expected
        m = int((n - have) * 1.5) + 64
    raise RuntimeError(f"could not draw {n} distinct tuples (have {have})")


def uniform_relation(n: int, dom_x: int, dom_y: int, seed: int = 0):
    """``n`` distinct pairs drawn uniformly from ``[0,dom_x) x [0,dom_y)``."""
    if n > dom_x * dom_y:
        raise ValueError("n exceeds the number of distinct pairs")
    rng = np.random.default_rng(seed)

    def draw(rng, m):
        x = rng.integers(0, dom_x, size=m, dtype=np.int64)
        y = rng.integers(0, dom_y, size=m, dtype=np.int64)
        return _pack(x, y)

    return _split(_draw_until(n, draw, rng))


def powerlaw_pmf(gamma: float, d_max: int) -> np.ndarray:
    """Probabilities of degrees 1..d_max under ``P(d) ~ d^-gamma``."""
    d = np.arange(1, d_max + 1, dtype=np.float64)
    w = d ** (-gamma)
    return w / w.sum()


def _pl_mean(gamma: float, d_max: int) -> float:
    d = np.arange(1, d_max + 1, dtype=np.float64)
    w = d ** (-gamma)
    return float((w * d).sum() / w.sum())


def solve_dmax(gamma: float, mean: float, limit: int = 1 << 26) -> int:
    """Smallest ``d_max`` whose truncated power law has mean >= ``mean``.

    The mean of the truncated law grows with ``d_max``; if even ``limit``
    cannot reach ``mean`` (possible for gamma > 2), ``limit`` is returned.
    """
    if mean <= 1.0:
        return 1
    lo, hi = 1, 2
    while _pl_mean(gamma, hi) < mean:
        if hi >= limit:
            return limit
        lo, hi = hi, min(hi * 2, limit)
    while lo + 1 < hi:
        mid = (lo + hi) // 2
        if _pl_mean(gamma, mid) >= mean:
            hi = mid
        else:
            lo = mid
    return hi


def _target_degrees(rng, dom: int, gamma: float, mean: float) -> np.ndarray:
    d_max = solve_dmax(gamma, mean)
    pmf = powerlaw_pmf(gamma, d_max)
    cdf = np.cumsum(pmf)
    cdf[-1] = 1.0
    u = rng.random(dom)
    return (np.searchsorted(cdf, u, side="right") + 1).astype(np.float64)


def _alias_sampler(weights: np.ndarray):
    cdf = np.cumsum(weights, dtype=np.float64)
    cdf /= cdf[-1]
    cdf[-1] = 1.0

    def sample(rng, m):
        return np.searchsorted(cdf, rng.random(m), side="right").astype(np.int64)

    return sample


def powerlaw_relation(n: int, dom_x: int, gamma_x: float, dom_y: int, gamma_y: float,
                      seed: int = 0):
    """Power-law bipartite relation with exactly ``n`` distinct tuples.

    x values lie in ``[0, dom_x)``, y values in ``[0, dom_y)``.  Values whose
    drawn endpoint weight never gets sampled simply do not appear.
    """
    if n <= 0:
        return np.empty(0, np.int32), np.empty(0, np.int32)
    rng = np.random.default_rng(seed)
    dx = _target_degrees(rng, dom_x, gamma_x, n / dom_x)
    dy = _target_degrees(rng, dom_y, gamma_y, n / dom_y)
    sx = _alias_sampler(dx)
    sy = _alias_sampler(dy)

    def draw(rng, m):
        return _pack(sx(rng, m), sy(rng, m))

    return _split(_draw_until(n, draw, rng))


def star_relations(k: int, n: int, dom_x: int, dom_y: int, gamma_y: float,
                   seed: int = 0):
    """``k`` relations ``R_i(x_i, y)`` sharing one power-law y degree sequence.

    The y target degrees are drawn once (from ``seed``) and reused on the same
    y ids by every relation; relation ``i`` draws its tuples with seed
    ``seed + i``, x uniform over ``[0, dom_x)``.
    """
    rng0 = np.random.default_rng(seed)
    dy = _target_degrees(rng0, dom_y, gamma_y, n / dom_y)
    sy = _alias_sampler(dy)
    rels = []
    for i in range(k):
        rng = np.random.default_rng(seed + i)

        def draw(rng, m):
            x = rng.integers(0, dom_x, size=m, dtype=np.int64)
            return _pack(x, sy(rng, m))

        rels.append(_split(_draw_until(n, draw, rng)))
    return rels


def random_small_relation(rng, n: int, dom_x: int, dom_y: int, offset_x: int = 0,
                          offset_y: int = 0, skew: float = 0.0):
    """Small random relation (possibly with duplicate tuples) for tests.

    ``skew > 0`` draws values from a Zipf-like rank law so that a few values
    get large degrees.  Values are shifted by the offsets (negative allowed).
    Duplicates are kept on purpose: relations are sets and the path must
    remove them.
    """
    if skew > 0:
        wx = np.arange(1, dom_x + 1, dtype=np.float64) ** (-skew)
        wy = np.arange(1, dom_y + 1, dtype=np.float64) ** (-skew)
        x = rng.choice(dom_x, size=n, p=wx / wx.sum())
        y = rng.choice(dom_y, size=n, p=wy / wy.sum())
    else:
        x = rng.integers(0, dom_x, size=n)
        y = rng.integers(0, dom_y, size=n)
    return ((x + offset_x).astype(np.int32), (y + offset_y).astype(np.int32))


def candidate_pairs(x_vals: np.ndarray, z_vals: np.ndarray, count: int, seed: int = 0,
                    absent: float = 0.0, x_weights=None, z_weights=None):
    """Candidate pairs (a, b) for a batch of boolean set intersection requests.

    ``a`` is drawn from ``x_vals`` and ``b`` from ``z_vals`` (with
    replacement, so pairs repeat), uniformly or with probability proportional
    to the given weights (e.g. the values' degrees: large sets are asked about
    more often); a fraction ``absent`` of the pairs names, on one side, a value
    outside the given ones.
    """
    rng = np.random.default_rng(seed)
    x_vals = np.asarray(x_vals)
    z_vals = np.asarray(z_vals)
    if count <= 0 or len(x_vals) == 0 or len(z_vals) == 0:
        return np.empty(0, np.int32), np.empty(0, np.int32)

    def draw(vals, w):
        if w is None:
            return vals[rng.integers(0, len(vals), count)].astype(np.int64)
        cdf = np.cumsum(np.asarray(w, np.float64))
        i = np.searchsorted(cdf, rng.random(count) * cdf[-1], side="right")
        return vals[np.minimum(i, len(vals) - 1)].astype(np.int64)

    a = draw(x_vals, x_weights)
    b = draw(z_vals, z_weights)
    miss = rng.random(count) < absent
    side = rng.random(count) < 0.5
    a[miss & side] = int(x_vals.max()) + 1 + rng.integers(0, 1000, int((miss & side).sum()))
    b[miss & ~side] = int(z_vals.max()) + 1 + rng.integers(0, 1000, int((miss & ~side).sum()))
    return (np.clip(a, -(1 << 31), (1 << 31) - 1).astype(np.int32),
            np.clip(b, -(1 << 31), (1 << 31) - 1).astype(np.int32))


# Named workloads with the paper-shaped sizes (Section 7.1 stand-ins).
WORKLOADS = {
    # two-path, uniform, N = 20,000, fixed thresholds floor(sqrt(N)) = 141
    "two_path_uniform_20k": dict(kind="two_path", gen="uniform", n=20_000,
                                 dom_x=2000, dom_y=500, seed=0),
    # two-path, power law, N = 10M, x: 2M values gamma 2.1, y: 1M values gamma 1.8
    "two_path_powerlaw_10m": dict(kind="two_path", gen="powerlaw", n=10_000_000,
                                  dom_x=2_000_000, gamma_x=2.1,
                                  dom_y=1_000_000, gamma_y=1.8, seed=0),
    # the same shape at 1/10 of the size (profiling captures, quick checks)
    "two_path_powerlaw_1m": dict(kind="two_path", gen="powerlaw", n=1_000_000,
                                 dom_x=200_000, gamma_x=2.1,
                                 dom_y=100_000, gamma_y=1.8, seed=0),
    # set similarity join on the 10M relation: pairs sharing >= 2 y, by decreasing count
    "ssj_powerlaw_10m": dict(kind="ssj", gen="powerlaw", n=10_000_000,
                             dom_x=2_000_000, gamma_x=2.1,
                             dom_y=1_000_000, gamma_y=1.8, seed=0, c_min=2),
    # the set similarity join on the 1M relation (profiling captures)
    "ssj_powerlaw_1m": dict(kind="ssj", gen="powerlaw", n=1_000_000,
                            dom_x=200_000, gamma_x=2.1,
                            dom_y=100_000, gamma_y=1.8, seed=0, c_min=2),
    # star k = 3, 3 x 2M tuples, shared y domain 200k gamma 1.5, x uniform 500k
    "star3_2m": dict(kind="star", gen="star", k=3, n=2_000_000, dom_x=500_000,
                     dom_y=200_000, gamma_y=1.5, seed=0),
    # a smaller star query for profiling captures: 3 x 1M tuples, y domain 250k (mean y
    # degree 4 instead of 10, so that the output, ~1.7e8 triples, stays a few GB)
    "star3_1m": dict(kind="star", gen="star", k=3, n=1_000_000, dom_x=250_000,
                     dom_y=250_000, gamma_y=1.5, seed=0),
}


def make(name: str, **override):
    """Draw a named workload; returns ``(x, y)`` or a list of them (star)."""
    w = dict(WORKLOADS[name])
    w.update(override)
    gen = w.pop("gen")
    w.pop("kind")
    if gen == "uniform":
        return uniform_relation(w["n"], w["dom_x"], w["dom_y"], w["seed"])
    if gen == "powerlaw":
        return powerlaw_relation(w["n"], w["dom_x"], w["gamma_x"], w["dom_y"],
                                 w["gamma_y"], w["seed"])
    if gen == "star":
        return star_relations(w["k"], w["n"], w["dom_x"], w["dom_y"], w["gamma_y"],
                              w["seed"])
    raise KeyError(gen)
