"""Refit the constants of the cost model (Section 5, Table 2's roles) on measured query times.

The cost model prices a threshold pair (Delta1, Delta2) of a relation as

  T_I * (light-y candidates + light-x candidates)        insertions into dedup structures
  + T_m * |dom x| + T_s * cdfx(Delta1) * |dom x|         per-x set-up and scan steps
  + [u, v, w > 0] * (2 u v w / mm_rate + mm_fixed + T_m (u v + u w))   the heavy block

with u, w the heavy x and z and v the heavy y.  The library's default constants
were measured on one relation.  Here they are fitted to the whole-query times
that learn.py records for a grid of fixed thresholds on each of many seeded
power-law relations (the same self-join query): the model is linear in
(T_I, T_s, 1/mm_rate, mm_fixed, T_m), so the fit is a non-negative least
squares with a free intercept per relation (costs that do not depend on the
thresholds: index build, output placement), each relation's times divided by
its fastest, so that large and small relations weigh the same.  Only grid
points within `cap` (default 3) times the relation's fastest enter the fit:
thresholds are chosen near the optimum, and far-off points (a product of
seconds, a light path ten times too slow) would otherwise set the constants.

  python -m paper_2002_12459_gb300.calibrate --data learn_data.npz --out cost_model.json

The relations are regenerated from their seeds (workloads.powerlaw_relation); no
GPU is needed.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(PKG, "predictor", "cost_model.json")

# the fitted constants, in the order of the feature columns
FIT_NAMES = ("T_I", "T_s", "inv_mm_rate", "mm_fixed", "T_m")


def degree_terms(x: np.ndarray, y: np.ndarray):
    """Degrees of a self-join relation's distinct tuples: (deg_x per x, deg_y per y,
    cand per x = sum over x's y of deg_y, N = distinct tuples)."""
    key = np.unique((x.astype(np.int64) << 32) | (y.astype(np.int64) & 0xFFFFFFFF))
    xs, ys = key >> 32, key & 0xFFFFFFFF
    _, xi = np.unique(xs, return_inverse=True)
    _, yi = np.unique(ys, return_inverse=True)
    degx = np.bincount(xi).astype(np.float64)
    degy = np.bincount(yi).astype(np.float64)
    cand = np.bincount(xi, weights=degy[yi])
    return degx, degy, cand, len(key)


def features(degx, degy, cand, d1: float, d2: float):
    """Feature row of the self-join at thresholds (d1, d2): a value is heavy when its degree
    exceeds the threshold (y against d1, x and z against d2).  Columns follow FIT_NAMES;
    the T_m * |dom x| term is the same at every threshold of a relation and is left to
    its intercept."""
    ly = degy <= d1
    lx = degx <= d2
    light = float((degy[ly] ** 2).sum() + cand[lx].sum())
    scan = float(degy[ly].sum()) * len(degx)
    u = float((~lx).sum())
    v = float((~ly).sum())
    w = u
    on = u > 0 and v > 0 and w > 0
    return [light, scan, 2.0 * u * v * w if on else 0.0, 1.0 if on else 0.0,
            (u * v + u * w) if on else 0.0]


def relation_rows(r, cap: float = math.inf):
    """Feature rows and relative times of one relation's grid points within cap times
    its fastest."""
    from paper_2002_12459_gb300 import learn
    x, y = learn.make_relation(r["spec"])
    degx, degy, cand, _ = degree_terms(x, y)
    grid = np.asarray(r["grid"], np.float64)
    best = np.min(grid)
    F, t = [], []
    for i, d1 in enumerate(r["d1_grid"]):
        for j, d2 in enumerate(r["d2_grid"]):
            if math.isfinite(grid[i, j]) and grid[i, j] <= cap * best:
                F.append(np.array(features(degx, degy, cand, d1, d2)) / (best * 1e-3))
                t.append(grid[i, j] / best)
    return F, t


def design(rows, log=None, workers=None, cap: float = math.inf):
    """(F, t, group) over every finite grid point of every relation: features, time
    divided by the relation's fastest, and the relation's index.  A row holds the
    relation's spec, its time grid (ms) and the grid's thresholds.  The relations are
    regenerated by a pool of spawned processes."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    F, t, grp = [], [], []
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as pool:
        for k, (f, tt) in enumerate(pool.map(relation_rows, rows, [cap] * len(rows))):
            F += f
            t += tt
            grp += [k] * len(tt)
            if log and k % 100 == 0:
                log(f"[calibrate] {k + 1}/{len(rows)} relations")
    return np.array(F), np.array(t), np.array(grp)


def fit(F, t, grp):
    """Non-negative least squares of t on F with a free intercept per group: the
    intercepts are eliminated by centring each group.  Returns (constants, rms of the
    residual, rms of the centred times)."""
    from scipy.optimize import nnls
    Fc, tc = F.astype(np.float64).copy(), t.astype(np.float64).copy()
    for g in np.unique(grp):
        m = grp == g
        Fc[m] -= Fc[m].mean(axis=0)
        tc[m] -= tc[m].mean()
    scale = np.maximum(np.abs(Fc).max(axis=0), 1e-300)    # column scaling for conditioning
    k, _ = nnls(Fc / scale, tc)
    k = k / scale
    res = tc - Fc @ k
    return k, float(np.sqrt(np.mean(res * res))), float(np.sqrt(np.mean(tc * tc)))


DEFAULT_BASE = dict(T_I=1.0 / 60e9, T_m=1.0 / 1.0e12, T_s=0.0, mm_rate=2.2e15, mm_fixed=20e-6,
                    eps=0.05, wcoj_factor=20.0, judge=3.0)


def constants(k, base: dict) -> dict:
    """The library's jp_cost_model fields from the fitted vector (unfitted fields from base)."""
    out = dict(base)
    out["T_I"], out["T_s"], inv_rate, out["mm_fixed"], out["T_m"] = (float(v) for v in k)
    out["mm_rate"] = 1.0 / inv_rate if inv_rate > 0 else base["mm_rate"]
    return out


def load_rows(path: str, part: str = "train"):
    """The relations' records (spec and time grid) of a learn.py --data file."""
    d = np.load(path, allow_pickle=False)
    d1, d2 = [int(v) for v in d["d1_grid"]], [int(v) for v in d["d2_grid"]]
    rows = []
    for s in d[part]:
        r = json.loads(str(s))
        r["d1_grid"], r["d2_grid"] = d1, d2
        rows.append(r)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", required=True, help="learn.py --data output (.npz)")
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--limit", type=int, default=0, help="use the first N relations only")
    ap.add_argument("--cap", type=float, default=3.0,
                    help="fit grid points within this factor of each relation's fastest")
    args = ap.parse_args(argv)

    def log(*a):
        print(*a, file=sys.stderr, flush=True)

    rows = load_rows(args.data)
    if args.limit:
        rows = rows[:args.limit]
    F, t, grp = design(rows, log, cap=args.cap)
    k, rms, rms0 = fit(F, t, grp)
    consts = constants(k, DEFAULT_BASE)
    res = dict(constants=consts, fit=dict(relations=len(rows), points=int(len(t)), cap=args.cap,
                                          rms_relative=rms, rms_relative_unfitted=rms0,
                                          vector=dict(zip(FIT_NAMES, map(float, k)))))
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
