"""Algorithm 1 (Section 3.1) and the star algorithm (Section 3.2), step by step.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy, in the
paper's order and notation, with no blocking, fusion or reordering:

two-path, thresholds Delta1, Delta2 >= 1 (Algorithm 1):
  1. partition R into R^-, R^+ and S into S^-, S^+ by degree;
  2. T <- light joins, projected (any worst-case optimal join: here a dict
     join on y);
  3. M1 <- adjacency matrix of R^+ (heavy x by heavy y), M2 <- adjacency of
     S^+ (heavy y by heavy z);
  4. M <- M1 x M2 (numpy int64 product, exact counts);
  5. T <- T union {(a, c) : M_ac > 0}.

Readings taken where the paper is ambiguous:

* y heaviness.  The Section 3.1 text measures y in S for both relations,
  Algorithm 1 measures y in each relation's own degree; the worked example
  (Section 3.1, Delta1 = Delta2 = 2) keeps S tuples (4,4), (5,4) heavy
  although y = 4 has degree 2 in S.  The reading that reproduces the
  example: y is heavy iff max(deg_R(y), deg_S(y)) > Delta1, and M1 and M2
  share that column set.  Light is ``<=``, heavy is ``>``.
* Light joins.  ``(R^- join S) union (R join S^-)`` counts witnesses in
  ``R^- join S^-`` twice; the same set is reached by the disjoint split
  ``(R^- join S) union (R^+ join S^-)``, which is what is computed here.
* Star partition (Section 3.2).  A tuple (a_i, b) is in R_i^diamond iff b
  has degree <= Delta1 in every other relation.  A witness combination
  (a_1..a_k, b) is left for the matrix product iff every a_i is heavy and no
  (a_i, b) is in R_i^diamond, i.e. iff at least two relations give b degree
  > Delta1.  V has the ceil(k/2)-tuples of heavy values as rows, W the
  floor(k/2)-tuples, both with the heavy y values as columns.
"""
from __future__ import annotations

from collections import defaultdict

import numpy as np


def _deg(pairs, idx):
    d = defaultdict(int)
    for t in pairs:
        d[t[idx]] += 1
    return d


def partition_two_path(R, S, d1: int, d2: int):
    """Algorithm 1, first two lines: returns (Rm, Rp, Sm, Sp, heavy x/y/z)."""
    R = sorted(set(R))
    S = sorted(set(S))
    degRx = _deg(R, 0)
    degRy = _deg(R, 1)
    degSz = _deg(S, 0)
    degSy = _deg(S, 1)
    ys = set(degRy) | set(degSy)
    y_heavy = {b for b in ys if max(degRy.get(b, 0), degSy.get(b, 0)) > d1}
    Rm = [(a, b) for (a, b) in R if degRx[a] <= d2 or b not in y_heavy]
    Sm = [(c, b) for (c, b) in S if degSz[c] <= d2 or b not in y_heavy]
    Rm_set, Sm_set = set(Rm), set(Sm)
    Rp = [t for t in R if t not in Rm_set]
    Sp = [t for t in S if t not in Sm_set]
    hx = sorted(a for a in degRx if degRx[a] > d2)
    hz = sorted(c for c in degSz if degSz[c] > d2)
    hy = sorted(y_heavy)
    return Rm, Rp, Sm, Sp, hx, hy, hz


def _join_project(A, B):
    """pi_{x,z} A(x,y) join B(z,y) via a dict on y."""
    by_y = defaultdict(list)
    for c, b in B:
        by_y[b].append(c)
    return {(a, c) for a, b in A for c in by_y.get(b, ())}


def algorithm1(R, S, d1: int, d2: int):
    """Run Algorithm 1; returns a dict with T (sorted list) and the matrices."""
    Rm, Rp, Sm, Sp, hx, hy, hz = partition_two_path(R, S, d1, d2)
    T = _join_project(Rm, S) | _join_project(Rp, Sm)
    ix = {a: i for i, a in enumerate(hx)}
    iy = {b: j for j, b in enumerate(hy)}
    iz = {c: l for l, c in enumerate(hz)}
    M1 = np.zeros((len(hx), len(hy)), np.int64)
    M2 = np.zeros((len(hy), len(hz)), np.int64)
    for a, b in Rp:
        M1[ix[a], iy[b]] = 1
    for c, b in Sp:
        M2[iy[b], iz[c]] = 1
    M = M1 @ M2
    heavy = {(hx[i], hz[l]) for i, l in zip(*np.nonzero(M))}
    T = T | heavy
    return dict(T=sorted(T), M1=M1, M2=M2, M=M, hx=hx, hy=hy, hz=hz,
                Rm=sorted(Rm), Sm=sorted(Sm), light=len(T - heavy))


def light_join_size(R, S, d1: int, d2: int) -> int:
    """Number of (a, b, c) witnesses the light part enumerates (before projection)."""
    Rm, Rp, Sm, Sp, *_ = partition_two_path(R, S, d1, d2)
    cnt_S = defaultdict(int)
    cnt_Sm = defaultdict(int)
    for c, b in S:
        cnt_S[b] += 1
    for c, b in Sm:
        cnt_Sm[b] += 1
    return sum(cnt_S[b] for _, b in Rm) + sum(cnt_Sm[b] for _, b in Rp)


def star_partition(rels, d1: int, d2: int):
    """Heavy x sets per relation and heavy y set for the star (Section 3.2)."""
    rels = [sorted(set(r)) for r in rels]
    degx = [_deg(r, 0) for r in rels]
    degy = [_deg(r, 1) for r in rels]
    ys = set().union(*[set(d) for d in degy])
    hy = sorted(b for b in ys if sum(1 for d in degy if d.get(b, 0) > d1) >= 2)
    hxs = [sorted(a for a in dx if dx[a] > d2) for dx in degx]
    return rels, hxs, hy


def star_algorithm(rels, d1: int, d2: int):
    """Section 3.2 steps 1-3; returns dict with the result and V, W."""
    import itertools
    k = len(rels)
    rels, hxs, hy = star_partition(rels, d1, d2)
    hsets = [set(h) for h in hxs]
    hyset = set(hy)
    by_y = [defaultdict(list) for _ in range(k)]
    for i, r in enumerate(rels):
        for a, b in r:
            by_y[i][b].append(a)
    # steps 1 and 2 (disjoint form): every witness combination except the
    # all-heavy ones (every a_i heavy and b heavy)
    T = set()
    for b in set(by_y[0]):
        lists = [by_y[i].get(b, []) for i in range(k)]
        for t in itertools.product(*lists):
            if b in hyset and all(t[i] in hsets[i] for i in range(k)):
                continue
            T.add(t)
    # step 3: V (ceil(k/2)-tuples x heavy y), W (floor(k/2)-tuples x heavy y)
    kv = (k + 1) // 2
    iy = {b: j for j, b in enumerate(hy)}
    relsets = [set(r) for r in rels]
    vrows = list(itertools.product(*hxs[:kv]))
    wrows = list(itertools.product(*hxs[kv:]))
    V = np.zeros((len(vrows), len(hy)), np.int64)
    W = np.zeros((len(wrows), len(hy)), np.int64)
    for r, t in enumerate(vrows):
        for b in hy:
            if all((t[i], b) in relsets[i] for i in range(kv)):
                V[r, iy[b]] = 1
    for r, t in enumerate(wrows):
        for b in hy:
            if all((t[i], b) in relsets[kv + i] for i in range(k - kv)):
                W[r, iy[b]] = 1
    P = V @ W.T
    for i, l in zip(*np.nonzero(P)):
        T.add(tuple(vrows[i]) + tuple(wrows[l]))
    return dict(T=sorted(T), V=V, W=W, vrows=vrows, wrows=wrows, hy=hy, hxs=hxs)
