"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each check is independent of the oracle's own code path: brute-force loops,
closed forms, invariants, the paper's worked examples (Section 3.1 and
Section 3.2, with the two printed errata corrected) and a numpy integer
matrix product for the all-heavy case.
"""
import json
import os

import numpy as np
import pytest

from oracle import algorithm1 as A1

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _pairs(cols):
    return list(zip(*[c.tolist() for c in cols]))


def _rand_rel(rng, n, dx, dy, ox=0, oy=0):
    x = rng.integers(0, dx, n) + ox
    y = rng.integers(0, dy, n) + oy
    return x.astype(np.int32), y.astype(np.int32)


@pytest.mark.parametrize("seed", range(24))
def test_two_path_matches_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 120))
    rx, ry = _rand_rel(rng, n, int(rng.integers(1, 15)), int(rng.integers(1, 12)), -7, -3)
    if seed % 3 == 0:
        sz, sy = rx, ry
    else:
        m = int(rng.integers(0, 120))
        sz, sy = _rand_rel(rng, m, int(rng.integers(1, 15)), int(rng.integers(1, 12)), -5, -3)
    got = _pairs(oracle_mod.two_path(rx, ry, sz, sy))
    assert got == oracle_mod.brute_two_path(rx, ry, sz, sy)


def test_two_path_not_symmetric_in_operands(oracle_mod):
    # R != S: swapping the operands transposes the result, it does not keep it
    R = (np.array([0, 0, 1], np.int32), np.array([5, 6, 6], np.int32))
    S = (np.array([7, 8], np.int32), np.array([5, 9], np.int32))
    assert _pairs(oracle_mod.two_path(*R, *S)) == [(0, 7)]
    assert _pairs(oracle_mod.two_path(*S, *R)) == [(7, 0)]


@pytest.mark.parametrize("k,seed", [(2, 0), (2, 1), (3, 2), (3, 3), (3, 4), (4, 5)])
def test_star_matches_brute_force(oracle_mod, k, seed):
    rng = np.random.default_rng(100 + seed)
    rels = [_rand_rel(rng, int(rng.integers(1, 40)), 6, 5, -2, 0) for _ in range(k)]
    got = _pairs(oracle_mod.star(rels))
    assert got == oracle_mod.brute_star(rels)


@pytest.mark.parametrize("a,b", [(1, 1), (3, 5), (17, 4), (40, 1)])
def test_complete_bipartite_gives_a_squared(oracle_mod, a, b):
    xs, ys = np.meshgrid(np.arange(a), np.arange(b), indexing="ij")
    ox, oz = oracle_mod.two_path(xs.ravel(), ys.ravel())
    assert len(ox) == a * a
    assert _pairs((ox, oz)) == [(i, j) for i in range(a) for j in range(a)]


def test_star_graph_gives_one_clique(oracle_mod):
    d = 37
    xs = np.arange(d, dtype=np.int32) * 3 - 50
    ys = np.full(d, 11, np.int32)
    ox, oz = oracle_mod.two_path(xs, ys)
    assert len(ox) == d * d
    assert set(_pairs((ox, oz))) == {(int(p), int(q)) for p in xs for q in xs}


def test_disjoint_communities_sum_of_squares(oracle_mod):
    # Example 1: communities of users sharing friends; each community is a
    # clique of pairs, so OUT = sum c_i^2 while the join is larger
    sizes = [5, 1, 9, 4]
    xs, ys = [], []
    base = 0
    for ci, c in enumerate(sizes):
        for u in range(c):
            for f in range(3):               # three shared friends per community
                xs.append(base + u)
                ys.append(1000 * ci + f)
        base += c
    ox, oz = oracle_mod.two_path(np.array(xs), np.array(ys))
    assert len(ox) == sum(c * c for c in sizes)


@pytest.mark.parametrize("seed", range(6))
def test_self_join_invariants(oracle_mod, seed):
    rng = np.random.default_rng(7 + seed)
    rx, ry = _rand_rel(rng, 400, 60, 40)
    ox, oz = oracle_mod.two_path(rx, ry)
    pairs = set(_pairs((ox, oz)))
    assert all((c, a) in pairs for a, c in pairs)                 # symmetric
    assert all((a, a) in pairs for a in set(rx.tolist()))         # diagonal
    ux, uy = oracle_mod.normalise(rx, ry)
    degy = np.unique(uy, return_counts=True)[1].astype(np.int64)
    out_join = int((degy * degy).sum())
    domx = len(np.unique(ux))
    assert domx <= len(pairs) <= min(domx * domx, out_join)       # Section 5 bounds


@pytest.mark.parametrize("seed", range(4))
def test_witness_counts_match_integer_product(oracle_mod, seed):
    rng = np.random.default_rng(50 + seed)
    rx, ry = _rand_rel(rng, 300, 30, 20)
    sz, sy = _rand_rel(rng, 250, 25, 20)
    ox, oz, oc = oracle_mod.two_path(rx, ry, sz, sy, with_counts=True)
    A = np.zeros((30, 20), np.int64)
    B = np.zeros((25, 20), np.int64)
    A[rx, ry] = 1
    B[sz, sy] = 1
    M = A @ B.T
    nz = np.nonzero(M)
    assert np.array_equal(ox, nz[0]) and np.array_equal(oz, nz[1])
    assert np.array_equal(oc, M[nz])


def test_row_oracle_matches_full(oracle_mod):
    rng = np.random.default_rng(3)
    rx, ry = _rand_rel(rng, 800, 50, 30, -20, 0)
    ox, oz = oracle_mod.two_path(rx, ry)
    srt = oracle_mod.SortedS(rx, ry)
    for a in np.unique(rx):
        row = oracle_mod.two_path_row(ry[rx == a], srt)
        assert np.array_equal(row, oz[ox == a])


def test_x_range_restriction(oracle_mod):
    rng = np.random.default_rng(4)
    rx, ry = _rand_rel(rng, 500, 40, 25)
    ox, oz = oracle_mod.two_path(rx, ry)
    px, pz = oracle_mod.two_path(rx, ry, x_lo=10, x_hi=19)
    sel = (ox >= 10) & (ox <= 19)
    assert np.array_equal(px, ox[sel]) and np.array_equal(pz, oz[sel])


def test_worked_two_path_example(oracle_mod):
    g = json.load(open(os.path.join(GOLD, "two_path_example.json")))
    R = [tuple(t) for t in g["R"]]
    S = [tuple(t) for t in g["S"]]
    res = A1.algorithm1(R, S, g["delta1"], g["delta2"])
    assert res["hx"] == g["heavy_x"] and res["hy"] == g["heavy_y"] and res["hz"] == g["heavy_z"]
    assert res["M1"].tolist() == g["M1"]
    assert res["M2"].tolist() == g["M2"]
    assert res["M"].tolist() == g["M"]
    assert res["Rm"] == sorted(tuple(t) for t in g["R_light_edges_drawn_red"])
    assert res["Sm"] == sorted(tuple(t) for t in g["S_light_edges_drawn_green"])
    rx, ry = np.array(R).T
    sz, sy = np.array(S).T
    full = _pairs(oracle_mod.two_path(rx, ry, sz, sy))
    assert res["T"] == full == oracle_mod.brute_two_path(rx, ry, sz, sy)


def test_worked_star_example(oracle_mod):
    g = json.load(open(os.path.join(GOLD, "star_example.json")))
    rels = [[tuple(t) for t in g[n]] for n in "RSTU"]
    res = A1.star_algorithm(rels, g["delta1"], g["delta2"])
    assert res["hy"] == g["heavy_y"]
    assert len(res["vrows"]) == g["heavy_pairs_per_side"] == len(res["wrows"])
    for key, row in g["V_rows"].items():
        t = tuple(int(v) for v in key.split(","))
        assert res["V"][res["vrows"].index(t)].tolist() == row
    for key, col in g["W_cols"].items():
        t = tuple(int(v) for v in key.split(","))
        assert res["W"][res["wrows"].index(t)].tolist() == col
    arrs = [tuple(np.array(r, np.int32).T) for r in rels]
    full = _pairs(oracle_mod.star(arrs))
    assert res["T"] == full == oracle_mod.brute_star(arrs)


@pytest.mark.parametrize("seed", range(5))
def test_algorithm1_invariant_to_thresholds(oracle_mod, seed):
    rng = np.random.default_rng(200 + seed)
    rx, ry = _rand_rel(rng, 250, 25, 12)
    sz, sy = (rx, ry) if seed % 2 else _rand_rel(rng, 200, 20, 12)
    R = list(zip(rx.tolist(), ry.tolist()))
    S = list(zip(sz.tolist(), sy.tolist()))
    want = _pairs(oracle_mod.two_path(rx, ry, sz, sy))
    for d1 in (1, 2, 3, 5, 8, 100):
        for d2 in (1, 2, 4, 7, 100):
            assert A1.algorithm1(R, S, d1, d2)["T"] == want


def test_all_heavy_reduces_to_boolean_product(oracle_mod):
    # every degree >= 2 and thresholds 1: every tuple is heavy, the light
    # part is empty and Q is the Boolean product of the adjacency matrices
    rng = np.random.default_rng(9)
    A = (rng.random((12, 9)) < 0.5).astype(np.int64)
    A[:, 0] = 1
    A[:, 1] = 1
    rx, ry = np.nonzero(A)
    R = list(zip(rx.tolist(), ry.tolist()))
    res = A1.algorithm1(R, R, 1, 1)
    assert res["light"] == 0 and len(res["Rm"]) == 0
    P = (A @ A.T) > 0
    want = [(int(i), int(j)) for i, j in zip(*np.nonzero(P))]
    assert res["T"] == want == _pairs(oracle_mod.two_path(rx, ry))


def test_all_light_when_threshold_exceeds_degrees():
    rng = np.random.default_rng(10)
    rx, ry = _rand_rel(rng, 300, 30, 15)
    R = list(zip(rx.tolist(), ry.tolist()))
    res = A1.algorithm1(R, R, 10 ** 6, 10 ** 6)
    assert res["M"].size == 0 and len(res["Rm"]) == len(set(R))


@pytest.mark.parametrize("seed", range(4))
def test_star_invariant_to_thresholds(oracle_mod, seed):
    rng = np.random.default_rng(300 + seed)
    k = 3
    rels = [_rand_rel(rng, 60, 8, 5) for _ in range(k)]
    tl = [list(zip(r[0].tolist(), r[1].tolist())) for r in rels]
    want = _pairs(oracle_mod.star(rels))
    for d1 in (1, 2, 4, 50):
        for d2 in (1, 3, 50):
            assert A1.star_algorithm(tl, d1, d2)["T"] == want


def test_two_path_rows_is_the_row_wise_definition(oracle_mod):
    """The batched per-row oracle equals the whole-relation oracle, row by row."""
    from paper_2002_12459_gb300 import workloads as W
    rng = np.random.default_rng(21)
    x, y = W.random_small_relation(rng, 3000, 200, 80, -100, -40, 0.7)
    s = oracle_mod.SortedS(x, y)
    key = np.unique((x.astype(np.int64) << 32) | (y.astype(np.int64) & 0xFFFFFFFF))
    ux = (key >> 32).astype(np.int32)
    uy = (key & 0xFFFFFFFF).astype(np.uint32).astype(np.int32)
    xs, start = np.unique(ux, return_index=True)
    off = np.append(start, len(ux)).astype(np.int64)
    z, cnt = oracle_mod.two_path_rows(off, uy, s)
    wx, wz = oracle_mod.two_path(x, y)
    assert np.array_equal(z, wz)
    assert np.array_equal(np.repeat(xs, cnt), wx)
    # a subset of rows, out of order of their x values
    pick = np.array([5, 1, 17, 3])
    sub_off = np.concatenate([[0], np.cumsum(off[pick + 1] - off[pick])]).astype(np.int64)
    sub_y = np.concatenate([uy[off[i]:off[i + 1]] for i in pick])
    z2, c2 = oracle_mod.two_path_rows(sub_off, sub_y, s)
    for k, i in enumerate(pick):
        assert np.array_equal(z2[sub_off[k] - sub_off[k] + c2[:k].sum():c2[:k + 1].sum()],
                              wz[wx == xs[i]])
