"""Pins of the oracle's set similarity join (Section 1) and its ordered form (Section 4).

The count of a pair is the number of y its two sets share, the entry M_ac of
the product M1 x M2 (Section 2.2).  Checked against pure-Python set
intersections, against a numpy integer matrix product on dense 0/1 matrices,
against the worked example's M on its heavy block, and for the order: count
descending with ties in (x, z) order, c_min = 1 giving the two-path query.
"""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand(rng, n, lo, hi):
    return rng.integers(lo, hi, n).astype(np.int32)


@pytest.mark.parametrize("seed", range(12))
def test_ssj_matches_set_intersections(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    rx, ry = _rand(rng, 60, -7, 7), _rand(rng, 60, -5, 6)
    sz, sy = (None, None) if seed % 3 == 0 else (_rand(rng, 50, -6, 9), _rand(rng, 50, -5, 6))
    for c in (1, 2, 3):
        got = list(zip(*[a.tolist() for a in oracle_mod.ssj(rx, ry, c, sz, sy)]))
        assert got == oracle_mod.brute_ssj(rx, ry, c, sz, sy)


@pytest.mark.parametrize("seed", range(4))
def test_counts_are_the_integer_matrix_product(oracle_mod, seed):
    rng = np.random.default_rng(40 + seed)
    rx, ry = _rand(rng, 3000, 0, 120), _rand(rng, 3000, 0, 80)
    sz, sy = _rand(rng, 2500, 0, 150), _rand(rng, 2500, 0, 80)
    M1 = np.zeros((120, 80), np.int64)
    M1[rx, ry] = 1
    M2 = np.zeros((150, 80), np.int64)
    M2[sz, sy] = 1
    M = M1 @ M2.T
    ox, oz, oc = oracle_mod.ssj(rx, ry, 2, sz, sy)
    a, c = np.nonzero(M >= 2)
    assert np.array_equal(ox, a) and np.array_equal(oz, c) and np.array_equal(oc, M[a, c])


def test_worked_example_counts(oracle_mod):
    """Heavy pairs of the worked example (Section 3.1): the count is the heavy product's
    entry M_ac plus the witnesses through a light tuple (the figure's red and green edges)."""
    ex = json.load(open(os.path.join(GOLD, "two_path_example.json")))
    R = np.array(ex["R"], np.int32)
    S = np.array(ex["S"], np.int32)
    ox, oz, oc = oracle_mod.ssj(R[:, 0], R[:, 1], 1, S[:, 0], S[:, 1])
    cnt = {(a, c): k for a, c, k in zip(ox.tolist(), oz.tolist(), oc.tolist())}
    red = {tuple(e) for e in ex["R_light_edges_drawn_red"]}
    green = {tuple(e) for e in ex["S_light_edges_drawn_green"]}
    Rs = {tuple(e) for e in ex["R"]}
    Ss = {tuple(e) for e in ex["S"]}
    ys = {y for _, y in Rs} | {y for _, y in Ss}
    for i, a in enumerate(ex["heavy_x"]):
        for j, c in enumerate(ex["heavy_z"]):
            light = sum(1 for y in ys if (a, y) in Rs and (c, y) in Ss
                        and ((a, y) in red or (c, y) in green))
            assert cnt.get((a, c), 0) == ex["M"][i][j] + light


def test_order_by_count(oracle_mod):
    rng = np.random.default_rng(7)
    rx, ry = _rand(rng, 4000, -300, 300), _rand(rng, 4000, 0, 60)
    ox, oz, oc = oracle_mod.ssj(rx, ry, 1, order="count")
    px, pz, pc = oracle_mod.ssj(rx, ry, 1)
    assert sorted(zip(ox.tolist(), oz.tolist(), oc.tolist())) == list(zip(px.tolist(), pz.tolist(), pc.tolist()))
    assert (np.diff(oc) <= 0).all()
    same = np.diff(oc) == 0
    key = ox.astype(np.int64) * (1 << 32) + (oz.astype(np.int64) + (1 << 31))
    assert (np.diff(key)[same] > 0).all()
    # the self-join's diagonal carries each set's size
    deg = {a: len(set(ry[rx == a].tolist())) for a in np.unique(rx).tolist()}
    diag = ox == oz
    assert all(deg[a] == k for a, k in zip(ox[diag].tolist(), oc[diag].tolist()))


def test_c_min_one_is_the_two_path_query(oracle_mod):
    rng = np.random.default_rng(8)
    rx, ry = _rand(rng, 2000, -100, 100), _rand(rng, 2000, -40, 40)
    ox, oz, _ = oracle_mod.ssj(rx, ry, 1)
    wx, wz = oracle_mod.two_path(rx, ry)
    assert np.array_equal(ox, wx) and np.array_equal(oz, wz)
    big = oracle_mod.ssj(rx, ry, 10 ** 6)
    assert len(big[0]) == 0
