"""Pins of the oracle's batch of boolean set intersection queries (Section 3.3).

Q_batch(x,z) = R(x,y), S(z,y), T(x,z): a pair (a, b) of T is answered iff the
sets R(a, .) and S(b, .) intersect.  The oracle computes it as a three-way join
and projection; the pins check it against a pure-Python loop, against the
two-path oracle (T holding every pair of the domains gives Q itself, and in
general the answer is T intersected with Q), against the worked example's
matrix product (Section 3.1), and on the degenerate cases.
"""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _pairs(cols):
    return list(zip(*[c.tolist() for c in cols]))


def _rand(rng, n, lo, hi):
    return rng.integers(lo, hi, n).astype(np.int32)


@pytest.mark.parametrize("seed", range(16))
def test_bsi_matches_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 40))
    rx, ry = _rand(rng, n, -6, 6), _rand(rng, n, -4, 5)
    m = int(rng.integers(0, 40))
    sz, sy = _rand(rng, m, -6, 7), _rand(rng, m, -4, 5)
    t = int(rng.integers(0, 50))
    # T also names values absent from R and S, and repeats pairs
    tx, tz = _rand(rng, t, -8, 9), _rand(rng, t, -8, 9)
    tx, tz = np.concatenate([tx, tx[: t // 3]]), np.concatenate([tz, tz[: t // 3]])
    got = _pairs(oracle_mod.bsi(rx, ry, tx, tz, sz, sy))
    assert got == oracle_mod.brute_bsi(rx, ry, tx, tz, sz, sy)


@pytest.mark.parametrize("seed", range(6))
def test_bsi_over_every_pair_is_the_two_path_query(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    rx, ry = _rand(rng, 400, -30, 30), _rand(rng, 400, 0, 25)
    sz, sy = _rand(rng, 300, -20, 40), _rand(rng, 300, 0, 25)
    a, b = np.meshgrid(np.unique(rx), np.unique(sz), indexing="ij")
    got = oracle_mod.bsi(rx, ry, a.ravel(), b.ravel(), sz, sy)
    want = oracle_mod.two_path(rx, ry, sz, sy)
    assert _pairs(got) == _pairs(want)


@pytest.mark.parametrize("seed", range(6))
def test_bsi_is_the_candidates_within_the_two_path_query(oracle_mod, seed):
    rng = np.random.default_rng(200 + seed)
    rx, ry = _rand(rng, 3000, -500, 500), _rand(rng, 3000, 0, 200)
    self_join = seed % 2 == 0
    sz, sy = (None, None) if self_join else (_rand(rng, 2000, -400, 600), _rand(rng, 2000, 0, 200))
    tx, tz = _rand(rng, 5000, -600, 600), _rand(rng, 5000, -600, 700)
    q = set(_pairs(oracle_mod.two_path(rx, ry, sz, sy)))
    want = sorted(set(zip(tx.tolist(), tz.tolist())) & q)
    assert _pairs(oracle_mod.bsi(rx, ry, tx, tz, sz, sy)) == want
    assert len(want) > 0


def test_bsi_follows_the_worked_example_product(oracle_mod):
    """Every heavy pair with a positive entry of M = M1 x M2 is answered."""
    ex = json.load(open(os.path.join(GOLD, "two_path_example.json")))
    R = np.array(ex["R"], np.int32)
    S = np.array(ex["S"], np.int32)
    hx, hz = ex["heavy_x"], ex["heavy_z"]
    tx = np.array([a for a in hx for _ in hz], np.int32)
    tz = np.array([b for _ in hx for b in hz], np.int32)
    got = set(_pairs(oracle_mod.bsi(R[:, 0], R[:, 1], tx, tz, S[:, 0], S[:, 1])))
    for i, a in enumerate(hx):
        for j, b in enumerate(hz):
            if ex["M"][i][j] > 0:
                assert (a, b) in got
    # x = 1 has the single y 6 and z = 3 the single y 3: no common y
    none = oracle_mod.bsi(R[:, 0], R[:, 1], np.array([1], np.int32), np.array([3], np.int32),
                          S[:, 0], S[:, 1])
    assert len(none[0]) == 0


def test_bsi_degenerate_cases(oracle_mod):
    rx = np.array([1, 1, 2], np.int32)
    ry = np.array([5, 6, 5], np.int32)
    e = np.empty(0, np.int32)
    assert len(oracle_mod.bsi(rx, ry, e, e)[0]) == 0                       # empty T
    assert len(oracle_mod.bsi(e, e, rx, ry)[0]) == 0                       # empty R
    assert len(oracle_mod.bsi(rx, ry, np.array([7], np.int32), np.array([1], np.int32))[0]) == 0
    # a pair and its repeats: one answer; (a, a) is answered for every a of R
    got = oracle_mod.bsi(rx, ry, np.array([2, 2, 2, 1], np.int32), np.array([1, 1, 1, 1], np.int32))
    assert _pairs(got) == [(1, 1), (2, 1)]
    lim = np.array([-(1 << 31), (1 << 31) - 1], np.int32)
    got = oracle_mod.bsi(lim, lim, lim[::-1], lim)
    assert _pairs(got) == []
    got = oracle_mod.bsi(lim, np.zeros(2, np.int32), lim[::-1], lim)
    assert _pairs(got) == [(-(1 << 31), (1 << 31) - 1), ((1 << 31) - 1, -(1 << 31))]
