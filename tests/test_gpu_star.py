"""Parity of the CUDA star query (Section 3.2) with the CPU oracle.

The result is a set of integer tuples: bit-exact equality of the sorted
distinct tuples and their count.  Thresholds are swept because the output
must not depend on them.
"""
import numpy as np
import pytest

from paper_2002_12459_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2002_12459_gb300 import build, jp
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the -m gpu tests")
    c = jp.Context(0)
    yield c
    c.close()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def run(ctx, rels, mode="fixed", d1=1, d2=1):
    ctx.set_threshold(mode, d1, d2)
    cols = ctx.star([(dev(x), dev(y)) for x, y in rels])
    return tuple(c.cpu().numpy() for c in cols)


def same(got, want):
    assert len(got) == len(want)
    for g, w in zip(got, want):
        assert len(g) == len(w), (len(g), len(w))
        assert np.array_equal(g, w)


def rel(rng, n, dx, dy, ox=0, oy=0, skew=0.0):
    return W.random_small_relation(rng, n, dx, dy, ox, oy, skew)


@pytest.mark.parametrize("seed", range(6))
def test_star3_threshold_sweep(ctx, oracle_mod, seed):
    rng = np.random.default_rng(seed)
    rels = [rel(rng, 900, 120, 60, -40 * i, -5, skew=0.7) for i in range(3)]
    want = oracle_mod.star(rels)
    for d1, d2 in [(1, 1), (2, 2), (3, 8), (8, 3), (30, 30), (10 ** 6, 10 ** 6)]:
        same(run(ctx, rels, d1=d1, d2=d2), want)


def test_star3_dense_core_uses_the_product(ctx, oracle_mod):
    # a dense core (every x of degree > Delta2, every y heavy in all three
    # relations) plus a sparse fringe: the heavy pairs go through the GEMM
    rng = np.random.default_rng(7)
    rels = []
    for i in range(3):
        xs, ys = np.meshgrid(np.arange(40), np.arange(30), indexing="ij")
        keep = rng.random(xs.shape) < 0.6
        fx, fy = rel(rng, 300, 500, 200, 100, 50)
        rels.append((np.concatenate([xs[keep], fx]).astype(np.int32),
                     np.concatenate([ys[keep], fy]).astype(np.int32)))
    want = oracle_mod.star(rels)
    same(run(ctx, rels, d1=3, d2=3), want)
    st = ctx.stats()
    assert st["u"] > 0 and st["v"] > 0 and st["w"] > 0
    same(run(ctx, rels, d1=1, d2=1), want)
    same(run(ctx, rels, mode="closed_form"), want)


def test_star3_identical_relations(ctx, oracle_mod):
    rng = np.random.default_rng(3)
    r = rel(rng, 1500, 200, 50, skew=0.5)
    want = oracle_mod.star([r, r, r])
    x, y = dev(r[0]), dev(r[1])
    for d in (1, 4, 10 ** 6):
        ctx.set_threshold("fixed", d, d)
        got = tuple(c.cpu().numpy() for c in ctx.star([(x, y), (x, y), (x, y)]))
        same(got, want)


def test_star3_worked_example_relations(ctx, oracle_mod):
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "star_example.json")))
    rels = [tuple(np.array(g[n], np.int32).T) for n in "RST"]
    want = oracle_mod.star(rels)
    for d in (1, 2, 3):
        same(run(ctx, rels, d1=d, d2=d), want)


def test_star2_is_two_path(ctx, oracle_mod):
    rng = np.random.default_rng(4)
    r1 = rel(rng, 2000, 300, 80, skew=0.6)
    r2 = rel(rng, 1500, 250, 80, -100, 0, skew=0.4)
    want = oracle_mod.two_path(r1[0], r1[1], r2[0], r2[1])
    same(run(ctx, [r1, r2], d1=3, d2=3), want)


def test_star_limits_and_empty(ctx):
    from paper_2002_12459_gb300 import jp
    e = np.empty(0, np.int32)
    got = run(ctx, [(e, e)] * 3)
    assert all(len(c) == 0 for c in got)
    one = (np.array([1], np.int32), np.array([2], np.int32))
    assert [c.tolist() for c in run(ctx, [one] * 4)] == [[1]] * 4
    with pytest.raises(jp.JPError) as ei:
        run(ctx, [one] * 9)
    assert ei.value.code == jp.JP_EINVAL
    # k = 5 with one relation sharing no y with the others: empty
    got = run(ctx, [one, one, one, (np.array([1], np.int32), np.array([3], np.int32)), one])
    assert len(got) == 5 and all(len(c) == 0 for c in got)
    # relations sharing no y: empty result
    got = run(ctx, [one, (np.array([1], np.int32), np.array([3], np.int32)), one])
    assert all(len(c) == 0 for c in got)


@pytest.mark.parametrize("k,seed", [(4, 0), (4, 1), (5, 2), (6, 3), (7, 4)])
def test_star_k_above_3(ctx, oracle_mod, k, seed):
    # the tail R3..Rk is grouped on y (pairs of relations, from the right) and
    # Q*_k answered as Q*_3; small shared y domain so that every y joins
    rng = np.random.default_rng(seed)
    n = {4: 400, 5: 200, 6: 110, 7: 80}[k]
    rels = [rel(rng, n, 60 + 7 * i, 25, -30 * (i % 2), 0, skew=0.5) for i in range(k)]
    want = oracle_mod.star(rels)
    assert len(want[0]) > 0
    for mode, d1, d2 in [("fixed", 1, 1), ("fixed", 3, 2), ("fixed", 10 ** 6, 10 ** 6),
                         ("cost_model", 1, 1)]:
        got = run(ctx, rels, mode, d1, d2)
        assert len(got) == k
        same(got, want)
