"""The seeded generators: determinism, exact sizes, distinctness, shape."""
import numpy as np
import pytest

from paper_2002_12459_gb300 import workloads as W


def _distinct(x, y):
    return len(np.unique(x.astype(np.int64) * (1 << 32) + y.astype(np.int64)))


def test_uniform_small_workload_shape():
    x, y = W.make("two_path_uniform_20k")
    assert len(x) == 20_000 and _distinct(x, y) == 20_000
    assert x.min() >= 0 and x.max() < 2000 and y.min() >= 0 and y.max() < 500
    x2, y2 = W.make("two_path_uniform_20k")
    assert np.array_equal(x, x2) and np.array_equal(y, y2)


def test_powerlaw_small_instance():
    x, y = W.powerlaw_relation(50_000, 10_000, 2.1, 5_000, 1.8, seed=3)
    assert len(x) == 50_000 and _distinct(x, y) == 50_000
    assert x.max() < 10_000 and y.max() < 5_000
    degy = np.unique(y, return_counts=True)[1]
    # heavy tail: the largest y degree is far above the mean
    assert degy.max() > 10 * degy.mean()


def test_solve_dmax_monotone():
    d = W.solve_dmax(1.8, 10.0)
    assert W._pl_mean(1.8, d) >= 10.0 > W._pl_mean(1.8, d - 1)
    assert abs(W.powerlaw_pmf(1.5, 100).sum() - 1) < 1e-12


def test_star_relations_share_y_sequence():
    rels = W.star_relations(3, 20_000, 5_000, 2_000, 1.5, seed=0)
    assert len(rels) == 3
    degs = [np.bincount(r[1], minlength=2000) for r in rels]
    # same target degrees on the same ids: realized degrees correlate strongly
    c = np.corrcoef(degs[0], degs[1])[0, 1]
    assert c > 0.8
    for x, y in rels:
        assert len(x) == 20_000 and _distinct(x, y) == 20_000


def test_candidate_pairs_draws():
    vals = np.array([-7, 3, 11, 40], np.int32)
    a, b = W.candidate_pairs(vals, vals, 4000, seed=2)
    assert set(a.tolist()) == set(vals.tolist()) and set(b.tolist()) == set(vals.tolist())
    # weights: all mass on one value for x, proportional draws for z
    a, b = W.candidate_pairs(vals, vals, 20000, seed=3, x_weights=[0, 0, 1, 0],
                             z_weights=[1, 1, 2, 0])
    assert (a == 11).all()
    frac = np.array([(b == v).mean() for v in vals])
    assert np.allclose(frac, [0.25, 0.25, 0.5, 0.0], atol=0.02)
    # absent values lie outside the given ones, on one side of each such pair
    a, b = W.candidate_pairs(vals, vals, 20000, seed=4, absent=0.3)
    miss_a = ~np.isin(a, vals)
    miss_b = ~np.isin(b, vals)
    assert not (miss_a & miss_b).any()
    assert abs((miss_a | miss_b).mean() - 0.3) < 0.02
    assert len(W.candidate_pairs(vals, vals, 0)[0]) == 0
