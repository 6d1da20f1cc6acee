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
