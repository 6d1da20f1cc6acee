"""Host logic of the product tile autotuner (no GPU)."""
import json
import os

import numpy as np

from paper_2002_12459_gb300 import tune


def test_dense_relation_makes_every_value_heavy_at_threshold_one():
    for u, v in [(256, 512), (2048, 512), (300, 7)]:
        x, y = tune.dense_relation(u, v, seed=1)
        k = np.unique(x.astype(np.int64) * 100000 + y)
        dx = np.bincount(k // 100000, minlength=u)
        dy = np.bincount(k % 100000, minlength=v)
        assert len(dx) == u and len(dy) == v
        assert dx.min() >= 2 and dy.min() >= 2


def test_crossover_sums_over_k_and_stops_at_the_first_loss():
    rows = [dict(wide_tiles=2, ms_128=1.0, ms_256=0.9), dict(wide_tiles=2, ms_128=1.0, ms_256=1.5),
            dict(wide_tiles=8, ms_128=1.0, ms_256=1.1), dict(wide_tiles=32, ms_128=2.0, ms_256=1.0),
            dict(wide_tiles=128, ms_128=1.0, ms_256=2.0)]
    assert tune.crossover(rows) == 8
    assert tune.crossover([dict(wide_tiles=2, ms_128=2.0, ms_256=1.0)]) == 0


def test_shipped_table_is_consistent():
    with open(tune.DEFAULT_OUT) as f:
        t = json.load(f)
    assert t["auto_max_tiles"] == tune.crossover(t["measurements"])
    assert {r["u"] for r in t["measurements"]} == set(tune.U_GRID)
