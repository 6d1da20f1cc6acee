"""Parity of threshold selection (the a3 step: Section 3.1 closed forms, Section 5's output
estimate and degree indexes, Algorithm 3) with the oracle's cost model.

The query's output does not depend on the thresholds, so the parity tests of the result cannot
see a wrong choice here; these tests compare the choice itself.  The library reports what it
used in jp_stats; the oracle recomputes every quantity from the relations with numpy
(``oracle.cost_model``), with the same calibration constants passed to both sides as numbers.
"""
import math

import numpy as np
import pytest

from oracle import cost_model as CM
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
    c.set_cost_model()
    c.close()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _run(ctx, rel, mode, d1=1, d2=1):
    rx, ry, sz, sy = rel
    ctx.set_threshold(mode, d1, d2)
    if sz is None:
        ox, _ = ctx.two_path(dev(rx), dev(ry))
    else:
        ox, _ = ctx.two_path(dev(rx), dev(ry), dev(sz), dev(sy))
    st = ctx.stats()
    assert st["out_count"] == ox.numel()
    return st


def _relations():
    rng = np.random.default_rng(11)
    rels = {}
    x, y = W.make("two_path_uniform_20k")
    rels["uniform_20k"] = (x, y, None, None)
    x, y = W.make("two_path_powerlaw_1m")
    rels["powerlaw_1m"] = (x, y, None, None)
    # R != S, skewed, with negatives, duplicates and dangling y on both sides
    rx, ry = W.random_small_relation(rng, 6000, 700, 60, -350, -20, 0.8)
    sz, sy = W.random_small_relation(rng, 9000, 900, 50, -2000, -12, 0.6)
    rels["skewed_r_ne_s"] = (rx, ry, sz, sy)
    # R != S, two power laws over one y domain (different seeds and exponents)
    rx, ry = W.powerlaw_relation(200_000, 40_000, 2.1, 3_000, 1.8, seed=3)
    sz, sy = W.powerlaw_relation(150_000, 30_000, 1.9, 3_000, 1.6, seed=4)
    rels["powerlaw_r_ne_s"] = (rx, ry, sz, sy)
    return rels


RELS = None


def rels():
    global RELS
    if RELS is None:
        RELS = _relations()
    return RELS


def _oracle_of(rel):
    rx, ry, sz, sy = rel
    return CM.index_of_relations(rx, ry, sz, sy)


# Constant sets: the library's defaults, and sets that move Algorithm 3's stopping point
# (cheap product: deep descent; light work nearly free: shallow; T_s and T_m weighted).
CONSTS = [
    None,
    # the constants measured on the 10M relation alone (the earlier defaults)
    dict(T_I=1.0 / 60e9, T_m=1e-12, T_s=0.0, mm_rate=2.2e15, mm_fixed=2e-5, eps=0.05),
    dict(T_I=1e-10, T_m=1e-12, T_s=0.0, mm_rate=1e17, mm_fixed=0.0, eps=0.05),
    dict(T_I=1e-13, T_m=1e-12, T_s=0.0, mm_rate=1e13, mm_fixed=1e-3, eps=0.05),
    dict(T_I=2e-11, T_m=5e-11, T_s=1e-14, mm_rate=3e15, mm_fixed=5e-5, eps=0.1),
    dict(T_I=1.0 / 60e9, T_m=1e-12, T_s=0.0, mm_rate=2.2e15, mm_fixed=2e-5, eps=0.2,
         wcoj_factor=0.0),
]


@pytest.mark.parametrize("name", ["uniform_20k", "powerlaw_1m", "skewed_r_ne_s", "powerlaw_r_ne_s"])
def test_indexes_and_output_estimate(ctx, name):
    rel = rels()[name]
    idx, info = _oracle_of(rel)
    st = _run(ctx, rel, "fixed", 5, 5)
    assert st["n_r"] == info["n_r"] and st["n_s"] == info["n_s"]
    assert st["dom_x"] == info["dom_x"] and st["dom_y"] == info["dom_y"]
    assert st["dom_z"] == info["dom_z"]
    assert st["out_join"] == float(info["out_join"])             # exact (below 2^53)
    est = CM.out_estimate(info["dom_x"], float(info["out_join"]), info["N"])
    assert st["out_estimate"] == pytest.approx(est, rel=1e-12)
    # the partition at fixed thresholds is the index's heavy counts
    assert (st["u"], st["v"], st["w"]) == (idx.heavy_x(5), idx.heavy_y(5), idx.heavy_z(5))


@pytest.mark.parametrize("name", ["uniform_20k", "powerlaw_1m", "skewed_r_ne_s", "powerlaw_r_ne_s"])
def test_closed_form_thresholds(ctx, name):
    rel = rels()[name]
    idx, info = _oracle_of(rel)
    st = _run(ctx, rel, "closed_form")
    N = info["N"]
    OUT = max(CM.out_estimate(info["dom_x"], float(info["out_join"]), N), 1.0)
    a, b = CM.closed_form(float(N), OUT)
    want = (CM.to_int_threshold(a, N), CM.to_int_threshold(b, N))
    assert (st["delta1"], st["delta2"]) == want, (a, b)
    d1, d2 = want
    assert (st["u"], st["v"], st["w"]) == (idx.heavy_x(d2), idx.heavy_y(d1), idx.heavy_z(d2))


@pytest.mark.parametrize("ci", range(len(CONSTS)))
@pytest.mark.parametrize("name", ["uniform_20k", "powerlaw_1m", "skewed_r_ne_s", "powerlaw_r_ne_s"])
def test_algorithm3_thresholds(ctx, name, ci):
    rel = rels()[name]
    idx, info = _oracle_of(rel)
    if CONSTS[ci] is None:
        ctx.set_cost_model()
    else:
        ctx.set_cost_model(**CONSTS[ci])
    K = ctx.cost_model()
    try:
        st = _run(ctx, rel, "cost_model")
    finally:
        ctx.set_cost_model()
    N = info["N"]
    OUT = max(CM.out_estimate(info["dom_x"], float(info["out_join"]), N), 1.0)
    mhat = lambda u, v, w: 2.0 * u * v * w / K["mm_rate"] + K["mm_fixed"]
    tr = []
    d1, d2, how = CM.algorithm3(idx, N, OUT, K["T_I"], K["T_s"], K["T_m"], mhat, eps=K["eps"],
                                wcoj_factor=K["wcoj_factor"], out_join=float(info["out_join"]),
                                trace=tr)
    assert (st["delta1"], st["delta2"]) == (d1, d2), (how, tr[-3:])
    assert (st["u"], st["v"], st["w"]) == (idx.heavy_x(d2), idx.heavy_y(d1), idx.heavy_z(d2))
    if how == "mm":
        assert len(tr) >= 2


def test_default_constants_are_the_shipped_fit(ctx):
    """The library's default constants are the calibration recorded in predictor/cost_model.json
    (rounded to three significant digits)."""
    import json
    import os
    from paper_2002_12459_gb300 import calibrate
    with open(os.path.join(calibrate.PKG, "predictor", "cost_model.json")) as f:
        fit = json.load(f)["constants"]
    ctx.set_cost_model()
    K = ctx.cost_model()
    for k, v in fit.items():
        assert K[k] == pytest.approx(v, rel=5e-3, abs=1e-30), k


def test_cost_model_constants_are_checked(ctx):
    from paper_2002_12459_gb300 import jp
    with pytest.raises(jp.JPError):
        ctx.set_cost_model(eps=1.5)
    with pytest.raises(jp.JPError):
        ctx.set_cost_model(mm_rate=0.0)
    with pytest.raises(jp.JPError):
        ctx.set_cost_model(T_I=math.nan)
    ctx.set_cost_model()
    assert ctx.cost_model()["eps"] == 0.05
