"""Batches of boolean set intersection queries (jp_two_path_filter, Section 3.3).

The GPU answer must equal the oracle's three-way join element by element:
relations from tiny to several tiles of the heavy product, self-joins and
distinct S, thresholds that make everything heavy, everything light and the
cost model's choice, candidate sets with repeats, absent values, extreme
int32 values and no hits at all, host and device columns; and on the
power-law relation of the benchmark (10M tuples) a candidate set the oracle
answers pair by pair.
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
    torch.cuda.empty_cache()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def run(ctx, R, T, S=None):
    sz, sy = (dev(S[0]), dev(S[1])) if S is not None else (None, None)
    ox, oz = ctx.two_path_filter(dev(T[0]), dev(T[1]), dev(R[0]), dev(R[1]), sz, sy)
    return ox.cpu().numpy(), oz.cpu().numpy()


def check(ctx, oracle_mod, R, T, S=None):
    got = run(ctx, R, T, S)
    sz, sy = S if S is not None else (None, None)
    want = oracle_mod.bsi(R[0], R[1], T[0], T[1], sz, sy)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    return len(want[0])


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("mode,d", [("fixed", 1), ("fixed", 10 ** 6), ("fixed", 3), ("cost_model", 1)])
def test_bsi_random_relations(ctx, oracle_mod, seed, mode, d):
    rng = np.random.default_rng(seed)
    R = W.random_small_relation(rng, 6000, 700, 300, offset_x=-200, offset_y=-50, skew=0.8)
    S = None if seed % 2 == 0 else W.random_small_relation(rng, 5000, 900, 300, offset_x=-100,
                                                           offset_y=-50, skew=0.6)
    zs = np.unique(R[0] if S is None else S[0])
    T = W.candidate_pairs(np.unique(R[0]), zs, 20000, seed=seed, absent=0.1)
    ctx.set_threshold(mode, d, d)
    hits = check(ctx, oracle_mod, R, T, S)
    st = ctx.stats()
    assert st["out_count"] == hits and hits > 0
    assert st["filter_pairs"] == len(np.unique((T[0].astype(np.int64) << 32) | (T[1].astype(np.int64) & 0xFFFFFFFF)))
    if mode == "fixed" and d == 1:
        assert st["u"] > 0                   # the heavy product ran on the reduced relations


@pytest.mark.parametrize("seed", range(2))
def test_bsi_powerlaw_several_tiles(ctx, oracle_mod, seed):
    R = W.make("two_path_powerlaw_1m", n=300_000, dom_x=60_000, dom_y=30_000, seed=seed)
    ux = np.unique(R[0])
    T = W.candidate_pairs(ux, ux, 200_000, seed=10 + seed, absent=0.05)
    ctx.set_threshold("fixed", 8, 8)
    check(ctx, oracle_mod, R, T)
    st = ctx.stats()
    assert st["u"] > 256 and st["w"] > 256       # more than one tile of the product each way
    ctx.set_threshold("cost_model")
    check(ctx, oracle_mod, R, T)


def test_bsi_degenerate_cases(ctx, oracle_mod):
    ctx.set_threshold("cost_model")
    rng = np.random.default_rng(3)
    R = W.random_small_relation(rng, 500, 60, 40, offset_x=-30)
    e = (np.empty(0, np.int32), np.empty(0, np.int32))
    assert len(run(ctx, R, e)[0]) == 0                                         # empty T
    assert len(run(ctx, e, (np.array([1], np.int32), np.array([2], np.int32)))[0]) == 0  # empty R
    # T disjoint from the domains: the reduced relations are empty
    far = (np.full(5, 10 ** 6, np.int32), np.arange(5, dtype=np.int32))
    assert len(run(ctx, R, far)[0]) == 0
    # one pair repeated many times
    a = int(R[0][0])
    T = (np.full(1000, a, np.int32), np.full(1000, a, np.int32))
    assert check(ctx, oracle_mod, R, T) == 1
    # extreme values
    lim = np.array([-(1 << 31), (1 << 31) - 1, 0], np.int32)
    R2 = (np.concatenate([R[0], lim]), np.concatenate([R[1], np.zeros(3, np.int32)]))
    T2 = (np.concatenate([lim, lim, R[0][:50]]), np.concatenate([lim[::-1], lim, R[0][50:100]]))
    check(ctx, oracle_mod, R2, T2)
    # every pair of the domains: the answer is the two-path query itself
    ux = np.unique(R[0])
    a, b = np.meshgrid(ux, ux, indexing="ij")
    got = run(ctx, R, (a.ravel().astype(np.int32), b.ravel().astype(np.int32)))
    want = oracle_mod.two_path(R[0], R[1])
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_bsi_from_host_columns(ctx, oracle_mod):
    import torch
    rng = np.random.default_rng(9)
    R = W.random_small_relation(rng, 4000, 400, 200, skew=0.7)
    T = W.candidate_pairs(np.unique(R[0]), np.unique(R[0]), 5000, seed=9)
    ctx.set_threshold("cost_model")
    pin = [torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for v in (*T, *R)]
    ox, oz = ctx.two_path_filter(*pin)
    want = oracle_mod.bsi(R[0], R[1], T[0], T[1])
    assert np.array_equal(ox.cpu().numpy(), want[0]) and np.array_equal(oz.cpu().numpy(), want[1])


def test_bsi_on_the_10m_relation(ctx, oracle_mod):
    import torch
    rx, ry = W.make("two_path_powerlaw_10m")
    vals, cnts = np.unique(rx, return_counts=True)
    # uniform candidates plus pairs of hub values (rows of the heavy product)
    T = W.candidate_pairs(vals, vals, 100_000, seed=4, absent=0.02)
    hubs = vals[np.argsort(-cnts)[:32]]
    ha, hb = np.meshgrid(hubs, hubs, indexing="ij")
    T = (np.concatenate([T[0], ha.ravel()]).astype(np.int32),
         np.concatenate([T[1], hb.ravel()]).astype(np.int32))
    ctx.set_threshold("cost_model")
    ox, oz = ctx.two_path_filter(dev(T[0]), dev(T[1]), dev(rx), dev(ry))
    want = oracle_mod.bsi(rx, ry, T[0], T[1])
    assert np.array_equal(ox.cpu().numpy(), want[0]) and np.array_equal(oz.cpu().numpy(), want[1])
    assert len(want[0]) > 500
    del ox, oz
    torch.cuda.empty_cache()
