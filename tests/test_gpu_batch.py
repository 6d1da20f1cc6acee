"""Batches of two-path self-joins in one pipeline pass (jp_two_path_batch).

Every query of a batch must come out exactly as the oracle answers it alone:
the queries share values on purpose (a small common domain), so a pair
mixing two queries, or a lost tagging, shows up as a wrong slice.  Batches
mix empty, single-tuple and skewed relations, and run at thresholds that
make everything heavy (one product over the union's heavy block), everything
light, and the cost model's choice.
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


def mixed_batch(seed, nq=40):
    rng = np.random.default_rng(seed)
    rels = []
    for q in range(nq):
        kind = q % 8
        if kind == 0:
            n = 0
        elif kind == 1:
            n = 1
        else:
            n = int(rng.integers(2, 3000))
        x = rng.integers(-60, 200, n).astype(np.int32)           # a domain shared by all queries
        y = (rng.zipf(1.6, n) % 90 - 20).astype(np.int32)
        if kind == 7 and n:                                       # duplicates and a hub
            x[: n // 2] = 5
        rels.append((x, y))
    return rels


def concat(rels):
    qoff = np.zeros(len(rels) + 1, np.int64)
    qoff[1:] = np.cumsum([len(x) for x, _ in rels])
    x = np.concatenate([x for x, _ in rels]).astype(np.int32)
    y = np.concatenate([y for _, y in rels]).astype(np.int32)
    return x, y, qoff


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("mode,d", [("fixed", 1), ("fixed", 10 ** 6), ("fixed", 4), ("cost_model", 1)])
def test_batch_equals_each_query_alone(ctx, oracle_mod, seed, mode, d):
    rels = mixed_batch(seed)
    x, y, qoff = concat(rels)
    ctx.set_threshold(mode, d, d)
    ox, oz, off = ctx.two_path_batch(dev(x), dev(y), qoff)
    st = ctx.stats()
    ox, oz = ox.cpu().numpy(), oz.cpu().numpy()
    assert off[0] == 0 and off[-1] == len(ox) == st["out_count"]
    if mode == "fixed" and d == 1:
        assert st["u"] > 0                   # the union's heavy product ran
    for q, (rx, ry) in enumerate(rels):
        wx, wz = oracle_mod.two_path(rx, ry)
        s, e = off[q], off[q + 1]
        assert np.array_equal(ox[s:e], wx) and np.array_equal(oz[s:e], wz), q


def test_batch_from_host_columns_and_single_query(ctx, oracle_mod):
    import torch
    rels = mixed_batch(11, nq=9)
    x, y, qoff = concat(rels)
    ctx.set_threshold("cost_model")
    hx = torch.from_numpy(x).pin_memory()
    hy = torch.from_numpy(y).pin_memory()
    ox, oz, off = ctx.two_path_batch(hx, hy, qoff)
    ox, oz = ox.cpu().numpy(), oz.cpu().numpy()
    for q, (rx, ry) in enumerate(rels):
        wx, wz = oracle_mod.two_path(rx, ry)
        assert np.array_equal(ox[off[q]:off[q + 1]], wx) and np.array_equal(oz[off[q]:off[q + 1]], wz)
    # a batch of one query is that query
    rx, ry = rels[3]
    bx, bz, off1 = ctx.two_path_batch(dev(rx), dev(ry), np.array([0, len(rx)]))
    gx, gz = ctx.two_path(dev(rx), dev(ry))
    assert off1.tolist() == [0, gx.numel()]
    assert torch.equal(bx, gx) and torch.equal(bz, gz)


def _oracle_all(rels):
    # the largest relations take ~20 s each in the oracle: run them in
    # processes started with spawn (never fork a process that holds a CUDA
    # context)
    import multiprocessing as mp
    import oracle
    with mp.get_context("spawn").Pool(min(len(rels), 8)) as pool:
        return pool.starmap(oracle.two_path, rels)


def test_power_law_batch_against_oracle(ctx, oracle_mod):
    # uneven sizes, 1e3 to 2e5 tuples, with heavy hubs: every slice of the
    # batch equals the oracle's answer for that query alone, and the query
    # run alone on the GPU at the same thresholds
    import torch
    rng = np.random.default_rng(3)
    rels = []
    for q in range(12):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(2e5))))
        rels.append(W.powerlaw_relation(n, max(n // 5, 1), float(rng.uniform(1.3, 2.2)),
                                        max(n // 10, 1), float(rng.uniform(1.3, 2.2)), 100 + q))
    want = _oracle_all(rels)
    x, y, qoff = concat(rels)
    for d1, d2 in [(16, 8), (200, 40)]:
        ctx.set_threshold("fixed", d1, d2)
        ox, oz, off = ctx.two_path_batch(dev(x), dev(y), qoff)
        hx, hz = ox.cpu().numpy(), oz.cpu().numpy()
        for q, (rx, ry) in enumerate(rels):
            wx, wz = want[q]
            assert off[q + 1] - off[q] == len(wx), q
            assert np.array_equal(hx[off[q]:off[q + 1]], wx), q
            assert np.array_equal(hz[off[q]:off[q + 1]], wz), q
            if q % 4 == 0:
                gx, gz = ctx.two_path(dev(rx), dev(ry))
                assert torch.equal(ox[off[q]:off[q + 1]], gx), q


def test_bad_offsets_are_rejected(ctx):
    from paper_2002_12459_gb300 import jp
    x = dev(np.arange(10))
    with pytest.raises(jp.JPError, match="EINVAL"):
        ctx.two_path_batch(x, x, np.array([0, 5, 3, 10]))
    with pytest.raises(jp.JPError, match="EINVAL"):
        ctx.two_path_batch(x, x, np.array([0, 9]))


def _star_queries(seed, count):
    rng = np.random.default_rng(seed)
    qs = []
    for q in range(count):
        n = int(rng.integers(50, 4000))
        dy = int(rng.integers(5, 120))
        rels = []
        for i in range(3):
            m = 0 if (q == 2 and i == 1) else n + int(rng.integers(-40, 40))   # one query has an empty relation
            x = rng.integers(-300, 300, max(m, 0)).astype(np.int32)
            y = (rng.integers(0, dy, max(m, 0)) - dy // 2).astype(np.int32)
            rels.append((x, y))
        qs.append(rels)
    return qs


_STAR_WANTS = {}


def _star_wants(oracle_mod, seed, qs):
    if seed not in _STAR_WANTS:
        _STAR_WANTS[seed] = [oracle_mod.star(rels) if all(len(r[0]) for r in rels)
                             else tuple(np.empty(0, np.int32) for _ in range(3)) for rels in qs]
    return _STAR_WANTS[seed]


@pytest.mark.parametrize("mode,d1,d2", [("fixed", 1, 1), ("fixed", 4, 3), ("fixed", 10 ** 6, 10 ** 6),
                                        ("cost_model", 1, 1)])
def test_star_batch_against_oracle(ctx, oracle_mod, mode, d1, d2):
    # every slice of the batch equals the oracle's answer for that query alone; the
    # queries' values overlap, so a witness shared across queries would show up
    qs = _star_queries(31, 9)
    wants = _star_wants(oracle_mod, 31, qs)
    ctx.set_threshold(mode, d1, d2)
    c0, c1, c2, off = ctx.star_batch([[(dev(x), dev(y)) for x, y in q] for q in qs])
    g = [c.cpu().numpy() for c in (c0, c1, c2)]
    assert off[0] == 0 and off[-1] == len(g[0])
    for q, rels in enumerate(qs):
        want = wants[q]
        assert off[q + 1] - off[q] == len(want[0]), q
        for i in range(3):
            assert np.array_equal(g[i][off[q]:off[q + 1]], want[i]), (q, i)


def test_star_batch_of_one_is_the_star_query(ctx, oracle_mod):
    import torch
    qs = _star_queries(5, 1)
    ctx.set_threshold("fixed", 3, 2)
    c = ctx.star_batch([[(dev(x), dev(y)) for x, y in qs[0]]])
    s = ctx.star([(dev(x), dev(y)) for x, y in qs[0]])
    assert c[3].tolist() == [0, s[0].numel()]
    for i in range(3):
        assert torch.equal(c[i], s[i])


def test_star_batch_bad_offsets_are_rejected(ctx):
    from paper_2002_12459_gb300 import jp
    import ctypes
    x = dev(np.arange(10))
    rels = (jp.jp_rel * 3)(*[jp._rel_of(x, x) for _ in range(3)])
    qoff = np.array([[0, 5, 3, 10]] * 3, np.int64)
    out_off = np.zeros(4, np.int64)
    res = jp.jp_result()
    i64p = ctypes.POINTER(ctypes.c_int64)
    rc = ctx.lib.jp_star_batch(ctx.h, 3, rels, qoff.ctypes.data_as(i64p), ctypes.byref(res),
                               out_off.ctypes.data_as(i64p))
    assert rc == jp.JP_EINVAL
