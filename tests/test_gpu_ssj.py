"""Witness counts and the set similarity join (jp_two_path_counts).

Every (x, z, count) must equal the oracle's element by element: relations
from tiny to several tiles of the heavy product, self-joins and distinct S,
thresholds that make everything heavy (counts only from the tensor cores),
everything light (counts only from the sorted candidates), mixed and the cost
model's; c_min of 1 and above; both orders; the light candidates cut into
many ranges (and a row larger than a range); degenerate inputs; and on the
benchmark's 10M-tuple relation, whole rows of an x range.
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


def run(ctx, R, S=None, c_min=1, order="pairs"):
    sz, sy = (dev(S[0]), dev(S[1])) if S is not None else (None, None)
    cols = ctx.two_path_counts(dev(R[0]), dev(R[1]), sz, sy, c_min=c_min, order=order)
    return tuple(c.cpu().numpy() for c in cols)


def check(ctx, oracle_mod, R, S=None, c_min=1, order="pairs"):
    got = run(ctx, R, S, c_min, order)
    sz, sy = S if S is not None else (None, None)
    want = oracle_mod.ssj(R[0], R[1], c_min, sz, sy, order=order)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    return len(want[0])


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("mode,d", [("fixed", 1), ("fixed", 10 ** 6), ("fixed", 3), ("cost_model", 1)])
def test_counts_random_relations(ctx, oracle_mod, seed, mode, d):
    rng = np.random.default_rng(seed)
    R = W.random_small_relation(rng, 5000, 600, 250, offset_x=-200, offset_y=-50, skew=0.8)
    S = None if seed % 2 == 0 else W.random_small_relation(rng, 4000, 700, 250, offset_x=-100,
                                                           offset_y=-50, skew=0.6)
    ctx.set_threshold(mode, d, d)
    for c_min, order in [(1, "pairs"), (2, "count"), (5, "pairs")]:
        n = check(ctx, oracle_mod, R, S, c_min, order)
        st = ctx.stats()
        assert n > 0 and st["out_count"] == n
        if c_min == 1:      # every pair has a light or a heavy witness, or both
            lp, hp = st["count_light_pairs"], st["heavy_pairs"]
            assert max(lp, hp) <= n <= lp + hp
    if mode == "fixed" and d == 1:
        assert ctx.stats()["u"] > 0


def test_counts_in_many_ranges(ctx, oracle_mod):
    rng = np.random.default_rng(11)
    R = W.random_small_relation(rng, 6000, 500, 300, skew=0.9)
    ctx.set_threshold("fixed", 6, 6)
    try:
        for chunk in (1, 997, 50_000):       # 1: every range is one x (rows larger than a range)
            ctx.set_count_chunk(chunk)
            check(ctx, oracle_mod, R, None, 2, "count")
            check(ctx, oracle_mod, R, None, 1, "pairs")
    finally:
        ctx.set_count_chunk(1 << 27)


@pytest.mark.parametrize("seed", range(2))
def test_counts_powerlaw_several_tiles(ctx, oracle_mod, seed):
    R = W.make("two_path_powerlaw_1m", n=300_000, dom_x=60_000, dom_y=30_000, seed=seed)
    ctx.set_threshold("fixed", 8, 8)
    check(ctx, oracle_mod, R, None, 3, "count")
    st = ctx.stats()
    assert st["u"] > 256 and st["w"] > 256
    ctx.set_threshold("cost_model")
    check(ctx, oracle_mod, R, None, 1, "pairs")


def test_counts_degenerate_cases(ctx, oracle_mod):
    ctx.set_threshold("cost_model")
    e = np.empty(0, np.int32)
    assert len(run(ctx, (e, e))[0]) == 0
    rng = np.random.default_rng(5)
    R = W.random_small_relation(rng, 300, 40, 30, offset_x=-20)
    assert len(run(ctx, R, None, 10 ** 6)[0]) == 0
    # R and S share no y
    S = (np.array([1, 2], np.int32), np.array([10 ** 6, 10 ** 6 + 1], np.int32))
    assert len(run(ctx, R, S)[0]) == 0
    big = np.iinfo(np.int32)
    lim = np.array([big.min, big.max, 0, big.min, -1, big.max], np.int32)
    R2 = (lim, np.array([0, 0, 0, big.max, big.max, big.min], np.int32))
    check(ctx, oracle_mod, R2, None, 1, "count")
    check(ctx, oracle_mod, R2, (lim[::-1].copy(), R2[1]), 1, "pairs")
    # one set containing every y: its count with each set is that set's size
    x = np.concatenate([np.zeros(50, np.int32), rng.integers(1, 30, 200).astype(np.int32)])
    y = np.concatenate([np.arange(50, dtype=np.int32), rng.integers(0, 50, 200).astype(np.int32)])
    ctx.set_threshold("fixed", 4, 4)
    check(ctx, oracle_mod, (x, y), None, 1, "count")


def test_counts_on_the_10m_relation(ctx, oracle_mod):
    import torch
    rx, ry = W.make("two_path_powerlaw_10m")
    ctx.set_threshold("cost_model")
    ox, oz, oc = ctx.two_path_counts(dev(rx), dev(ry), c_min=3)
    st = ctx.stats()
    assert st["u"] > 0 and ox.numel() == st["out_count"]
    # whole rows of one x range, including the x of largest degree
    vals, cnts = np.unique(rx, return_counts=True)
    hub = int(vals[np.argmax(cnts)])
    for lo, hi in [(hub, hub), (1000, 1400)]:
        wx, wz, wc = oracle_mod.two_path(rx, ry, x_lo=lo, x_hi=hi, with_counts=True)
        keep = wc >= 3
        s = int(torch.searchsorted(ox, torch.tensor([lo], dtype=torch.int32, device="cuda")))
        e = int(torch.searchsorted(ox, torch.tensor([hi], dtype=torch.int32, device="cuda"), right=True))
        assert np.array_equal(ox[s:e].cpu().numpy(), wx[keep])
        assert np.array_equal(oz[s:e].cpu().numpy(), wz[keep])
        assert np.array_equal(oc[s:e].cpu().numpy(), wc[keep])
    assert bool((ox[1:] >= ox[:-1]).all())
    del ox, oz, oc
    torch.cuda.empty_cache()


def test_counts_from_host_columns(ctx, oracle_mod):
    import torch
    rng = np.random.default_rng(9)
    R = W.random_small_relation(rng, 3000, 300, 150, skew=0.7)
    ctx.set_threshold("cost_model")
    pin = [torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for v in R]
    got = ctx.two_path_counts(*pin, c_min=2, order="count")
    want = oracle_mod.ssj(R[0], R[1], 2, order="count")
    for g, w in zip(got, want):
        assert np.array_equal(g.cpu().numpy(), w)
