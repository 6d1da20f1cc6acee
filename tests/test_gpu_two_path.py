"""Parity of the CUDA two-path path (through the C-ABI) with the CPU oracle.

The result is a set of integer pairs, so the bar is bit-exact equality of
the sorted distinct pairs and of their count.  Inputs are seeded and
synthetic; thresholds are swept because Algorithm 1's output must not depend
on them (the correctness argument after Algorithm 1).
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


def run(ctx, rx, ry, sz=None, sy=None, mode="fixed", d1=1, d2=1):
    ctx.set_threshold(mode, d1, d2)
    if sz is None:
        ox, oz = ctx.two_path(dev(rx), dev(ry))
    else:
        ox, oz = ctx.two_path(dev(rx), dev(ry), dev(sz), dev(sy))
    return ox.cpu().numpy(), oz.cpu().numpy()


def assert_same(got, want):
    gx, gz = got
    wx, wz = want
    assert len(gx) == len(wx), (len(gx), len(wx))
    assert np.array_equal(gx, wx)
    assert np.array_equal(gz, wz)


def rand_rel(rng, n, dx, dy, ox=0, oy=0, skew=0.0):
    return W.random_small_relation(rng, n, dx, dy, ox, oy, skew)


@pytest.mark.parametrize("seed", range(8))
def test_small_self_join_threshold_sweep(ctx, oracle_mod, seed):
    rng = np.random.default_rng(seed)
    rx, ry = rand_rel(rng, 3000, 400, 150, -200, -70, skew=0.8)
    want = oracle_mod.two_path(rx, ry)
    for d1, d2 in [(1, 1), (2, 2), (3, 7), (10, 3), (25, 25), (10 ** 6, 10 ** 6), (1, 10 ** 6),
                   (10 ** 6, 1)]:
        assert_same(run(ctx, rx, ry, d1=d1, d2=d2), want)


@pytest.mark.parametrize("seed", range(6))
def test_small_two_relations(ctx, oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    rx, ry = rand_rel(rng, 2500, 300, 120, 5, -60, skew=0.7)
    sz, sy = rand_rel(rng, 1800, 250, 150, -1000, -60, skew=0.5)
    want = oracle_mod.two_path(rx, ry, sz, sy)
    for d1, d2 in [(1, 1), (2, 5), (8, 8), (10 ** 6, 10 ** 6)]:
        assert_same(run(ctx, rx, ry, sz, sy, d1=d1, d2=d2), want)


def test_uniform_20k_fixed_sqrt_threshold(ctx, oracle_mod):
    rx, ry = W.make("two_path_uniform_20k")
    want = oracle_mod.two_path(rx, ry)
    assert_same(run(ctx, rx, ry, d1=141, d2=141), want)
    st = ctx.stats()
    assert st["delta1"] == 141 and st["u"] == 0          # every x degree <= 23: all light
    assert st["out_count"] == len(want[0])


def test_uniform_20k_all_heavy(ctx, oracle_mod):
    # thresholds 1: every x (degree >= 2) and y (degree >= 25) is heavy,
    # so the answer comes from the tensor-core product alone
    rx, ry = W.make("two_path_uniform_20k")
    want = oracle_mod.two_path(rx, ry)
    assert_same(run(ctx, rx, ry, d1=1, d2=1), want)
    st = ctx.stats()
    assert st["u"] == 2000 and st["v"] == 500 and st["light_candidates"] == 0


@pytest.mark.parametrize("mode", ["closed_form", "cost_model"])
def test_uniform_20k_model_thresholds(ctx, oracle_mod, mode):
    rx, ry = W.make("two_path_uniform_20k")
    want = oracle_mod.two_path(rx, ry)
    assert_same(run(ctx, rx, ry, mode=mode), want)


def test_complete_bipartite(ctx):
    a, b = 700, 300
    xs, ys = np.meshgrid(np.arange(a), np.arange(b), indexing="ij")
    for d in (1, 100, 10 ** 6):
        ox, oz = run(ctx, xs.ravel(), ys.ravel(), d1=d, d2=d)
        assert len(ox) == a * a
        assert np.array_equal(ox, np.repeat(np.arange(a), a))
        assert np.array_equal(oz, np.tile(np.arange(a), a))


def test_star_graph_and_duplicates(ctx):
    d = 5000
    xs = (np.arange(d) * 7 - 20000).astype(np.int32)
    ys = np.full(d, -3, np.int32)
    xs2 = np.concatenate([xs, xs[:100]])                  # duplicate tuples
    ys2 = np.concatenate([ys, ys[:100]])
    ox, oz = run(ctx, xs2, ys2, d1=10 ** 6, d2=10 ** 6)
    assert len(ox) == d * d
    srt = np.sort(xs)
    assert np.array_equal(ox, np.repeat(srt, d)) and np.array_equal(oz, np.tile(srt, d))


def test_empty_and_single(ctx):
    e = np.empty(0, np.int32)
    ox, oz = run(ctx, e, e)
    assert len(ox) == 0
    ox, oz = run(ctx, np.array([5], np.int32), np.array([-9], np.int32))
    assert ox.tolist() == [5] and oz.tolist() == [5]
    # disjoint y: R and S share no y value
    ox, oz = run(ctx, np.array([1, 2], np.int32), np.array([3, 4], np.int32),
                 np.array([7], np.int32), np.array([5], np.int32))
    assert len(ox) == 0


def test_extreme_values(ctx, oracle_mod):
    big = np.iinfo(np.int32)
    rx = np.array([big.min, big.max, 0, big.min, -1, big.max], np.int32)
    ry = np.array([big.max, big.max, big.min, big.min, big.max, 0], np.int32)
    want = oracle_mod.two_path(rx, ry)
    for d in (1, 1000):
        assert_same(run(ctx, rx, ry, d1=d, d2=d), want)


def test_bitmap_window_wider_than_shared_memory(ctx, oracle_mod):
    # 2.1M distinct x values (z domain > one 1.835M-bit window) and a few
    # heavy x whose candidates span both windows
    n = 2_100_000
    base = np.arange(n, dtype=np.int32)
    rx = np.concatenate([base, np.full(3, -1, np.int32), np.full(3, -2, np.int32)])
    ry = np.concatenate([base % 700_000, np.array([0, 1, 699_999, 5, 6, 7], np.int32)])
    ox, oz = run(ctx, rx, ry, d1=10 ** 6, d2=2)
    st = ctx.stats()
    assert st["u"] == 2
    # rows of the heavy x and a sample of light x against the per-row oracle
    srt = oracle_mod.SortedS(rx, ry)
    starts = np.searchsorted(ox, [-2, -1, 0, 12345, 2_000_001], side="left")
    ends = np.searchsorted(ox, [-2, -1, 0, 12345, 2_000_001], side="right")
    for a, s, e in zip([-2, -1, 0, 12345, 2_000_001], starts, ends):
        want = oracle_mod.two_path_row(ry[rx == a], srt)
        assert np.array_equal(oz[s:e], want)
    # each base x shares its y with two others (3 pairs); the 18 base x on the
    # six special y gain the special x; each special x reaches 3 * 3 + 1 z
    assert len(ox) == 3 * n + 18 + 2 * 10


def _class_relation(seed):
    """x rows whose candidate counts span every light class: y values of
    degree 20..400, x rows of 1..300 neighbour lists (c from a few to ~70k;
    rows of 128 lists or more take the bitmap kernel's hub path)."""
    rng = np.random.default_rng(seed)
    ny = 400
    ydeg = rng.integers(20, 400, ny)
    xs, ys = [], []
    nx = 3000
    for a in range(nx):
        d = int(rng.choice([1, 2, 3, 6, 12, 20, 40, 64, 70, 150, 300], p=[.1] * 9 + [.05] * 2))
        ys.append(rng.choice(ny, min(d, ny), replace=False, p=ydeg / ydeg.sum()))
        xs.append(np.full(len(ys[-1]), a))
    low = np.argsort(ydeg)[:60]          # rows of 2-3 small lists: c <= 256
    for a in range(nx, nx + 200):
        ys.append(rng.choice(low, int(rng.integers(2, 4)), replace=False))
        xs.append(np.full(len(ys[-1]), a))
    nx += 200
    # 100 further y of small degree and 20 rows of 66-70 of them: more than 64
    # lists with c <= 2048 (the warp bucket class)
    small = np.arange(ny, ny + 100)
    for a in range(nx, nx + 20):
        ys.append(rng.choice(small, int(rng.integers(66, 71)), replace=False))
        xs.append(np.full(len(ys[-1]), a))
    nx += 20
    for k, b in enumerate(small):        # five more tuples on each
        ys.append(np.full(5, b))
        xs.append(nx + 5 * k + np.arange(5))
    nx += 5 * len(small)
    ydeg = np.concatenate([ydeg, np.zeros(len(small), ydeg.dtype)])
    rx = np.concatenate(xs).astype(np.int32)
    ry = np.concatenate(ys).astype(np.int32)
    # top up every y to its degree with extra x values (they are light rows too)
    have = np.bincount(ry, minlength=len(ydeg))
    extra_y = np.repeat(np.arange(len(ydeg)), np.maximum(ydeg - have, 0))
    extra_x = nx + np.arange(len(extra_y))
    rx = np.concatenate([rx, extra_x]).astype(np.int64)
    # x -> x * 2654435761 + 12345 (mod 2^32, as int32) is one-to-one: values spread
    # over the whole signed range, in an order unrelated to the draw order
    rx = ((rx * 2654435761 + 12345) & 0xFFFFFFFF).astype(np.uint32).view(np.int32)
    return rx, np.concatenate([ry, extra_y.astype(np.int32)])


@pytest.mark.parametrize("seed", range(2))
def test_every_light_class(ctx, oracle_mod, seed):
    rx, ry = _class_relation(seed)
    want = oracle_mod.two_path(rx, ry)
    # all light: the warp, bucket, copy, bitmap, three merge and the hub classes are used
    assert_same(run(ctx, rx, ry, d1=10 ** 6, d2=10 ** 6), want)
    st = ctx.stats()
    assert all(st["light_x"][q] > 0 for q in range(8)), st["light_x"]
    # heavy x and heavy y mixed in
    for d1, d2 in [(200, 30), (60, 8), (350, 65)]:
        assert_same(run(ctx, rx, ry, d1=d1, d2=d2), want)


def test_two_path_into_device_and_pinned_host_columns(ctx, oracle_mod):
    # jp_two_path_into writes the sorted distinct pairs into caller-owned columns: device
    # tensors, or pinned host tensors written by the output kernel over the host link
    import torch
    from paper_2002_12459_gb300 import jp
    rng = np.random.default_rng(77)
    rx, ry = rand_rel(rng, 5000, 500, 120, -300, 11, skew=0.8)
    sz, sy = rand_rel(rng, 4000, 400, 130, 50, 0, skew=0.5)
    for S in (None, (sz, sy)):
        want = oracle_mod.two_path(rx, ry) if S is None else oracle_mod.two_path(rx, ry, sz, sy)
        n = len(want[0])
        for d1, d2 in [(1, 1), (4, 6), (10 ** 6, 10 ** 6)]:
            ctx.set_threshold("fixed", d1, d2)
            args = () if S is None else (dev(sz), dev(sy))
            ox = torch.full((n + 5,), -7, dtype=torch.int32, device="cuda")
            oz = torch.full((n + 5,), -7, dtype=torch.int32, device="cuda")
            assert ctx.two_path_into(dev(rx), dev(ry), ox, oz, *args) == n
            assert np.array_equal(ox[:n].cpu().numpy(), want[0])
            assert np.array_equal(oz[:n].cpu().numpy(), want[1])
            assert int(ox[n]) == -7                                # nothing past the result
            hx = torch.zeros(n, dtype=torch.int32, pin_memory=True)
            hz = torch.zeros(n, dtype=torch.int32, pin_memory=True)
            hrx = torch.from_numpy(np.ascontiguousarray(rx, np.int32)).pin_memory()
            hry = torch.from_numpy(np.ascontiguousarray(ry, np.int32)).pin_memory()
            hargs = () if S is None else (torch.from_numpy(sz.astype(np.int32)),
                                          torch.from_numpy(sy.astype(np.int32)))
            assert ctx.two_path_into(hrx, hry, hx, hz, *hargs) == n
            assert np.array_equal(hx.numpy(), want[0]) and np.array_equal(hz.numpy(), want[1])
    # buffers one pair short: JP_EOVERFLOW, the needed size reported, nothing written
    ctx.set_threshold("fixed", 4, 6)
    want = oracle_mod.two_path(rx, ry)
    n = len(want[0])
    ox = torch.full((n - 1,), -7, dtype=torch.int32, device="cuda")
    oz = torch.full((n - 1,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(jp.JPError, match="EOVERFLOW") as ei:
        ctx.two_path_into(dev(rx), dev(ry), ox, oz)
    assert ei.value.count == n
    assert bool((ox == -7).all()) and bool((oz == -7).all())


@pytest.mark.parametrize("width", [128, 256])
def test_product_tile_widths(ctx, oracle_mod, width):
    # both tile widths of the tcgen05 product give the oracle's answer: an all-heavy
    # query (the product alone), a mixed one, R != S, and a batch (per-tile K ranges)
    rng = np.random.default_rng(width)
    rx, ry = W.make("two_path_uniform_20k")
    sx, sy = rand_rel(rng, 6000, 900, 140, -400, 3, skew=0.6)
    saved = ctx.gemm_tile()
    ctx.set_gemm_tile(width, 0)
    try:
        assert_same(run(ctx, rx, ry, d1=1, d2=1), oracle_mod.two_path(rx, ry))
        assert ctx.stats()["gemm_tile"] == width
        assert_same(run(ctx, sx, sy, d1=3, d2=4), oracle_mod.two_path(sx, sy))
        assert_same(run(ctx, sx, sy, rx[:7000], ry[:7000], d1=2, d2=2),
                    oracle_mod.two_path(sx, sy, rx[:7000], ry[:7000]))
        rels = [rand_rel(rng, n, 300, 60, 0, 0, skew=0.5) for n in (2500, 800, 4000)]
        x = np.concatenate([a for a, _ in rels])
        y = np.concatenate([b for _, b in rels])
        qoff = np.concatenate([[0], np.cumsum([len(a) for a, _ in rels])]).astype(np.int64)
        ctx.set_threshold("fixed", 2, 2)
        ox, oz, off = ctx.two_path_batch(dev(x), dev(y), qoff)
        ox, oz = ox.cpu().numpy(), oz.cpu().numpy()
        for q, (a, b) in enumerate(rels):
            wx, wz = oracle_mod.two_path(a, b)
            assert np.array_equal(ox[off[q]:off[q + 1]], wx) and np.array_equal(oz[off[q]:off[q + 1]], wz)
    finally:
        ctx.set_gemm_tile(*saved)


def test_auto_tile_follows_the_crossover(ctx):
    rx, ry = W.make("two_path_uniform_20k")
    saved = ctx.gemm_tile()
    try:
        ctx.set_gemm_tile(0, 10 ** 6)          # every product is "small": narrow tiles
        run(ctx, rx, ry, d1=1, d2=1)
        assert ctx.stats()["gemm_tile"] == 128
        ctx.set_gemm_tile(0, 0)                # none is: wide tiles
        run(ctx, rx, ry, d1=1, d2=1)
        assert ctx.stats()["gemm_tile"] == 256
    finally:
        ctx.set_gemm_tile(*saved)
