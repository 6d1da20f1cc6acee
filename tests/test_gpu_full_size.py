"""Full-size parity in the launch configuration bench.py times.

The 10M-tuple power-law two-path query (2.9e9 output pairs) and the
3 x 2M star query (1.25e10 output triples) are too large for the oracle as a
whole, so sampled outputs are checked exactly: whole rows of random and hub
x values against the oracle's per-row form, one x1 range of the star against
the oracle restricted to that range, plus properties that hold at any size
(strict lexicographic order, every x on its own diagonal for a self-join).
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


def test_two_path_powerlaw_10m_sampled_rows(ctx, oracle_mod):
    import torch
    rx, ry = W.make("two_path_powerlaw_10m")
    ctx.set_threshold("cost_model")
    ox, oz = ctx.two_path(torch.from_numpy(rx).cuda(), torch.from_numpy(ry).cuda())
    n = ox.numel()
    st = ctx.stats()
    assert n == st["out_count"] and st["u"] > 0 and st["light_candidates"] > 0
    # strictly increasing (x, z): sorted and distinct
    dx = ox[1:] - ox[:-1]
    assert bool((dx >= 0).all())
    same = dx == 0
    assert bool((oz[1:][same] > oz[:-1][same]).all())
    del dx, same
    # self-join: every x value is paired with itself
    ux = np.unique(rx)
    assert int((ox == oz).sum()) == len(ux)
    # whole rows: random x values and the ten largest-degree x
    srt = oracle_mod.SortedS(rx, ry)
    vals, cnts = np.unique(rx, return_counts=True)
    rng = np.random.default_rng(5)
    sample = list(rng.choice(vals, 40, replace=False)) + list(vals[np.argsort(-cnts)[:10]])
    q = torch.tensor(sorted(sample), dtype=torch.int32, device="cuda")
    lo = torch.searchsorted(ox, q, right=False).cpu().numpy()
    hi = torch.searchsorted(ox, q, right=True).cpu().numpy()
    for a, s, e in zip(sorted(sample), lo, hi):
        want = oracle_mod.two_path_row(ry[rx == a], srt)
        got = oz[int(s):int(e)].cpu().numpy()
        assert np.array_equal(got, want), int(a)
    del ox, oz


def test_star3_2m_sampled_range(ctx, oracle_mod):
    import torch
    rels = W.make("star3_2m")
    ctx.set_threshold("cost_model")
    cols = ctx.star([(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()) for x, y in rels])
    assert cols[0].numel() == ctx.stats()["out_count"] > 1e10
    x1 = np.unique(rels[0][0])
    for lo, hi in [(int(x1[5]), int(x1[12])), (int(x1[-9]), int(x1[-1]))]:
        want = oracle_mod.star(rels, x_lo=lo, x_hi=hi)
        b = torch.searchsorted(cols[0], torch.tensor([lo, hi + 1], dtype=torch.int32, device="cuda"))
        s, e = int(b[0]), int(b[1])
        assert e - s == len(want[0])
        for c, w in zip(cols, want):
            assert np.array_equal(c[s:e].cpu().numpy(), w)
    del cols
