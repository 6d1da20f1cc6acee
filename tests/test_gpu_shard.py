"""x-range shards run one after another on one GPU: each shard is the query
R_r(x,y), S(z,y) with R_r the tuples of R in rank r's x range and S all of
R; the shards' outputs, concatenated in rank order, must equal the unsharded
GPU result and the oracle (output rows are independent, Section 6)."""
import numpy as np
import pytest

from paper_2002_12459_gb300 import shard, workloads as W

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


@pytest.mark.parametrize("world,mode", [(2, "cost_model"), (4, "cost_model"), (8, "fixed")])
def test_shards_concatenate_to_unsharded(ctx, oracle_mod, world, mode):
    rx, ry = W.powerlaw_relation(60000, 12000, 2.1, 6000, 1.8, 7)
    ctx.set_threshold(mode, 6, 4)
    fx, fz = ctx.two_path(dev(rx), dev(ry))
    full = (fx.cpu().numpy(), fz.cpu().numpy())
    b = shard.x_bounds(rx, ry, world)
    gx, gz = [], []
    for r in range(world):
        px, py = shard.shard(rx, ry, r, b)
        if len(px) == 0:
            continue
        ox, oz = ctx.two_path(dev(px), dev(py), dev(rx), dev(ry))
        gx.append(ox.cpu().numpy())
        gz.append(oz.cpu().numpy())
    gx, gz = np.concatenate(gx), np.concatenate(gz)
    assert np.array_equal(gx, full[0]) and np.array_equal(gz, full[1])
    wx, wz = oracle_mod.two_path(rx, ry)
    assert np.array_equal(gx, wx) and np.array_equal(gz, wz)
