"""Failure detection without a GPU fault: a device-side wait that nothing
satisfies must end by its own time limit, report JP_ETIMEOUT through the
status word, and leave the context usable for the next query."""
import time

import numpy as np
import pytest

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


@pytest.mark.parametrize("wait_ms", [20, 100])
def test_bounded_wait_runs_out_and_the_context_stays_usable(ctx, oracle_mod, wait_ms):
    import torch
    from paper_2002_12459_gb300 import jp, workloads as W
    t0 = time.perf_counter()
    rc = ctx.selftest_wait(wait_ms * 1_000_000)
    dt = time.perf_counter() - t0
    assert rc == jp.JP_ETIMEOUT
    assert wait_ms / 1e3 <= dt < wait_ms / 1e3 + 2.0
    assert b"bounded device wait" in ctx.lib.jp_last_error(ctx.h)
    rx, ry = W.uniform_relation(5000, 500, 120, seed=9)
    ctx.set_threshold("fixed", 30, 10)
    ox, oz = ctx.two_path(torch.from_numpy(rx).cuda(), torch.from_numpy(ry).cuda())
    wx, wz = oracle_mod.two_path(rx, ry)
    assert np.array_equal(ox.cpu().numpy(), wx) and np.array_equal(oz.cpu().numpy(), wz)
    assert ctx.stats()["u"] > 0                     # the heavy product ran after the timeout


def test_selftest_rejects_bad_limits(ctx):
    from paper_2002_12459_gb300 import jp
    assert ctx.selftest_wait(0) == jp.JP_EINVAL
    assert ctx.selftest_wait(10 ** 10) == jp.JP_EINVAL
