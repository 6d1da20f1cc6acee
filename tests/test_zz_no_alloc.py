"""The allocation-free two-path entry point (jp_two_path_noalloc).

Some callers cannot allocate device memory when they query: services that
reserve their whole device-memory budget at start-up and forbid later
allocations, plug-ins inside a host program that owns every device
allocation, and latency-bound loops for which an allocation costs more than
the query.  jp_two_path_noalloc serves them from a static device scratch
array and the caller's own output buffers.  These tests call it through the
C-ABI, twice in a row, and check each result against jp_two_path on the same
input and against the CPU oracle; the result is a set of integer pairs, so the
bar is bit-exact.  This file is collected last on purpose and also passes
alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2002_12459_gb300 import workloads as W

pytestmark = pytest.mark.gpu

JP_FIXED = 0
JP_EUNSUPPORTED = -6
JP_EOVERFLOW = -4


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2002_12459_gb300 import build, jp
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the -m gpu tests")
    lib = jp.load()
    f = lib.jp_two_path_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(jp.jp_rel), ctypes.POINTER(jp.jp_rel), ctypes.c_int,
                  ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    ctx = jp.Context(0)
    yield torch, jp, f, ctx
    ctx.close()


def _noalloc(env, rx, ry, d1, d2, cap):
    torch, jp, f, _ = env
    R = jp.jp_rel(ctypes.c_void_p(rx.data_ptr()), ctypes.c_void_p(ry.data_ptr()), rx.numel())
    ox = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
    oz = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(0)
    stream = torch.cuda.current_stream().cuda_stream
    rc = f(ctypes.byref(R), None, JP_FIXED, d1, d2, ctypes.c_void_p(ox.data_ptr()),
           ctypes.c_void_p(oz.data_ptr()), cap, ctypes.byref(cnt), ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return rc, cnt.value, ox, oz


def _inputs(torch):
    # a skewed relation with heavy values (tensor-core part) and a uniform
    # one (light part only at its thresholds)
    rng = np.random.default_rng(11)
    a = W.random_small_relation(rng, 40_000, 3_000, 400, -500, 7, skew=0.9)
    b = W.uniform_relation(20_000, 2_000, 500, seed=0)
    return [(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), d1, d2)
            for (x, y), (d1, d2) in zip([a, b], [(6, 6), (141, 141)])]


def test_noalloc_matches_two_path_twice_in_a_row(env, oracle_mod):
    torch, jp, f, ctx = env
    for rx, ry, d1, d2 in _inputs(torch):
        ctx.set_threshold("fixed", d1, d2)
        wx, wz = ctx.two_path(rx, ry)
        ox_, oz_ = oracle_mod.two_path(rx.cpu().numpy(), ry.cpu().numpy())
        rc, n, ox, oz = _noalloc(env, rx, ry, d1, d2, wx.numel() + 16)
        assert rc == 0, rc
        assert n == wx.numel() == len(ox_)
        assert torch.equal(ox[:n], wx) and torch.equal(oz[:n], wz)
        assert np.array_equal(ox[:n].cpu().numpy(), ox_)
        assert np.array_equal(oz[:n].cpu().numpy(), oz_)


def test_noalloc_reports_size_when_output_too_small(env):
    torch, jp, f, ctx = env
    rx, ry, d1, d2 = _inputs(torch)[1]
    ctx.set_threshold("fixed", d1, d2)
    wx, _ = ctx.two_path(rx, ry)
    rc, n, _, _ = _noalloc(env, rx, ry, d1, d2, 10)
    assert rc == JP_EOVERFLOW and n == wx.numel()


def test_noalloc_rejects_inputs_above_its_limit(env):
    torch, jp, f, ctx = env
    n = (1 << 19) + 1
    x = torch.zeros(n, dtype=torch.int32, device="cuda")
    rc, cnt, _, _ = _noalloc(env, x, x, 1, 1, 0)
    assert rc == JP_EUNSUPPORTED and cnt == 0


def test_noalloc_query_beyond_the_array_fails_and_the_next_one_works(env, oracle_mod):
    # 160,000 tuples (below the input limit) over 4 y values: nearly every pair
    # of the 40,000 x shares a y, so the deduplicated lists alone would need
    # gigabytes of scratch.  The call must fail with JP_EUNSUPPORTED after some
    # kernels already ran, leave nothing running, and the array must serve the
    # next query correctly.
    torch, jp, f, ctx = env
    x = np.repeat(np.arange(40_000, dtype=np.int32), 4)
    y = np.tile(np.arange(4, dtype=np.int32), 40_000)
    big_x, big_y = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    rc, n, _, _ = _noalloc(env, big_x, big_y, 10 ** 6, 10 ** 6, 0)
    assert rc == JP_EUNSUPPORTED and n == 0
    rx, ry, d1, d2 = _inputs(torch)[0]
    ox_, oz_ = oracle_mod.two_path(rx.cpu().numpy(), ry.cpu().numpy())
    rc, n, ox, oz = _noalloc(env, rx, ry, d1, d2, len(ox_) + 16)
    assert rc == 0 and n == len(ox_)
    assert np.array_equal(ox[:n].cpu().numpy(), ox_)
    assert np.array_equal(oz[:n].cpu().numpy(), oz_)
