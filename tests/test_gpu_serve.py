"""Serving a mixed trace of two-path and star k = 3 requests (batched and one at a time):
every request's answer equals the CPU oracle's, bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def reqs():
    from paper_2002_12459_gb300 import serve
    # drawn by spawned workers before this process touches the GPU
    return serve.make_requests(36, seed=3, n_lo=200, n_hi=2e4, star_n_hi=4e3, star_frac=0.4,
                               max_join=5e6, max_star=2e6, workers=4)


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


@pytest.mark.parametrize("mode", ["batched", "single"])
def test_every_request_matches_the_oracle(ctx, reqs, oracle_mod, mode):
    from paper_2002_12459_gb300 import serve
    ctx.set_threshold("cost_model")
    times = serve.arrivals(len(reqs), 5000.0, 3)    # requests queue up: batches form
    keep = {}
    lat, outs, busy, span, calls = serve.serve(ctx, reqs, times, mode, keep=keep)
    assert len(keep) == len(reqs)
    if mode == "batched":
        assert calls < len(reqs)                      # some requests shared a call
    for i, r in enumerate(reqs):
        want = oracle_mod.two_path(r["x"], r["y"]) if r["kind"] == "two_path" else oracle_mod.star(r["rels"])
        got = keep[i]
        assert outs[i] == len(want[0]), i
        for g, w in zip(got, want):
            assert np.array_equal(g, w), (i, r["kind"])
    s = serve.summary(lat, outs, busy, span, calls, reqs)
    assert s["p99_ms"] >= s["p50_ms"] > 0
