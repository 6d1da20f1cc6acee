"""The learned threshold predictor's CUDA kernels against the CPU oracle.

Features are integer counts turned into fractions: compared to 1e-6.  The
network runs bfloat16 weights with float32 arithmetic; the oracle runs the
same bfloat16-rounded weights in float64, so forward values and gradients
agree to float32 accumulation error (relative 1e-4 per tensor, 3e-3 per
output value).
"""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2002_12459_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(128, 256), (256,), (256, 256), (256,), (256, 2), (2,)]


def flat(params):
    return np.concatenate([p.ravel() for p in params]).astype(np.float32)


def unflat(v):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(v[o:o + n], np.float64).reshape(s))
        o += n
    return out


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2002_12459_gb300 import build, jp
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the -m gpu tests")
    ctx = jp.Context(0)
    pred = jp.Predictor(0)
    yield torch, jp, ctx, pred
    pred.close()
    ctx.close()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def degrees(x, y):
    key = np.unique(x.astype(np.int64) * (1 << 32) + (y.astype(np.int64) & 0xFFFFFFFF))
    xs = key >> 32
    ys = key & 0xFFFFFFFF
    return np.unique(xs, return_counts=True)[1], np.unique(ys, return_counts=True)[1]


def test_features_match_oracle(env):
    torch, jp, ctx, pred = env
    rng = np.random.default_rng(0)
    x, y = W.random_small_relation(rng, 30_000, 3_000, 800, skew=1.1)
    f = ctx.features(dev(x), dev(y))
    dx, dy = degrees(x, y)
    assert np.allclose(f, M.features(dx, dy), atol=1e-6)


def test_feature_bins_at_quarter_octave_edges(env):
    torch, jp, ctx, pred = env
    # x value i has exactly degs[i] neighbours: degrees straddle bin edges
    degs = [1, 2, 3, 4, 5, 6, 7, 8, 9, 11, 13, 16, 19, 22, 23, 26, 27, 32, 38, 45, 46, 53, 54,
            64, 76, 90, 91, 107, 108, 128, 152, 181, 182, 215, 216, 256, 1000, 1024, 4096, 5000]
    xs = np.concatenate([np.full(d, i) for i, d in enumerate(degs)]).astype(np.int32)
    ys = np.concatenate([np.arange(d) for d in degs]).astype(np.int32)
    f = ctx.features(dev(xs), dev(ys))
    want = M.bin_feature(M.histogram(degs))
    assert np.allclose(f[:64], want, atol=1e-7)


def test_forward_and_gradients_match_oracle(env):
    torch, jp, ctx, pred = env
    rng = np.random.default_rng(1)
    params = M.init_params(5)
    params = [p + rng.normal(0, 0.05, p.shape) for p in params]     # non-zero biases too
    pred.set_params(flat(params))
    q = M.bf16_round(flat(params))
    P = unflat(q)
    X = rng.random((37, 128))
    T = rng.normal(size=(37, 2))
    Y = pred.forward(X)
    Yr, cache = M.forward(P, X.astype(np.float32).astype(np.float64))
    assert np.allclose(Y, Yr, rtol=3e-3, atol=3e-3 * np.abs(Yr).max())
    g, loss = pred.gradients(X, T)
    gr = M.backward(P, cache, Yr, T.astype(np.float32).astype(np.float64))
    assert abs(loss - M.mse(Yr, T)) <= 1e-4 * max(1.0, M.mse(Yr, T))
    for a, b in zip(unflat(g), gr):
        assert np.linalg.norm(a - b) <= 1e-4 * max(np.linalg.norm(b), 1e-12)
        # element by element: float32 sums of at most 256 terms against float64
        assert np.allclose(a, b, rtol=2e-3, atol=2e-5 * max(np.abs(b).max(), 1e-12))


def test_adam_step_matches_oracle(env):
    torch, jp, ctx, pred = env
    rng = np.random.default_rng(2)
    params = M.init_params(7)
    pred.set_params(flat(params))
    X = rng.random((16, 128))
    T = rng.normal(size=(16, 2))
    g, _ = pred.gradients(X, T)
    pred.set_params(flat(params))                 # reset Adam state
    pred.train_step(X, T, 1e-3)
    got = pred.get_params()
    master = [np.asarray(p, np.float32).astype(np.float64) for p in params]
    G = unflat(g)
    want, _, _ = M.adam_update(master, G, [np.zeros_like(p) for p in master],
                               [np.zeros_like(p) for p in master], 1, 1e-3)
    assert np.allclose(got, flat(want), rtol=1e-5, atol=1e-6)


def test_training_reduces_loss(env):
    torch, jp, ctx, pred = env
    rng = np.random.default_rng(3)
    X = rng.random((256, 128))
    T = np.stack([X[:, :64].sum(1) * 0.1, X[:, 64:].sum(1) * 0.05], 1)
    pred.set_params(flat(M.init_params(11)))
    first = pred.gradients(X, T)[1]
    for _ in range(300):
        last = pred.train_step(X, T, 1e-3)
    assert last < 0.05 * first


def test_learned_mode_uses_the_model(env, oracle_mod):
    torch, jp, ctx, pred = env
    params = [np.zeros(s) for s in SHAPES]
    params[5] = np.array([np.log(37.0), np.log(9.0)])          # constant prediction
    pred.set_params(flat(params))
    ctx.set_predictor(pred)
    ctx.set_threshold("learned")
    rng = np.random.default_rng(4)
    x, y = W.random_small_relation(rng, 20_000, 1_500, 400, skew=0.9)
    ox, oz = ctx.two_path(dev(x), dev(y))
    st = ctx.stats()
    b = M.bf16_round(params[5])
    want = [int(np.floor(np.exp(np.float64(np.float32(v))))) for v in b]
    # the cost model keeps the prediction (1) or overrules it with its own (2)
    assert st["learned_judged"] in (1, 2)
    wx, wz = oracle_mod.two_path(x, y)
    assert np.array_equal(ox.cpu().numpy(), wx) and np.array_equal(oz.cpu().numpy(), wz)
    ctx.set_threshold("cost_model")
    ctx.two_path(dev(x), dev(y))
    cm = ctx.stats()
    assert cm["learned_judged"] == 0
    if st["learned_judged"] == 1:
        assert (st["delta1"], st["delta2"]) == tuple(want)
    else:
        assert (st["delta1"], st["delta2"]) == (cm["delta1"], cm["delta2"])
    ctx.set_predictor(None)
    ctx.set_threshold("closed_form")


def test_cost_model_overrules_a_costly_prediction(env):
    # a constant prediction of (1, 1) makes every x of degree > 1 heavy: on this
    # relation a ~2e4-cube Boolean product, far above the cost model's choice
    torch, jp, ctx, pred = env
    params = [np.zeros(s) for s in SHAPES]
    pred.set_params(flat(params))                      # exp(0) = 1 for both
    x, y = W.powerlaw_relation(200_000, 40_000, 2.1, 20_000, 1.8, 5)
    ctx.set_threshold("cost_model")
    cx, cz = ctx.two_path(dev(x), dev(y))
    cm = ctx.stats()
    ctx.set_predictor(pred)
    ctx.set_threshold("learned")
    lx, lz = ctx.two_path(dev(x), dev(y))
    st = ctx.stats()
    assert st["learned_judged"] == 2
    assert (st["delta1"], st["delta2"]) == (cm["delta1"], cm["delta2"])
    assert torch.equal(cx, lx) and torch.equal(cz, lz)
    ctx.set_predictor(None)
    ctx.set_threshold("closed_form")
