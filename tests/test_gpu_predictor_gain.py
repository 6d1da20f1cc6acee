"""What learning from measured threshold sweeps gains over the method's hand-set constants.

Held-out relations (drawn with a seed the training never used, same recipe:
power-law x and y degrees, exponents uniform in [1.2, 2.5]) are run four
ways on the GPU: at every point of the threshold grid (the fastest is the
best-threshold time); with Algorithm 3 at the library's default constants
(fitted to the measured sweeps of 789 relations, predictor/cost_model.json);
with Algorithm 3 at the constants measured on the 10M relation alone (the
method without the fit); and at the shipped network's predicted thresholds
(JP_LEARNED).  All give the same tuples.  On the 256 held-out relations of
predictor/report.json the fitted constants reach 1.007x the best-grid time,
the single-relation constants 1.109x and the network 1.10x; here, on six
small relations where timing noise is larger, the fitted constants must stay
within 1.15x of the best and not lose to the single-relation constants, and
the network within 1.2x.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SINGLE = dict(T_I=1.0 / 60e9, T_m=1e-12, T_s=0.0, mm_rate=2.2e15, mm_fixed=2e-5)


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2002_12459_gb300 import build, jp, learn
    # relations first (spawned workers), before this process uses the GPU
    specs = learn.draw_specs(6, seed=7, n_lo=1e5, n_hi=6e5, max_join=3e8, log=lambda *a: None,
                             workers=4)
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the -m gpu tests")
    ctx = jp.Context(0)
    pred = jp.Predictor.trained(0)
    yield ctx, pred, specs, learn
    ctx.set_predictor(None)
    ctx.set_cost_model()
    pred.close()
    ctx.close()


def test_fitted_constants_and_learned_thresholds_against_best(env):
    import torch
    ctx, pred, specs, learn = env
    rows = []
    for spec, x, y in specs:
        dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ctx.set_predictor(None)
        ctx.set_cost_model()
        ctx.set_threshold("cost_model")
        cx, cz = ctx.two_path(dx, dy)
        t_fit = learn.query_ms(ctx, dx, dy, "cost_model", reps=3)[0]
        ctx.set_cost_model(**SINGLE)
        t_single = learn.query_ms(ctx, dx, dy, "cost_model", reps=3)[0]
        ctx.set_cost_model()
        ctx.set_predictor(pred)
        ctx.set_threshold("learned")
        lx, lz = ctx.two_path(dx, dy)
        st = ctx.stats()
        assert st["threshold_mode"] == 3
        assert torch.equal(cx, lx) and torch.equal(cz, lz)
        t_learn = learn.query_ms(ctx, dx, dy, "learned", reps=3)[0]
        ctx.set_predictor(None)
        times = learn.sweep(ctx, dx, dy, x, y)
        t_best = min(times.values())
        assert math.isfinite(t_best)
        rows.append((spec["n"], t_best, t_fit, t_single, t_learn))
        del cx, cz, lx, lz

    def g(i):
        return float(np.exp(np.mean([np.log(r[i] / r[1]) for r in rows])))

    g_fit, g_single, g_learn = g(2), g(3), g(4)
    for r in rows:
        print(f"N={r[0]} best {r[1]:.3f} ms  fitted {r[2]:.3f}  single-relation {r[3]:.3f}  "
              f"learned {r[4]:.3f}")
    print(f"over best: fitted {g_fit:.3f}  single-relation {g_single:.3f}  learned {g_learn:.3f}")
    assert g_fit <= 1.15, (g_fit, g_single, g_learn)
    assert g_fit <= g_single + 0.02, (g_fit, g_single)
    assert g_learn <= 1.2, (g_learn, g_fit)
