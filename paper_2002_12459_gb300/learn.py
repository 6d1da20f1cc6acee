"""Train the learned threshold predictor on thresholds the GPU method finds best.

For each seeded power-law relation (N log-uniform, x and y degree exponents
uniform in [1.2, 2.5], |dom x| = N/5, |dom y| = N/10) the two-path self-join
is timed over a grid of fixed thresholds (device time of the whole query,
best of two runs); the fastest grid point is the label (ln Delta1,
ln Delta2) and the relation's 128 degree features (jp_features) the input.
The network is trained with the library's own kernels (jp_mlp_train_step)
and evaluated on held-out relations: the query time at the predicted
thresholds is compared with the best grid time ("oracle-best threshold") and
with the time at the cost-model thresholds (Algorithm 3), which is also the
fallback when no model is set and the judge of every prediction (a
prediction whose modelled cost exceeds 3x that of Algorithm 3's choice, or
whose heavy block would not fit in half of the free device memory, is
replaced by that choice).

  python -m paper_2002_12459_gb300.learn --train 200 --test 48 --n-hi 5e6 --max-join 2e9 \
      --out params.npy --report report.json
  python -m paper_2002_12459_gb300.learn ... --eval params.npy --report report.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

D1_GRID = (8, 16, 32, 64, 128, 256, 1024)
D2_GRID = (4, 8, 16, 32, 64, 128, 512)


def relation_spec(i: int, seed: int, n_lo: float, n_hi: float):
    rng = np.random.default_rng(seed * 100003 + i)
    n = int(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))
    gx, gy = rng.uniform(1.2, 2.5, 2)
    return dict(n=n, dom_x=max(n // 5, 1), gamma_x=float(gx), dom_y=max(n // 10, 1),
                gamma_y=float(gy), seed=seed * 100003 + i)


def make_relation(spec):
    from paper_2002_12459_gb300 import workloads as W
    return W.powerlaw_relation(spec["n"], spec["dom_x"], spec["gamma_x"], spec["dom_y"],
                               spec["gamma_y"], spec["seed"])


def query_ms(ctx, dx, dy, mode, d1=1, d2=1, reps=2):
    ctx.set_threshold(mode, d1, d2)
    best = math.inf
    st = None
    for _ in range(reps):
        ox, oz = ctx.two_path(dx, dy)
        del ox, oz
        st = ctx.stats()
        best = min(best, st["ms_pass"][12])
    return best, st


def heavy_bound(x, y, d1, d2):
    """Upper bounds (u, v) of the heavy block at (d1, d2): x of degree > d2, y
    of degree > d1 (self-join, so w = u)."""
    _, cx = np.unique(x, return_counts=True)
    _, cy = np.unique(y, return_counts=True)
    return int((cx > d2).sum()), int((cy > d1).sum())


# grid points whose heavy block is beyond these bounds are not run (their time
# is taken as infinite): FP8 operands and the product's bit matrix over 16 GB,
# or a product over ~2 s
MAX_BLOCK_BYTES = 16e9
MAX_BLOCK_OPS = 4e15


def sweep(ctx, dx, dy, x, y, log=None, reps=2):
    import torch
    from paper_2002_12459_gb300 import jp
    times = {}
    for d1 in D1_GRID:
        for d2 in D2_GRID:
            u, v = heavy_bound(x, y, d1, d2)
            if 2.0 * u * v + u * u / 8.0 > MAX_BLOCK_BYTES or 2.0 * u * v * u > MAX_BLOCK_OPS:
                times[(d1, d2)] = math.inf
                continue
            try:
                times[(d1, d2)] = query_ms(ctx, dx, dy, "fixed", d1, d2, reps=reps)[0]
            except jp.JPError as e:      # out of device memory at this grid point
                times[(d1, d2)] = math.inf
                torch.cuda.empty_cache()
                if log:
                    log(f"[learn] grid point {d1},{d2}: {e}")
    return times


def join_size(x, y) -> float:
    """sum_y deg(y)^2 of the distinct tuples (the self-join's full join size)."""
    key = np.unique(x.astype(np.int64) * (1 << 32) + (y.astype(np.int64) & 0xFFFFFFFF))
    d = np.unique(key & 0xFFFFFFFF, return_counts=True)[1].astype(np.float64)
    return float((d * d).sum())


def _draw_one(args):
    """(spec, x, y) of relation i, or (spec, None, reason) when it is rejected."""
    i, seed, n_lo, n_hi, max_join = args
    spec = relation_spec(i, seed, n_lo, n_hi)
    try:
        x, y = make_relation(spec)
    except RuntimeError as e:   # the degree targets admit too few distinct tuples
        return spec, None, str(e)
    oj = join_size(x, y)
    if oj > max_join:
        return spec, None, f"full join {oj:.3g} > {max_join:.3g}"
    spec["out_join"] = oj
    return spec, x, y


def draw_specs(count, seed, n_lo, n_hi, max_join, log, workers=None):
    """The first `count` seeded relations (spec, x, y) whose full join is at
    most max_join (heavier tails give outputs beyond one GPU's memory).
    Relations are drawn by a pool of spawned processes, in index order; call
    this before the first GPU call of the process."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    out, i = [], 0
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as pool:
        while len(out) < count:
            batch = [(j, seed, n_lo, n_hi, max_join) for j in range(i, i + 2 * workers)]
            for (j, *_), (spec, x, y) in zip(batch, pool.map(_draw_one, batch)):
                if x is None:
                    log(f"[learn] skip relation {j}: {y}")
                elif len(out) < count:
                    out.append((spec, x, y))
            i += len(batch)
    return out


def stream_specs(count, seed, n_lo, n_hi, max_join, log, workers=None, first=0):
    """Like draw_specs, but yields the relations as the spawned workers produce them
    (in index order), so that drawing overlaps the GPU sweeps of earlier relations."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    done, i = 0, first
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as pool:
        while done < count:
            batch = [(j, seed, n_lo, n_hi, max_join) for j in range(i, i + 4 * workers)]
            for (j, *_), (spec, x, y) in zip(batch, pool.map(_draw_one, batch)):
                if x is None:
                    log(f"[learn] skip relation {j}: {y}")
                elif done < count:
                    done += 1
                    yield spec, x, y
            i += len(batch)


def collect(ctx, specs, log, reps=2, keep=True):
    """Features, labels (the best grid point) and per-relation rows for (spec, x, y) items.
    With keep, a row also holds the relation (host columns) for a later evaluation."""
    import torch
    feats, labels, rows = [], [], []
    for k, (spec, x, y) in enumerate(specs):
        dx = torch.from_numpy(x).cuda()
        dy = torch.from_numpy(y).cuda()
        f = ctx.features(dx, dy)
        times = sweep(ctx, dx, dy, x, y, log, reps=reps)
        (b1, b2), tbest = min(times.items(), key=lambda kv: kv[1])
        tcost, st = query_ms(ctx, dx, dy, "cost_model", reps=max(reps, 2))
        feats.append(f)
        labels.append([math.log(b1), math.log(b2)])
        grid = [[times[(d1, d2)] for d2 in D2_GRID] for d1 in D1_GRID]
        row = dict(spec=spec, best=(b1, b2), t_best=tbest, t_cost=tcost,
                   cost_delta=(st["delta1"], st["delta2"]), grid=grid)
        if keep:
            row.update(hx=x, hy=y)
        rows.append(row)
        del dx, dy
        if k % 25 == 0 or k < 5:
            log(f"[learn] {k + 1} N={spec['n']} best={b1},{b2} {tbest:.2f} ms "
                f"cost-model {tcost:.2f} ms")
    return np.array(feats, np.float32), np.array(labels, np.float32), rows


def _remake(spec):
    x, y = make_relation(spec)
    return spec, x, y


def remake_rows(rows, workers=None):
    """Regenerate the relations of saved held-out rows (their seeded specs), by spawned
    workers; call before the first GPU call of the process."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as pool:
        for r, (_, x, y) in zip(rows, pool.map(_remake, [r["spec"] for r in rows])):
            r.update(hx=x, hy=y)
    return rows


def compare(ctx, rows, arms, log):
    """Query time of each arm on each saved held-out relation (rows hold the relation and
    the grid's best time).  arms: name -> (threshold mode, cost-model constants or None,
    predictor or None).  A failed query is recorded and counted at infinity."""
    import torch
    from paper_2002_12459_gb300 import jp
    out = []
    for r in rows:
        dx, dy = torch.from_numpy(r["hx"]).cuda(), torch.from_numpy(r["hy"]).cuda()
        rec = dict(n=r["spec"]["n"], t_best=r["t_best"], best=r["best"])
        for name, (mode, consts, pred) in arms.items():
            if consts:
                ctx.set_cost_model(**consts)
            else:
                ctx.set_cost_model()
            ctx.set_predictor(pred)
            try:
                t, st = query_ms(ctx, dx, dy, mode)
                rec[name] = dict(t=t, delta=(st["delta1"], st["delta2"]),
                                 judged=st["learned_judged"])
            except jp.JPError as e:
                torch.cuda.empty_cache()
                rec[name] = dict(t=math.inf, error=str(e))
                log(f"[learn] N={r['spec']['n']} {name}: {e}")
        ctx.set_predictor(None)
        ctx.set_cost_model()
        del dx, dy
        out.append(rec)
    summary = dict(relations=len(out))
    for name in arms:
        ratio = np.array([o[name]["t"] / o["t_best"] for o in out])
        summary[name] = dict(over_best_geomean=float(np.exp(np.mean(np.log(ratio)))),
                             within_10pct=int((ratio <= 1.1).sum()),
                             total_ms=float(sum(o[name]["t"] for o in out)),
                             failed=int((~np.isfinite(ratio)).sum()))
    summary["best_total_ms"] = float(sum(o["t_best"] for o in out))
    log("[learn] " + ", ".join(f"{k} {v['over_best_geomean']:.3f}" for k, v in summary.items()
                               if isinstance(v, dict)))
    return summary, out


def init_params(seed: int = 0) -> np.ndarray:
    """He-initialised weights, zero biases, in the library's flat layout."""
    rng = np.random.default_rng(seed)
    dims = (128, 256, 256, 2)
    parts = []
    for i in range(3):
        parts.append(rng.normal(0.0, math.sqrt(2.0 / dims[i]), (dims[i], dims[i + 1])).ravel())
        parts.append(np.zeros(dims[i + 1]))
    return np.concatenate(parts).astype(np.float32)


def fit(pred, X, T, steps: int, lr: float, seed: int, log, batch: int = 1024):
    """Adam on the library's kernels; each step a seeded random mini-batch of at most
    `batch` relations (the kernels take up to JP_MLP_MAX_BATCH rows)."""
    pred.set_params(init_params(seed))
    rng = np.random.default_rng(seed + 1)
    loss = None
    for s in range(steps):
        if len(X) > batch:
            pick = rng.choice(len(X), batch, replace=False)
            loss = pred.train_step(X[pick], T[pick], lr)
        else:
            loss = pred.train_step(X, T, lr)
        if s % 500 == 0 or s == steps - 1:
            log(f"[learn] step {s}: loss {loss:.4f}")
    return loss


def evaluate(ctx, pred, rows, log):
    """Query time at the learned thresholds on each held-out relation.  A query that
    fails (out of device memory) is recorded with its error and counted at the
    cost-model time, so that one failure neither ends the run nor flatters the model."""
    import torch
    from paper_2002_12459_gb300 import jp
    ctx.set_predictor(pred)
    out = []
    for r in rows:
        dx, dy = torch.from_numpy(r["hx"]).cuda(), torch.from_numpy(r["hy"]).cuda()
        err = None
        try:
            t_learn, st = query_ms(ctx, dx, dy, "learned")
            ld, judged = (st["delta1"], st["delta2"]), st["learned_judged"]
        except jp.JPError as e:
            torch.cuda.empty_cache()
            err, t_learn, ld, judged = str(e), r["t_cost"], None, 0
            log(f"[learn] held-out N={r['spec']['n']}: {e}")
        del dx, dy
        out.append(dict(n=r["spec"]["n"], best=r["best"], t_best=r["t_best"], t_cost=r["t_cost"],
                        t_learned=t_learn, learned_delta=ld, cost_delta=r["cost_delta"],
                        overruled=judged == 2, error=err))
    ctx.set_predictor(None)
    ratio_l = [o["t_learned"] / o["t_best"] for o in out]
    ratio_c = [o["t_cost"] / o["t_best"] for o in out]
    summary = dict(relations=len(out),
                   learned_over_best_geomean=float(np.exp(np.mean(np.log(ratio_l)))),
                   cost_over_best_geomean=float(np.exp(np.mean(np.log(ratio_c)))),
                   learned_total_ms=float(sum(o["t_learned"] for o in out)),
                   cost_total_ms=float(sum(o["t_cost"] for o in out)),
                   best_total_ms=float(sum(o["t_best"] for o in out)),
                   overruled_by_cost_model=int(sum(o["overruled"] for o in out)),
                   failed=int(sum(o["error"] is not None for o in out)))
    log(f"[learn] held-out: learned/best {summary['learned_over_best_geomean']:.3f}, "
        f"cost-model/best {summary['cost_over_best_geomean']:.3f}")
    return summary, out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=160)
    ap.add_argument("--test", type=int, default=48)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--n-lo", type=float, default=1e5)
    ap.add_argument("--n-hi", type=float, default=5e5)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--max-join", type=float, default=1e9)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--reps", type=int, default=1, help="runs per grid point (the fastest is kept)")
    ap.add_argument("--out", default=None, help="write the trained float32 parameters (.npy)")
    ap.add_argument("--report", default=None, help="write a JSON report")
    ap.add_argument("--data", default=None, help="write the features and labels (.npz)")
    ap.add_argument("--budget-s", type=float, default=0.0,
                    help="stop drawing training relations after this many seconds (0: no limit)")
    ap.add_argument("--eval", default=None, metavar="PARAMS",
                    help="no training: evaluate these parameters (.npy) on the held-out relations")
    ap.add_argument("--compare", default=None, metavar="DATA",
                    help="no sweep: time the held-out relations of a --data file at Algorithm "
                         "3's default constants, at --cost-json's and at --params' predictions")
    ap.add_argument("--params", default=None, help="predictor parameters (.npy) for --compare")
    ap.add_argument("--cost-json", action="append", default=None,
                    help="cost-model constants ({'constants': ...}, e.g. calibrate.py output) for "
                         "--compare; repeatable, each an arm named after its file")
    args = ap.parse_args(argv)

    from paper_2002_12459_gb300 import build, jp
    build.build()

    def log(*a):
        print(*a, file=sys.stderr, flush=True)

    if args.compare:
        d = np.load(args.compare, allow_pickle=False)
        rows = remake_rows([json.loads(str(v)) for v in d["held"]][:args.test])
        ctx = jp.Context(0)
        arms = {"cost_default": ("cost_model", None, None)}
        for path in args.cost_json or []:
            with open(path) as f:
                name = "cost_" + os.path.splitext(os.path.basename(path))[0]
                arms[name] = ("cost_model", json.load(f)["constants"], None)
        pred = None
        if args.params:
            pred = jp.Predictor(0)
            pred.set_params(np.load(args.params))
            arms["learned"] = ("learned", None, pred)
        summary, detail = compare(ctx, rows, arms, log)
        if args.report:
            with open(args.report, "w") as f:
                json.dump(dict(summary=summary, held_out=detail), f, indent=1, default=str)
        print(json.dumps(summary))
        if pred:
            pred.close()
        ctx.close()
        return

    t0 = time.time()
    # the relations are drawn by spawned workers while the GPU sweeps earlier ones; the
    # held-out relations are the ones after the training relations in the same draw
    stream = stream_specs(args.train + args.test, args.seed, args.n_lo, args.n_hi,
                          args.max_join, log)
    ctx = jp.Context(0)
    pred = jp.Predictor(0)
    if args.eval:
        import itertools
        X, T, rows = collect(ctx, itertools.islice(stream, args.test), log, reps=args.reps)
        pred.set_params(np.load(args.eval))
        summary, detail = evaluate(ctx, pred, rows, log)
        summary.update(train_relations=args.train, evaluated=os.path.basename(args.eval),
                       seconds=time.time() - t0, grid=[list(D1_GRID), list(D2_GRID)])
    else:
        import itertools
        # held-out relations first (the first args.test of the draw), then training
        # relations until args.train or the time budget
        Xte, Tte, rows = collect(ctx, itertools.islice(stream, args.test), log, reps=args.reps)
        budget = args.budget_s

        def until_budget(it):
            for item in it:
                if budget and time.time() - t0 > budget:
                    log(f"[learn] time budget reached")
                    return
                yield item
        Xtr, Ttr, trows = collect(ctx, until_budget(stream), log, reps=args.reps, keep=False)
        log(f"[learn] {len(Xtr)} training and {len(Xte)} held-out relations swept in "
            f"{time.time() - t0:.0f} s")
        if args.data:            # kept before fitting: the sweeps are the expensive part
            def meta(rs):
                return np.array([json.dumps({k: v for k, v in r.items() if k not in ("hx", "hy")},
                                            default=str) for r in rs])
            np.savez(args.data, Xtr=Xtr, Ttr=Ttr, Xte=Xte, Tte=Tte, held=meta(rows),
                     train=meta(trows), d1_grid=np.array(D1_GRID), d2_grid=np.array(D2_GRID))
        loss = fit(pred, Xtr, Ttr, args.steps, args.lr, args.seed, log)
        summary, detail = evaluate(ctx, pred, rows, log)
        summary.update(train_relations=len(Xtr), final_train_loss=loss, reps_per_point=args.reps,
                       n_range=[args.n_lo, args.n_hi], max_join=args.max_join,
                       seconds=time.time() - t0, grid=[list(D1_GRID), list(D2_GRID)])
    if args.out:
        np.save(args.out, pred.get_params())
    if args.report:
        with open(args.report, "w") as f:
            json.dump(dict(summary=summary, held_out=detail), f, indent=1, default=str)
    print(json.dumps(summary))
    pred.close()
    ctx.close()


if __name__ == "__main__":
    main()
