"""Serving many join-project queries: arrivals, dynamic batching, latency.

A stream of requests -- two-path self-joins Q(x,z) = R(x,y), R(z,y) and
star queries Q*_3 -- arrives as a Poisson process at a stated rate.  Two
servers answer the same trace on one GPU:

  batched   whenever the GPU is free, every two-path request that has
            arrived and waits is answered by one jp_two_path_batch call (the
            whole batch in one pass of the pipeline, each pass one launch),
            and every waiting star request by one jp_star_batch call;
  single    one request at a time, in arrival order.

A request is received when it arrives: its columns are copied to the
device then.  Its latency runs from arrival to the moment its result (the
sorted distinct tuples, in device memory) and their count are ready.
Reported: p50 / p99 / mean latency, requests/s and distinct tuples/s over
the trace's span, and GPU busy time.

Relations follow the power-law recipe of the other workloads: N log-uniform
in [n_lo, n_hi] (star relations capped at star_n_hi), degree exponents
uniform in [g_lo, g_hi], |dom x| = N/5, |dom y| = N/10 for two-path; for the
star, x uniform over N/4 values and one y degree sequence over N/10 values.
Requests whose full join is above a cap are redrawn (their outputs would
not fit a serving memory budget).

  python -m paper_2002_12459_gb300.serve --requests 1000 --rate 100 400 --out serve.json
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np


def _request(args):
    i, seed, n_lo, n_hi, star_n_hi, g_lo, g_hi, star_frac, max_join, max_star = args
    from paper_2002_12459_gb300 import workloads as W
    rng = np.random.default_rng(seed * 1000003 + i)
    star = bool(rng.random() < star_frac)
    for attempt in range(32):
        hi = min(n_hi, star_n_hi) if star else n_hi
        n = int(math.exp(rng.uniform(math.log(n_lo), math.log(hi))))
        g1, g2 = (float(v) for v in rng.uniform(g_lo, g_hi, 2))
        s = int(rng.integers(1 << 30))
        try:
            if star:
                rels = W.star_relations(3, n, max(n // 4, 1), max(n // 10, 1), g1, s)
                d = np.bincount(rels[0][1] - rels[0][1].min()).astype(np.float64)
                size = float((d ** 3).sum())
                if size <= max_star:
                    return dict(i=i, kind="star", n=n, rels=rels, join=size)
            else:
                x, y = W.powerlaw_relation(n, max(n // 5, 1), g1, max(n // 10, 1), g2, s)
                d = np.bincount(y - y.min()).astype(np.float64)
                size = float((d ** 2).sum())
                if size <= max_join:
                    return dict(i=i, kind="two_path", n=n, x=x, y=y, join=size)
        except RuntimeError:
            pass
    raise RuntimeError(f"request {i}: no relation within the caps")


def make_requests(count, seed, n_lo=1e3, n_hi=2e6, star_n_hi=2e5, g_lo=1.3, g_hi=2.2,
                  star_frac=0.2, max_join=5e8, max_star=2e8, workers=None):
    """Seeded requests, drawn by spawned workers (call before the GPU is used)."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    jobs = [(i, seed, n_lo, n_hi, star_n_hi, g_lo, g_hi, star_frac, max_join, max_star)
            for i in range(count)]
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as pool:
        return list(pool.map(_request, jobs, chunksize=4))


def arrivals(count, rate, seed):
    """Poisson arrival times (seconds from the start of the trace)."""
    rng = np.random.default_rng(seed + 77)
    return np.cumsum(rng.exponential(1.0 / rate, count))


class _Clock:
    def __init__(self):
        self.t0 = time.perf_counter()

    def now(self):
        return time.perf_counter() - self.t0


def _receive(req, torch):
    """Copy a request's columns to the device (done when it arrives)."""
    if req["kind"] == "two_path":
        req["dx"] = torch.from_numpy(req["x"]).cuda()
        req["dy"] = torch.from_numpy(req["y"]).cuda()
    else:
        req["drels"] = [(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
                        for x, y in req["rels"]]


def serve(ctx, reqs, times, mode, max_batch_tuples=3e7, log=None, keep=None):
    """Run the trace; returns per-request latency (s), output tuples and GPU busy time.

    With ``keep`` (a dict), every request's answer is stored there as numpy columns.
    """
    import torch
    clock = _Clock()
    n = len(reqs)
    lat = np.zeros(n)
    outs = np.zeros(n, np.int64)
    nxt = 0            # next request not yet received
    waiting = []       # received, not answered
    busy = 0.0
    batches = 0
    done = 0

    def kept(i, cols):
        if keep is not None:
            keep[i] = tuple(c.cpu().numpy() for c in cols)

    while done < n:
        now = clock.now()
        while nxt < n and times[nxt] <= now:
            _receive(reqs[nxt], torch)
            waiting.append(nxt)
            nxt += 1
        if not waiting:
            time.sleep(max(0.0, min(times[nxt] - clock.now(), 0.01)))
            continue
        t_start = clock.now()
        if mode == "single":
            group = [waiting.pop(0)]
        else:
            group = []
            for kind, size in (("two_path", 1), ("star", 3)):
                total = 0
                for i in list(waiting):
                    if reqs[i]["kind"] != kind:
                        continue
                    if group and total + size * reqs[i]["n"] > max_batch_tuples:
                        break
                    group.append(i)
                    total += size * reqs[i]["n"]
            for i in group:
                waiting.remove(i)
        two = [i for i in group if reqs[i]["kind"] == "two_path"]
        stars = [i for i in group if reqs[i]["kind"] == "star"]
        if mode == "batched" and len(two) > 1:
            xs = torch.cat([reqs[i]["dx"] for i in two])
            ys = torch.cat([reqs[i]["dy"] for i in two])
            qoff = np.zeros(len(two) + 1, np.int64)
            qoff[1:] = np.cumsum([reqs[i]["n"] for i in two])
            ox, oz, off = ctx.two_path_batch(xs, ys, qoff)
            torch.cuda.synchronize()
            t_end = clock.now()
            for k, i in enumerate(two):
                outs[i] = off[k + 1] - off[k]
                lat[i] = t_end - times[i]
                kept(i, (ox[off[k]:off[k + 1]], oz[off[k]:off[k + 1]]))
            del ox, oz, xs, ys
            batches += 1
        else:
            for i in two:
                ox, oz = ctx.two_path(reqs[i]["dx"], reqs[i]["dy"])
                torch.cuda.synchronize()
                outs[i] = ox.numel()
                lat[i] = clock.now() - times[i]
                kept(i, (ox, oz))
                del ox, oz
                batches += 1
        if mode == "batched" and len(stars) > 1:
            c0, c1, c2, off = ctx.star_batch([reqs[i]["drels"] for i in stars])
            torch.cuda.synchronize()
            t_end = clock.now()
            for k, i in enumerate(stars):
                outs[i] = off[k + 1] - off[k]
                lat[i] = t_end - times[i]
                kept(i, tuple(c[off[k]:off[k + 1]] for c in (c0, c1, c2)))
            del c0, c1, c2
            batches += 1
        else:
            for i in stars:
                cols = ctx.star(reqs[i]["drels"])
                torch.cuda.synchronize()
                outs[i] = cols[0].numel()
                lat[i] = clock.now() - times[i]
                kept(i, cols)
                del cols
                batches += 1
        for i in group:
            for key in ("dx", "dy", "drels"):
                reqs[i].pop(key, None)
        busy += clock.now() - t_start
        done += len(group)
        if log and done % 200 < len(group):
            log(f"[serve] {mode}: {done}/{n} answered, t = {clock.now():.2f} s")
    span = clock.now()
    return lat, outs, busy, span, batches


def summary(lat, outs, busy, span, batches, reqs):
    two = np.array([r["kind"] == "two_path" for r in reqs])
    return {"requests": len(lat), "calls": batches,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3),
            "p50_ms_two_path": float(np.percentile(lat[two], 50) * 1e3) if two.any() else None,
            "p99_ms_two_path": float(np.percentile(lat[two], 99) * 1e3) if two.any() else None,
            "p50_ms_star": float(np.percentile(lat[~two], 50) * 1e3) if (~two).any() else None,
            "p99_ms_star": float(np.percentile(lat[~two], 99) * 1e3) if (~two).any() else None,
            "span_s": span, "gpu_busy_s": busy, "requests_per_s": len(lat) / span,
            "tuples_per_s": float(outs.sum() / span), "output_tuples": int(outs.sum())}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--rate", type=float, nargs="+", default=[100.0],
                    help="Poisson arrival rates, requests/s (the same requests at every rate)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--star-frac", type=float, default=0.2)
    ap.add_argument("--mode", default="cost_model", choices=["fixed", "closed_form", "cost_model"])
    ap.add_argument("--max-batch-tuples", type=float, default=3e7)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)

    def log(*a):
        print(*a, file=sys.stderr, flush=True)

    t0 = time.time()
    reqs = make_requests(args.requests, args.seed, star_frac=args.star_frac)
    log(f"[serve] {len(reqs)} requests drawn in {time.time() - t0:.1f} s")
    import torch
    from paper_2002_12459_gb300 import build, jp
    build.build()
    ctx = jp.Context(0)
    ctx.set_threshold(args.mode)
    # warm-up: one small query of each kind
    w = next(r for r in reqs if r["kind"] == "two_path")
    ctx.two_path(torch.from_numpy(w["x"]).cuda(), torch.from_numpy(w["y"]).cuda())
    result = {"config": {"requests": args.requests, "rates_per_s": args.rate, "seed": args.seed,
                         "star_fraction": args.star_frac, "threshold_mode": args.mode,
                         "n_range": [1e3, 2e6], "star_n_max": 2e5, "gamma_range": [1.3, 2.2],
                         "max_batch_tuples": args.max_batch_tuples,
                         "input_tuples": int(sum(r["n"] * (3 if r["kind"] == "star" else 1)
                                                 for r in reqs))}}
    result["runs"] = []
    for rate in args.rate:
        times = arrivals(args.requests, rate, args.seed)
        run = {"rate_per_s": rate, "trace_s": float(times[-1])}
        for mode in ("batched", "single"):
            lat, outs, busy, span, calls = serve(ctx, reqs, times, mode, args.max_batch_tuples, log)
            run[mode] = summary(lat, outs, busy, span, calls, reqs)
            log(f"[serve] rate {rate}/s {mode}: p50 {run[mode]['p50_ms']:.2f} ms, "
                f"p99 {run[mode]['p99_ms']:.2f} ms, {run[mode]['tuples_per_s']:.3g} tuples/s, "
                f"{calls} calls")
            if mode == "batched":
                first = outs.copy()
            else:
                assert np.array_equal(first, outs), "batched and single answers differ in size"
        result["runs"].append(run)
    ctx.close()
    print(json.dumps(result))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(result, f, indent=1)


if __name__ == "__main__":
    main()
