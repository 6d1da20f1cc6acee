"""Boolean set intersection requests answered in batches (Section 3.3).

Requests Q_ab() = R(a,y), S(b,y) -- do the sets of a and b intersect? --
arrive as a Poisson process at rate B against one resident relation (here a
self-join, S = R); a and b are drawn with probability proportional to their
degree (large sets are asked about more often) or uniformly.  A server collects them into batches: the C pairs of a
batch form the relation T(x,z), and one jp_two_path_filter call answers
Q_batch(x,z) = R(x,y), S(z,y), T(x,z) on the GPU.  A request's latency runs
from its arrival to the end of its batch's call.

Batching policies:

  fixed C   a batch is the C oldest waiting requests, started once C have
            arrived (or the trace has ended) and the GPU is free;
  greedy    whenever the GPU is free, every waiting request (up to a cap).

The paper sizes the batch from its cost model: C queries cost N * C^(1/3)
time units, so the mean latency C/B + N / C^(2/3) is least near
C = (B N)^(3/5) (Proposition 4, omega = 2).  ``prop4_batch`` evaluates that
rule with the time unit calibrated on the GPU (kappa seconds per tuple, fitted
to measured batch times t(C) = kappa N C^(1/3)), and ``best_batch`` picks C
from the measured times directly: the least modelled latency
(C - 1) / (2B) + t(C) among batch sizes that keep up (t(C) <= C / B).

  python -m paper_2002_12459_gb300.bsi_serve --rate 1000 --requests 5000 --out bsi.json
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np


def arrivals(count, rate, seed):
    """Poisson arrival times (seconds from the start of the trace)."""
    rng = np.random.default_rng(seed + 91)
    return np.cumsum(rng.exponential(1.0 / rate, count))


class WallClock:
    def __init__(self):
        self.t0 = time.perf_counter()

    def now(self):
        return time.perf_counter() - self.t0

    def sleep_until(self, t):
        d = t - self.now()
        if d > 0:
            time.sleep(min(d, 0.01))


def run_trace(times, policy, answer, clock, cap=1 << 20):
    """Serve requests arriving at ``times`` (sorted) with a batching policy.

    ``policy`` is ``("fixed", C)`` or ``("greedy",)``; ``answer(lo, hi)``
    answers requests lo..hi-1 (consecutive in arrival order) and returns when
    their results are ready.  Returns per-request latency, the batch sizes
    and the time the server was busy.
    """
    n = len(times)
    lat = np.zeros(n)
    sizes = []
    busy = 0.0
    head = 0                       # oldest request not yet answered
    while head < n:
        now = clock.now()
        arrived = int(np.searchsorted(times, now, side="right"))
        if policy[0] == "fixed":
            want = min(int(policy[1]), n - head)
            if arrived - head < want:
                clock.sleep_until(times[head + want - 1])
                continue
            hi = head + want
        else:
            if arrived <= head:
                clock.sleep_until(times[head])
                continue
            hi = min(arrived, head + cap)
        t0 = clock.now()
        answer(head, hi)
        t1 = clock.now()
        busy += t1 - t0
        lat[head:hi] = t1 - times[head:hi]
        sizes.append(hi - head)
        head = hi
    return lat, np.array(sizes), busy


def best_batch(rate, sizes, seconds):
    """Batch size of least modelled mean latency (C - 1) / (2 B) + t(C) that keeps up."""
    best = None
    for c, t in zip(sizes, seconds):
        if t > c / rate:
            continue
        m = (c - 1) / (2 * rate) + t
        if best is None or m < best[1]:
            best = (int(c), m)
    return best[0] if best else int(max(sizes))


def fit_kappa(n_tuples, sizes, seconds):
    """Least-squares kappa of t(C) = kappa N C^(1/3) (the Section 3.3 batch cost)."""
    f = n_tuples * np.cbrt(np.asarray(sizes, np.float64))
    t = np.asarray(seconds, np.float64)
    return float((f * t).sum() / (f * f).sum())


def prop4_batch(rate, n_tuples, kappa):
    """Proposition 4's C = (B N)^(3/5), with time measured in units of kappa seconds."""
    return (rate * kappa * n_tuples) ** 0.6


def summary(lat, sizes, busy, span):
    return {"requests": int(len(lat)), "batches": int(len(sizes)),
            "mean_batch": float(sizes.mean()) if len(sizes) else 0.0,
            "mean_ms": float(lat.mean() * 1e3), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "span_s": float(span),
            "gpu_busy_frac": float(busy / span) if span > 0 else 0.0,
            "requests_per_s": float(len(lat) / span) if span > 0 else 0.0}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="two_path_powerlaw_10m")
    ap.add_argument("--requests", type=int, default=5000)
    ap.add_argument("--rate", type=float, nargs="+", default=[1000.0])
    ap.add_argument("--batches", type=int, nargs="+", default=[1, 10, 30, 100, 300, 1000, 3000])
    ap.add_argument("--absent", type=float, default=0.02)
    ap.add_argument("--draw", default="degree", choices=["degree", "uniform"],
                    help="request values drawn proportionally to their degree, or uniformly")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)

    def log(*a):
        print(*a, file=sys.stderr, flush=True)

    import torch
    from paper_2002_12459_gb300 import build, jp
    from paper_2002_12459_gb300 import workloads as W
    rx, ry = W.make(args.workload)
    vals, deg = np.unique(rx, return_counts=True)
    w = deg if args.draw == "degree" else None
    tx, tz = W.candidate_pairs(vals, vals, args.requests, seed=args.seed + 1, absent=args.absent,
                               x_weights=w, z_weights=w)
    build.build()
    ctx = jp.Context(0)
    ctx.set_threshold("cost_model")
    R = (torch.from_numpy(rx).cuda(), torch.from_numpy(ry).cuda())
    T = (torch.from_numpy(tx).cuda(), torch.from_numpy(tz).cuda())   # received requests
    answered = [0]

    def answer(lo, hi):
        ox, oz = ctx.two_path_filter(T[0][lo:hi], T[1][lo:hi], *R)
        torch.cuda.synchronize()
        answered[0] += ox.numel()        # distinct pairs of the batch whose sets intersect

    # the batch cost t(C), measured on the first requests
    ctx.two_path_filter(T[0][:8], T[1][:8], *R)
    ladder, secs = [], []
    for c in args.batches:
        c = min(c, args.requests)
        reps = 5 if c <= 1000 else 2
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in range(reps):
            lo = (r * c) % max(1, args.requests - c)
            answer(lo, lo + c)
        ladder.append(c)
        secs.append((time.perf_counter() - t0) / reps)
        log(f"[bsi] t({c}) = {secs[-1] * 1e3:.2f} ms")
    kappa = fit_kappa(len(rx), ladder, secs)
    result = {"config": {"workload": args.workload, "relation_tuples": int(len(rx)),
                         "requests": args.requests, "absent_fraction": args.absent,
                         "request_values": args.draw,
                         "seed": args.seed, "threshold_mode": "cost_model"},
              "batch_cost": {"sizes": ladder, "ms": [s * 1e3 for s in secs],
                             "kappa_s_per_tuple": kappa},
              "runs": []}
    for rate in args.rate:
        times = arrivals(args.requests, rate, args.seed)
        chosen = best_batch(rate, ladder, secs)
        p4 = prop4_batch(rate, len(rx), kappa)
        run = {"rate_per_s": rate, "best_batch": chosen, "prop4_batch": p4, "policies": {}}
        policies = [("fixed", c) for c in sorted(set(ladder + [chosen]))
                    if c * 4 <= args.requests] + [("greedy",)]
        for pol in policies:
            name = "greedy" if pol[0] == "greedy" else f"fixed_{pol[1]}"
            # skip fixed sizes that cannot keep up (their queue grows without bound)
            if pol[0] == "fixed":
                i = ladder.index(pol[1]) if pol[1] in ladder else None
                if i is not None and secs[i] > 1.5 * pol[1] / rate:
                    run["policies"][name] = {"skipped": "t(C) > 1.5 C / B: the queue grows"}
                    continue
            clock = WallClock()
            answered[0] = 0
            lat, sizes, busy = run_trace(times, pol, answer, clock)
            run["policies"][name] = summary(lat, sizes, busy, clock.now())
            run["policies"][name]["answered_yes"] = answered[0]
            s = run["policies"][name]
            log(f"[bsi] rate {rate}/s {name}: mean {s['mean_ms']:.2f} ms, p99 {s['p99_ms']:.2f} ms, "
                f"{s['batches']} batches, busy {s['gpu_busy_frac']:.2f}")
        result["runs"].append(run)
    ctx.close()
    print(json.dumps(result))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(result, f, indent=1)


if __name__ == "__main__":
    main()
