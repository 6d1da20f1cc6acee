"""Tile autotuner for the heavy product (the tcgen05 Boolean matrix product).

The product kernel computes one tile of 128 heavy x by W heavy z per CTA, W =
128 or 256.  Wide tiles read B once per 256 columns (less traffic per MMA);
narrow tiles give twice as many CTAs, which matters when a product has too few
wide tiles to occupy the GPU's SMs (small queries, serving batches).

The tuner times both widths through the C-ABI on products of many shapes and
writes the crossover: the largest number of 128 x 256 tiles up to which the
narrow tile was at least as fast, its times summed over the measured K sizes of
each tile count (crossover()).  Each product is made all
heavy on purpose: a seeded random bipartite relation over u x values and v y
values in which every value has degree >= 2, queried at fixed thresholds
Delta1 = Delta2 = 1, so the heavy block is exactly u x v x u; the product's
device time is the query's jp_stats.ms_pass[4].

  python -m paper_2002_12459_gb300.tune [--out paper_2002_12459_gb300/predictor/gemm_tiles.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(PKG, "predictor", "gemm_tiles.json")

U_GRID = (256, 512, 1024, 2048, 4096, 8192, 16384)
V_GRID = (512, 2048, 8192)


def dense_relation(u: int, v: int, seed: int):
    """Seeded (x, y) pairs over [0, u) x [0, v) in which every x and every y has degree >= 2.

    Every x gets two y and every y two x by construction (so all values are heavy at
    thresholds 1); then random pairs fill the relation to about max(4 (u + v), u v / 16).
    """
    rng = np.random.default_rng(seed)
    ax, ay = np.arange(u), np.arange(v)
    xs = [ax, ax, ay % u, (ay + 1) % u]                # x a: y a and a + 1 (mod v) ...
    ys = [ax % v, (ax + 1) % v, ay, ay]                # ... y b: x b and b + 1 (mod u)
    m = max(4 * (u + v), (u * v) // 16)
    xs.append(rng.integers(0, u, m))
    ys.append(rng.integers(0, v, m))
    return (np.concatenate(xs).astype(np.int32), np.concatenate(ys).astype(np.int32))


def product_ms(ctx, dx, dy, width, reps=3):
    """Best-of-reps device ms of the product (jp_stats.ms_pass[4]) at one tile width."""
    ctx.set_gemm_tile(width, 0)
    best = None
    for _ in range(reps + 1):
        ox, oz = ctx.two_path(dx, dy)
        st = ctx.stats()
        del ox, oz
        if st["gemm_tile"] != width:
            raise RuntimeError(f"asked for width {width}, the product used {st['gemm_tile']}")
        ms = st["ms_pass"][4]
        best = ms if best is None else min(best, ms)
    return best, st


def tune(u_grid=U_GRID, v_grid=V_GRID, log=None):
    import torch
    from paper_2002_12459_gb300 import build, jp
    build.build()
    ctx = jp.Context(0)
    ctx.set_threshold("fixed", 1, 1)
    rows = []
    try:
        for u in u_grid:
            for v in v_grid:
                x, y = dense_relation(u, v, seed=u * 7919 + v)
                dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
                ms128, st = product_ms(ctx, dx, dy, 128)
                ms256, _ = product_ms(ctx, dx, dy, 256)
                assert st["u"] == u and st["v"] == v, (st["u"], st["v"], u, v)
                wide = -(-u // 128) * -(-u // 256)
                rows.append({"u": u, "v": v, "w": u, "wide_tiles": wide, "ms_128": ms128,
                             "ms_256": ms256, "faster": 128 if ms128 < ms256 else 256})
                if log:
                    log(f"[tune] u=w={u} v={v}: {wide} wide tiles, 128: {ms128:.4f} ms, "
                        f"256: {ms256:.4f} ms")
                del dx, dy
    finally:
        ctx.close()
    return {"measurements": rows, "auto_max_tiles": crossover(rows)}


def crossover(rows):
    """Largest wide-tile count T such that, for every tile count up to T, the narrow tile's
    time summed over the measured K sizes is at most the wide tile's (0: the wide tile
    always wins).  Sums over K damp the noise of microsecond products."""
    by = {}
    for r in rows:
        a = by.setdefault(r["wide_tiles"], [0.0, 0.0])
        a[0] += r["ms_128"]
        a[1] += r["ms_256"]
    best = 0
    for t in sorted(by):
        if by[t][0] <= by[t][1]:
            best = t
        else:
            break
    return best


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args(argv)
    res = tune(log=lambda *a: print(*a, file=sys.stderr, flush=True))
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps({"auto_max_tiles": res["auto_max_tiles"]}))


if __name__ == "__main__":
    main()
