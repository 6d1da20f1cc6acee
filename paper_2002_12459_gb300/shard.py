"""x-range sharding of the two-path query across ranks (host-side logic).

Output rows of Q(x,z) = R(x,y), S(z,y) are independent: the row of x = a is
determined by a's own tuples of R and by all of S.  So rank r of W takes the
tuples of R whose x lies in its range [b_r, b_{r+1}) together with the whole
of S, runs the query, and the ranks' outputs, concatenated in rank order,
are the sorted result (the paper partitions the output the same way to run
its product in parallel, Section 6).  No data moves between ranks.

The same ranges shard the set similarity join with its counts (a pair's
count depends only on a's row; ordered by count, the ranks' lists are merged
by count, ``merge_by_count``) and batches of set intersection requests (each
rank answers the requests whose a lies in its range, ``shard_pairs``).

The ranges are contiguous in x and balance the light join size: the weight
of x = a is sum over its y of deg_S(y), the number of candidates the light
expansion enumerates for a when everything is light (Section 3, the light
cost term).
"""
from __future__ import annotations

import numpy as np


def x_weights(rx: np.ndarray, ry: np.ndarray, sz=None, sy=None):
    """Distinct x values of R (sorted) and their candidate weights."""
    rx = np.asarray(rx, np.int64)
    ry = np.asarray(ry, np.int64)
    key = np.unique((rx << 32) | (ry & 0xFFFFFFFF))
    ux_all = key >> 32
    uy_all = (key & 0xFFFFFFFF).astype(np.uint32).astype(np.int32).astype(np.int64)
    if sz is None:
        s_y = uy_all
    else:
        skey = np.unique((np.asarray(sz, np.int64) << 32) | (np.asarray(sy, np.int64) & 0xFFFFFFFF))
        s_y = (skey & 0xFFFFFFFF).astype(np.uint32).astype(np.int32).astype(np.int64)
    yv, deg = np.unique(s_y, return_counts=True)
    pos = np.searchsorted(yv, uy_all)
    pos = np.minimum(pos, len(yv) - 1)
    w = np.where(yv[pos] == uy_all, deg[pos], 0).astype(np.int64)
    ux, start = np.unique(ux_all, return_index=True)
    wx = np.add.reduceat(w, start) if len(start) else np.zeros(0, np.int64)
    return ux, wx


def x_bounds(rx, ry, world: int, sz=None, sy=None):
    """Rank boundaries b_0 <= ... <= b_W (int64; b_0 = -2^31, b_W = 2^31) with
    contiguous x ranges of near-equal candidate weight."""
    if world < 1:
        raise ValueError("world must be >= 1")
    lo, hi = -(1 << 31), 1 << 31
    ux, wx = x_weights(rx, ry, sz, sy)
    b = [lo]
    if len(ux):
        cum = np.cumsum(wx + 1)            # +1: x with no S partner still costs a row
        total = cum[-1]
        for r in range(1, world):
            i = int(np.searchsorted(cum, total * r / world, side="left"))
            b.append(int(ux[min(i, len(ux) - 1)]) if i < len(ux) else hi)
    else:
        b += [hi] * (world - 1)
    b.append(hi)
    for r in range(1, len(b)):             # keep the boundaries monotone
        b[r] = max(b[r], b[r - 1])
    return np.array(b, np.int64)


def shard(rx, ry, rank: int, bounds):
    """R's tuples with x in [bounds[rank], bounds[rank + 1])."""
    rx = np.asarray(rx)
    ry = np.asarray(ry)
    lo, hi = int(bounds[rank]), int(bounds[rank + 1])
    m = (rx.astype(np.int64) >= lo) & (rx.astype(np.int64) < hi)
    return rx[m], ry[m]


def shard_pairs(tx, tz, rank: int, bounds):
    """Candidate pairs (a, b) of a set intersection batch whose a lies in the rank's x range.

    Rank r answers them against its shard of R and all of S; the ranks' answers,
    concatenated in rank order, are the batch's sorted answer.
    """
    tx = np.asarray(tx)
    tz = np.asarray(tz)
    lo, hi = int(bounds[rank]), int(bounds[rank + 1])
    m = (tx.astype(np.int64) >= lo) & (tx.astype(np.int64) < hi)
    return tx[m], tz[m]


def merge_by_count(parts):
    """Rank outputs (x, z, count), each by decreasing count with ties in (x, z) order, into
    one such list: ranks hold increasing x ranges, so a stable sort of their concatenation
    by decreasing count keeps equal counts in (x, z) order."""
    if not parts:
        return (np.empty(0, np.int32),) * 3
    x = np.concatenate([np.asarray(p[0]) for p in parts])
    z = np.concatenate([np.asarray(p[1]) for p in parts])
    c = np.concatenate([np.asarray(p[2]) for p in parts])
    perm = np.argsort(-c.astype(np.int64), kind="stable")
    return x[perm], z[perm], c[perm]
