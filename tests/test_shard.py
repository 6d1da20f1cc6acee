"""x-range sharding (the multi-GPU path) on CPU: boundaries, coverage, and a
world-size-2 gloo run whose ranks each answer their shard with the oracle;
the concatenation in rank order must equal the unsharded oracle result."""
import os
import socket
import sys
import tempfile

import numpy as np
import pytest

from paper_2002_12459_gb300 import shard, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_bounds_partition_relation(world):
    rx, ry = W.powerlaw_relation(20000, 4000, 2.1, 2000, 1.8, 3)
    b = shard.x_bounds(rx, ry, world)
    assert len(b) == world + 1 and b[0] == -(1 << 31) and b[-1] == 1 << 31
    assert np.all(np.diff(b) >= 0)
    parts = [shard.shard(rx, ry, r, b) for r in range(world)]
    assert sum(len(p[0]) for p in parts) == len(rx)
    for r, (px, _) in enumerate(parts):
        if len(px):
            assert px.min() >= b[r] and px.max() < b[r + 1]
    # balance: no rank carries much more than its share of the candidate weight
    ux, wx = shard.x_weights(rx, ry)
    tot = float((wx + 1).sum())
    for r in range(world):
        m = (ux >= b[r]) & (ux < b[r + 1])
        assert (wx[m] + 1).sum() <= tot / world + (wx + 1).max() + 1


def test_weights_match_definition():
    rx = np.array([0, 0, 1, 2, 2, 2], np.int32)
    ry = np.array([5, 6, 5, 5, 6, 7], np.int32)
    ux, wx = shard.x_weights(rx, ry)
    # deg(5)=3, deg(6)=2, deg(7)=1
    assert ux.tolist() == [0, 1, 2] and wx.tolist() == [5, 3, 6]
    sz = np.array([9, 9, 8], np.int32)
    sy = np.array([5, 6, 6], np.int32)
    ux, wx = shard.x_weights(rx, ry, sz, sy)
    assert wx.tolist() == [3, 1, 3]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    from paper_2002_12459_gb300 import shard as sh, workloads as wl
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    rx, ry = wl.powerlaw_relation(6000, 1200, 2.1, 600, 1.8, 11)
    b = sh.x_bounds(rx, ry, world)
    px, py = sh.shard(rx, ry, rank, b)
    ox, oz = oracle.two_path(px, py, rx, ry)
    parts = [None] * world
    dist.all_gather_object(parts, (ox, oz))
    if rank == 0:
        gx = np.concatenate([p[0] for p in parts])
        gz = np.concatenate([p[1] for p in parts])
        fx, fz = oracle.two_path(rx, ry)
        ok = np.array_equal(gx, fx) and np.array_equal(gz, fz)
        with open(os.path.join(out_dir, "ok"), "w") as f:
            f.write(f"{int(ok)} {len(fx)}")
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_world2_sharded_equals_unsharded(oracle_mod):
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True,
                           start_method="spawn")
        ok, n = open(os.path.join(d, "ok")).read().split()
    assert ok == "1" and int(n) > 0


def test_merge_by_count_keeps_pair_order_for_ties():
    a = (np.array([1, 1, 2], np.int32), np.array([5, 3, 1], np.int32), np.array([4, 2, 2], np.int32))
    b = (np.array([7, 9], np.int32), np.array([0, 2], np.int32), np.array([4, 3], np.int32))
    x, z, c = shard.merge_by_count([a, b])
    assert list(zip(x.tolist(), z.tolist(), c.tolist())) == [
        (1, 5, 4), (7, 0, 4), (9, 2, 3), (1, 3, 2), (2, 1, 2)]
    assert all(len(v) == 0 for v in shard.merge_by_count([]))


def test_shard_pairs_cover_the_batch():
    rx, ry = W.powerlaw_relation(5000, 1000, 2.1, 500, 1.8, 4)
    ux = np.unique(rx)
    tx, tz = W.candidate_pairs(ux, ux, 3000, seed=2, absent=0.1)
    b = shard.x_bounds(rx, ry, 3)
    parts = [shard.shard_pairs(tx, tz, r, b) for r in range(3)]
    assert sum(len(p[0]) for p in parts) == len(tx)


def _rank_apps(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    from paper_2002_12459_gb300 import shard as sh, workloads as wl
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    rx, ry = wl.powerlaw_relation(6000, 1200, 2.1, 600, 1.8, 12)
    ux = np.unique(rx)
    tx, tz = wl.candidate_pairs(ux, ux, 4000, seed=3, absent=0.05)
    b = sh.x_bounds(rx, ry, world)
    px, py = sh.shard(rx, ry, rank, b)
    counts = oracle.ssj(px, py, 2, rx, ry, order="count")
    qx, qz = sh.shard_pairs(tx, tz, rank, b)
    answers = oracle.bsi(px, py, qx, qz, rx, ry)
    parts = [None] * world
    dist.all_gather_object(parts, (counts, answers))
    if rank == 0:
        mx, mz, mc = sh.merge_by_count([p[0] for p in parts])
        wx, wz, wc = oracle.ssj(rx, ry, 2, order="count")
        ok = np.array_equal(mx, wx) and np.array_equal(mz, wz) and np.array_equal(mc, wc)
        gx = np.concatenate([p[1][0] for p in parts])
        gz = np.concatenate([p[1][1] for p in parts])
        fx, fz = oracle.bsi(rx, ry, tx, tz)
        ok = ok and np.array_equal(gx, fx) and np.array_equal(gz, fz)
        with open(os.path.join(out_dir, "ok"), "w") as f:
            f.write(f"{int(ok)} {len(wx)} {len(fx)}")
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_world2_sharded_counts_and_batches(oracle_mod):
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_apps, args=(2, _free_port(), d), nprocs=2, join=True,
                           start_method="spawn")
        ok, n1, n2 = open(os.path.join(d, "ok")).read().split()
    assert ok == "1" and int(n1) > 0 and int(n2) > 0
