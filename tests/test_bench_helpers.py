"""Host logic of bench.py (no GPU): the oracle sample, the roofline arithmetic, the traffic
gate and the clock record."""
import os

import numpy as np
import pytest

import bench


def test_cpu_sample_takes_a_prefix_of_x_by_candidates():
    rx = np.array([0, 0, 1, 2, 2, 3], np.int32)
    ry = np.array([5, 6, 5, 5, 7, 6], np.int32)
    # deg(5) = 3, deg(6) = 2, deg(7) = 1: candidates per x 5, 3, 4, 2
    ux, cand = bench.candidate_counts(rx, ry)
    assert ux.tolist() == [0, 1, 2, 3] and cand.tolist() == [5, 3, 4, 2]
    lo, hi, k, c, nx, tot = bench.cpu_sample(rx, ry, 7)
    assert (lo, hi, k, c, nx, tot) == (0, 1, 2, 8.0, 4, 14.0)


def test_stratified_rows_take_every_kth_by_candidates_with_the_largest():
    cand = np.array([5.0, 100.0, 1.0, 7.0, 30.0, 2.0, 9.0, 3.0])
    rows, k = bench.stratified_rows(cand, cand.sum() / 4)
    # decreasing order: 1 (100), 4 (30), 6 (9), 3 (7), 0 (5), 7 (3), 5 (2), 2 (1): every 4th
    assert k == 4 and rows.tolist() == [0, 1]
    rows, k = bench.stratified_rows(cand, 1e9)
    assert k == 1 and rows.tolist() == list(range(8))


def test_split_rows_and_sub_csr():
    cand = np.array([4.0, 4.0, 4.0, 4.0, 8.0, 8.0])
    groups = bench.split_rows(np.arange(6), cand, 2)
    assert [g.tolist() for g in groups] == [[0, 1, 2, 3], [4, 5]]
    off = np.array([0, 2, 3, 6], np.int64)
    y = np.array([10, 11, 20, 30, 31, 32], np.int32)
    so, sy = bench.sub_csr(off, y, np.array([2, 0]))
    assert so.tolist() == [0, 3, 5] and sy.tolist() == [30, 31, 32, 10, 11]


def test_oracle_rows_single_and_pool_count_the_distinct_pairs(oracle_mod):
    from paper_2002_12459_gb300 import workloads as W
    rng = np.random.default_rng(4)
    rx, ry = W.random_small_relation(rng, 4000, 300, 120, -50, 9, 0.8)
    ox, oz = oracle_mod.two_path(rx, ry)
    one = bench.OracleRows(rx, ry, 1)
    n, secs = one.run(np.arange(len(one.ux)))
    assert n == len(ox) and secs >= 0
    # candidates per x are sum_{y in R[x]} deg(y)
    ux, cand = bench.candidate_counts(rx, ry)
    assert np.array_equal(one.ux, ux) and np.array_equal(one.cand, cand)
    rows, _ = bench.stratified_rows(one.cand, one.cand.sum() / 5)
    want = sum(int((ox == one.ux[r]).sum()) for r in rows)
    two = bench.OracleRows(rx, ry, 2)
    try:
        assert two.run(rows)[0] == want == one.run(rows)[0]
    finally:
        two.close()


def _stats(**kw):
    st = {"out_count": 1000, "u": 256, "v": 128, "w": 512, "dom_x": 10, "k": 2,
          "light_cand": [100, 0, 0, 50, 0, 0, 25, 0], "light_x": [4, 0, 0, 2, 0, 0, 1, 0],
          "light_deg": [8, 0, 0, 4, 0, 0, 2, 0], "light_candidates": 175,
          "count_light_pairs": 90}
    st.update(kw)
    return st


def test_gemm_roofline_is_flops_over_time_against_the_measured_rate():
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 2000.0, "fp8_tcgen05_tflops": 4800.0,
             "int8_mma_sync_tflops": 160.0}
    r = bench.kernel_roofline(4, _stats(), peaks, "measured", 0.5)
    flops = 2.0 * 256 * 128 * 512
    assert r["bound"] == "tensor" and r["achieved"] == pytest.approx(flops / 0.5e-3 / 1e12)
    assert r["peak"] == 4800.0 and r["frac"] == pytest.approx(r["achieved"] / 4800.0)
    assert r["frac_of_bf16_burst_x2"] == pytest.approx(r["achieved"] / 4000.0)


def test_light_roofline_counts_its_class_bytes():
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 2000.0}
    r = bench.kernel_roofline(9, _stats(), peaks, "measured", 1.0)   # bitmap: classes 3 and 6
    cand, nxq = 75, (2 + 4) + (1 + 2)
    want = 4.0 * cand + 4.0 * nxq + 4.0 * min(cand, 1000)
    assert r["bound"] == "hbm" and r["achieved"] == pytest.approx(want / 1e-3 / 1e9)
    top, per = bench.roofline(_stats(), peaks, "measured", {9: 1.0, 6: 0.2, 4: 0.1})
    assert top["kernel"] == "light_bitmap_kernel" and set(per) == {
        "light_bitmap_kernel", "light_warp_kernel<256>", "heavy_gemm_kernel"}


def test_ssj_rooflines_pick_the_slowest_phase():
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 2000.0, "fp8_tcgen05_tflops": 4800.0}
    top, per = bench.ssj_rooflines(_stats(out_count=40), peaks, {4: 0.1, 13: 0.2, 14: 3.0, 15: 0.5},
                                   175, 90)
    assert top["kernel"] == "radix sort + run lengths"
    assert top["achieved"] == pytest.approx((8.0 * 175 + 12.0 * 90) / 3e-3 / 1e9)
    assert per["cand_fill_kernel"]["achieved"] == pytest.approx(12.0 * 175 / 0.2e-3 / 1e9)


@pytest.mark.parametrize("kernel", ["light_bitmap_kernel", "place_kernel"])
def test_traffic_is_reported_only_for_the_captured_source(kernel):
    m = bench.MEASURED_TRAFFIC[kernel]
    same = bench.code_hash(os.path.join(bench.ROOT, m["source"])) == m["code_sha1"]
    got = bench.measured_traffic(kernel, m["workload"])
    assert got == (m["bytes"] if same else None)
    assert bench.measured_traffic(kernel, "star3_2m") is None
    assert bench.measured_traffic("light_merge_kernel", m["workload"]) is None


def test_code_hash_ignores_comments_only(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("// one\nint f(int x) {  /* add */ return x + 1; }\n")
    b.write_text("// two, longer\nint f(int x) {\n    return x + 1;  // add\n}\n")
    c.write_text("int f(int x) { return x + 2; }\n")
    assert bench.code_hash(str(a)) == bench.code_hash(str(b))
    assert bench.code_hash(str(a)) != bench.code_hash(str(c))


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_median_under_load_and_reasons(tmp_path):
    path = tmp_path / "clocks.csv"
    rows = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2070, 2070, 950.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1980, 2070, 880.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 345, 2070, 90.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage"]
    path.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.proc, cs.path, cs.fh = _Proc(), str(path), open(os.devnull, "w")
    rec = cs.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0   # idle sample left out
    assert rec["reasons"] == ["sw_power_cap"] and rec["samples"] == 4


def _sharded_rank(rank, world, port, out_path):
    import os
    import torch.distributed as dist
    import oracle
    from paper_2002_12459_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(9)
        rx, ry = W.random_small_relation(rng, 3000, 250, 90, -120, 5, 0.8)
        bounds, (qx, qy) = bench.shard_plan(rx, ry, world, rank)
        ox, oz = oracle.two_path(qx, qy, rx, ry)           # the rank's shard against all of S
        total = bench.reduce_over_ranks(len(ox), "sum", world)
        slowest = bench.reduce_over_ranks(float(rank + 1), "max", world)
        parts = [None] * world
        dist.all_gather_object(parts, (ox.tolist(), oz.tolist()))
        if rank == 0:
            wx, wz = oracle.two_path(rx, ry)
            gx = np.concatenate([np.array(p[0], np.int32) for p in parts])
            gz = np.concatenate([np.array(p[1], np.int32) for p in parts])
            ok = (total == len(wx) and slowest == float(world) and np.array_equal(gx, wx)
                  and np.array_equal(gz, wz))
            with open(out_path, "w") as f:
                f.write("ok" if ok else f"bad {total} {len(wx)} {slowest}")
    finally:
        dist.destroy_process_group()


def test_sharded_bench_logic_on_two_gloo_ranks(tmp_path, oracle_mod):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = tmp_path / "result.txt"
    mp.start_processes(_sharded_rank, args=(2, port, str(out)), nprocs=2, join=True,
                       start_method="spawn")
    assert out.read_text() == "ok"
