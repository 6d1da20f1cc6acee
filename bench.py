"""Benchmark of the two-path join-project query on GB300.

One step = one ``jp_two_path`` call through the C-ABI on device-resident
inputs: index build, threshold selection (Algorithm 3 by default),
partition, heavy matrices + tensor-core product, light expansion and
deduplication, union and output placement, ending with the sorted distinct
(x, z) columns in HBM.  The workload is the 10M-tuple power-law relation
(x: 2M values, degree exponent 2.1; y: 1M values, exponent 1.8), self-join.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead (bounded samples of the same workload).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "two-path/star query ms & distinct tuples/s, learned vs cost-model Δ, bit-exact"
UNIT = "distinct tuples/s"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ----------------------------------------------------------------- workload
def make_workload(name):
    from paper_2002_12459_gb300 import workloads as W
    t = time.time()
    rx, ry = W.make(name)
    log(f"[bench] workload {name}: {len(rx)} tuples drawn in {time.time() - t:.1f}s")
    return rx, ry, W.WORKLOADS[name]


def candidate_counts(rx, ry):
    """Per distinct x (sorted): number of join candidates sum_{y in R[x]} deg(y)."""
    key = np.unique((rx.astype(np.int64) << 32) | (ry.astype(np.int64) & 0xFFFFFFFF))
    x = (key >> 32).astype(np.int64)
    y = (key & 0xFFFFFFFF).astype(np.int64)
    uy, yi, cy = np.unique(y, return_inverse=True, return_counts=True)
    ux, xi = np.unique(x, return_inverse=True)
    cand = np.bincount(xi, weights=cy[yi].astype(np.float64), minlength=len(ux))
    return ux, cand


# ----------------------------------------------------------------- ranks
def shard_plan(rx, ry, world, rank):
    """Rank boundaries over x (contiguous ranges of near-equal light-candidate weight) and
    rank `rank`'s tuples of R (paper_2002_12459_gb300.shard)."""
    from paper_2002_12459_gb300 import shard as SH
    bounds = SH.x_bounds(rx, ry, world)
    return bounds, SH.shard(rx, ry, rank, bounds)


def reduce_over_ranks(value, op, world):
    """max or sum of a host number over the ranks (torch.distributed; the value itself when
    there is one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s, p in zip(sm, power) if p > 0.25 * max(power)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- oracle baseline
# The oracle is timed on the host cores on rows of the same relation.  What it
# needs once per relation -- S sorted by y, R grouped by x -- is built before
# the clock starts, so the timed work is the per-row join, sort and unique.
# Rows are a stratified sample: every k-th x in decreasing candidate order
# (the largest x included), so hubs and light rows keep their shares.
def rows_csr(rx, ry):
    """Distinct tuples of R grouped by x: (x values, row offsets, y values)."""
    key = np.unique((rx.astype(np.int64) << 32) | (ry.astype(np.int64) & 0xFFFFFFFF))
    x = (key >> 32).astype(np.int32)
    y = (key & 0xFFFFFFFF).astype(np.uint32).astype(np.int32)
    ux, start = np.unique(x, return_index=True)
    return ux, np.append(start, len(x)).astype(np.int64), y


def stratified_rows(cand, target):
    """Row indices (sorted): every k-th row in decreasing candidate order, k set by target."""
    order = np.argsort(-cand, kind="stable")
    k = max(1, int(round(float(cand.sum()) / max(target, 1.0))))
    return np.sort(order[::k]), k


def split_rows(rows, cand, parts):
    """Consecutive groups of rows with about equal candidate counts."""
    if len(rows) == 0:
        return []
    cum = np.cumsum(cand[rows])
    cuts = np.searchsorted(cum, cum[-1] * np.arange(1, parts) / parts, side="right")
    return [g for g in np.split(rows, cuts) if len(g)]


def sub_csr(off, y, rows):
    lens = off[rows + 1] - off[rows]
    sub_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    idx = np.repeat(off[rows] - sub_off[:-1], lens) + np.arange(int(sub_off[-1]))
    return sub_off, y[idx]


_POOL_S = None


def _pool_init(sy, sz):
    global _POOL_S
    import oracle

    class _S:
        pass
    _POOL_S = _S()
    _POOL_S.y, _POOL_S.z = sy, sz
    oracle.build()


def _pool_rows(args):
    import oracle
    sub_off, sub_y, cap = args
    z, _ = oracle.two_path_rows(sub_off, sub_y, _POOL_S, cap_hint=cap)
    return len(z)


class OracleRows:
    """The oracle's per-row join over R's rows, single-threaded or on a process pool."""

    def __init__(self, rx, ry, procs=1):
        import oracle
        oracle.build()
        self.ux, self.off, self.y = rows_csr(rx, ry)
        self.S = oracle.SortedS(rx, ry)
        ys, cy = np.unique(self.S.y, return_counts=True)
        deg = np.zeros(len(self.y), np.float64)
        at = np.searchsorted(ys, self.y)
        ok = (at < len(ys)) & (ys[np.minimum(at, len(ys) - 1)] == self.y)
        deg[ok] = cy[at[ok]]
        self.cand = np.add.reduceat(deg, self.off[:-1]) if len(self.y) else np.zeros(0)
        self.procs = procs
        self.pool = None
        if procs > 1:
            import multiprocessing as mp
            self.pool = mp.get_context("spawn").Pool(procs, _pool_init, (self.S.y, self.S.z))
            self.pool.map(_pool_rows, [(np.zeros(1, np.int64), np.zeros(0, np.int32), 1)] * procs)

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None

    def run(self, rows):
        """Distinct pairs of the given rows and the wall seconds the oracle took."""
        import oracle
        if self.pool is None:
            sub_off, sub_y = sub_csr(self.off, self.y, rows)
            t = time.perf_counter()
            z, _ = oracle.two_path_rows(sub_off, sub_y, self.S, cap_hint=int(self.cand[rows].sum()))
            return len(z), time.perf_counter() - t
        groups = split_rows(rows, self.cand, 8 * self.procs)
        tasks = []
        for g in groups:
            so, sy = sub_csr(self.off, self.y, g)
            tasks.append((so, sy, int(self.cand[g].sum())))
        t = time.perf_counter()
        n = sum(self.pool.map(_pool_rows, tasks, chunksize=1))
        return n, time.perf_counter() - t


def cpu_sample(rx, ry, target_cand):
    """Prefix of x values whose join candidates add up to about target_cand (the set
    similarity join's oracle sample, which needs the witness counts of whole x ranges)."""
    ux, cand = candidate_counts(rx, ry)
    cum = np.cumsum(cand)
    k = int(np.searchsorted(cum, target_cand)) + 1
    k = max(1, min(k, len(ux)))
    return int(ux[0]), int(ux[k - 1]), k, float(cum[k - 1]), len(ux), float(cum[-1])


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(rx, ry, target_cand=3.0e8, full=False):
    """The oracle on the host cores: one core on a stratified sample, all cores on a sample
    as many times larger (or, with full, on every row)."""
    procs = os.cpu_count() or 1
    one = OracleRows(rx, ry, 1)
    rows1, k1 = stratified_rows(one.cand, target_cand)
    n1, s1 = one.run(rows1)
    c1 = float(one.cand[rows1].sum())
    res = {"value": n1 / s1, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": (f"every {k1}-th x in decreasing candidate order ({len(rows1)} of "
                      f"{len(one.ux)} x values, {c1:.3g} of {one.cand.sum():.3g} join candidates, "
                      f"the largest x included); S sorted and R grouped once before timing; "
                      f"{n1} distinct pairs in {s1:.2f}s"),
           "cpu": cpu_model()}
    if procs > 1:
        many = OracleRows(rx, ry, procs)
        try:
            if full:
                rowsP, kP = np.arange(len(many.ux)), 1
            else:
                rowsP, kP = stratified_rows(many.cand, target_cand * procs)
            nP, sP = many.run(rowsP)
        finally:
            many.close()
        cP = float(many.cand[rowsP].sum())
        res["all_cores"] = {
            "value": nP / sP, "unit": UNIT, "cores": procs,
            "sample": ("every x of the relation" if full else
                       f"every {kP}-th x in decreasing candidate order ({len(rowsP)} x values, "
                       f"{cP:.3g} join candidates)") +
                      f"; {procs} processes over groups of rows; {nP} distinct pairs in {sP:.2f}s"}
    return res


# ----------------------------------------------------------------- roofline
KERNEL_SLOTS = {4: "heavy_gemm_kernel", 6: "light_warp_kernel<256>",
                7: "light_bucket_kernel<2048,256>", 8: "light_merge_kernel",
                9: "light_bitmap_kernel", 11: "place_kernel"}
# timer slot -> light class index of jp_stats.light_* arrays
SLOT_CLASS = {6: (0,), 7: (1,), 8: (4, 5, 7), 9: (3, 6)}

# DRAM bytes (read + write) of one launch, from one ncu capture of the bench
# workload at the default thresholds (profiles/bitmap_and_place_powerlaw_10m_dram.md);
# reported only while the kernel's source code (code_hash) is the one that was captured
MEASURED_TRAFFIC = {
    "light_bitmap_kernel": {"bytes": 1241229568 + 5222891776, "workload": "two_path_powerlaw_10m",
                            "source": "paper_2002_12459_gb300/csrc/jp_light.cu",
                            "code_sha1": "81bbaee3bc3c6373a09c1eb8bff30eac8d55b31b"},
    "place_kernel": {"bytes": 11679594496 + 23196820736, "workload": "two_path_powerlaw_10m",
                     "source": "paper_2002_12459_gb300/csrc/jp_output.cu",
                     "code_sha1": "45d64df23739de5881e8a3a2f151c0b3d4740a3c"},
}


def code_hash(path):
    """sha1 of a CUDA/C++ source's code: comments removed and whitespace runs collapsed, so
    that an edit of comments alone keeps a capture while any code change drops it (the
    sources hold no comment markers inside string literals)."""
    import hashlib
    import re
    with open(path, encoding="utf-8") as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = re.sub(r"\s+", " ", src).strip()
    return hashlib.sha1(src.encode()).hexdigest()


def measured_traffic(kernel, workload):
    m = MEASURED_TRAFFIC.get(kernel)
    if not m or m["workload"] != workload:
        return None
    if code_hash(os.path.join(ROOT, m["source"])) != m["code_sha1"]:
        return None
    return m["bytes"]


def kernel_roofline(slot, st, peaks, peak_kind, ms):
    """Algorithmic work of one launch of a kernel slot / its event-timed duration."""
    hbm = peaks["hbm_gbs"]
    fp8_burst = 2.0 * peaks["bf16_tflops"]          # nominal fp8/bf16 dense ratio 4.5/2.25
    out = st["out_count"]
    if slot == 4:
        flops = 2.0 * st["u"] * st["v"] * st["w"]
        ach = flops / (ms * 1e-3) / 1e12
        r = {"kernel": KERNEL_SLOTS[slot], "ms": ms, "bound": "tensor", "achieved": ach,
             "peak": fp8_burst, "unit": "TFLOP/s", "frac": ach / fp8_burst, "traffic": None,
             "peak_source": f"{peak_kind} bf16 burst x 2 (fp8 nominal ratio)"}
        if peaks.get("fp8_tcgen05_tflops"):
            # this GPU's own FP8 tcgen05 rate, measured in this run (jp_measure_peaks)
            f8 = peaks["fp8_tcgen05_tflops"]
            r.update(peak=f8, frac=ach / f8,
                     peak_source="measured: tcgen05 kind::f8f6f4 128x256x32 issue loop, this run",
                     frac_of_bf16_burst_x2=ach / fp8_burst,
                     frac_of_int8_mma_sync=ach / peaks["int8_mma_sync_tflops"])
        return r
    if slot == 11:
        # read each list entry (4 B), write the k output columns (4 B each),
        # gather the value of each id of a bitmap row (4 B; the other lists
        # hold values); per row: offsets, list start, row values
        k = st.get("k", 2)
        ids = min(out, st["light_cand"][3] + st["light_cand"][6])
        byts = (4.0 + 4.0 * k) * out + 4.0 * ids + 20.0 * st["dom_x"]
    else:
        # candidates gathered (4 B), neighbour lists and per-x records read
        # (4 B each), distinct values written (bounded by the candidates)
        cand = sum(st["light_cand"][q] for q in SLOT_CLASS[slot])
        nxq = sum(st["light_x"][q] + st["light_deg"][q] for q in SLOT_CLASS[slot])
        byts = 4.0 * cand + 4.0 * nxq + 4.0 * min(cand, out)
    ach = byts / (ms * 1e-3) / 1e9
    return {"kernel": KERNEL_SLOTS[slot], "ms": ms, "bound": "hbm", "achieved": ach, "peak": hbm,
            "unit": "GB/s", "frac": ach / hbm, "traffic": None,
            "peak_source": f"{peak_kind} hbm copy"}


def roofline(st, peaks, peak_kind, ms_by_slot, workload=None):
    """Roofline of the slowest single kernel of the step, and of every kernel."""
    per = {KERNEL_SLOTS[s]: kernel_roofline(s, st, peaks, peak_kind, ms_by_slot[s])
           for s in KERNEL_SLOTS if ms_by_slot.get(s, 0.0) > 0}
    for name, r in per.items():
        r["traffic"] = measured_traffic(name, workload) if workload else None
    slot = max(KERNEL_SLOTS, key=lambda s: ms_by_slot.get(s, 0.0))
    top = dict(per[KERNEL_SLOTS[slot]])
    return top, per


# ----------------------------------------------------------------- learned thresholds
# thresholds Algorithm 3 picks on the 10M relation with the constants measured on that
# relation alone (the fitted defaults switch the heavy product off there)
PRODUCT_DELTAS = (271, 35)


def product_record(ctx, dx, dy, flush, args, peaks, kind):
    """The same query at fixed thresholds with a heavy product (PRODUCT_DELTAS): its time and
    the tensor-core product kernel's roofline, timed like the headline steps."""
    import torch
    ctx.set_threshold("fixed", *PRODUCT_DELTAS)
    ms, gm, st = [], [], None
    try:
        for i in range(1 + max(args.steps, 3)):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(ctx.stream)
            ox, oz = ctx.two_path(dx, dy)
            ev1.record(ctx.stream)
            torch.cuda.synchronize()
            st = ctx.stats()
            if i > 0:
                ms.append(ev0.elapsed_time(ev1))
                gm.append(st["ms_pass"][4])
            del ox, oz
    finally:
        ctx.set_threshold(args.mode, args.delta1, args.delta2)
    mean_ms, gemm_ms = sum(ms) / len(ms), sum(gm) / len(gm)
    log(f"[bench] fixed thresholds {PRODUCT_DELTAS}: {mean_ms:.2f} ms, product {gemm_ms:.3f} ms")
    return {"thresholds": list(PRODUCT_DELTAS), "ms_per_step": mean_ms, "steps": len(ms),
            "u": st["u"], "v": st["v"], "w": st["w"], "out_count": st["out_count"],
            "pass_ms": {k: round(v, 3) for k, v in enumerate(st["ms_pass"]) if v > 0},
            "heavy_gemm": kernel_roofline(4, st, peaks, kind, gemm_ms),
            "note": "Algorithm 3's choice with the constants measured on this relation alone; "
                    "the headline uses the defaults fitted on 789 relations, which choose no "
                    "heavy y here"}


def learned_vs_cost_model(ctx, dx, dy, flush, cost_ms, st_cost, args):
    """Query time at the shipped predictor's thresholds (JP_LEARNED) next to
    the cost-model time just measured, plus the held-out summary written when
    the predictor was trained."""
    import torch
    from paper_2002_12459_gb300 import jp
    pred = jp.Predictor.trained(0)
    ctx.set_predictor(pred)
    ctx.set_threshold("learned")
    ms, st = [], None
    try:
        for i in range(1 + args.steps):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(ctx.stream)
            ox, oz = ctx.two_path(dx, dy)
            ev1.record(ctx.stream)
            torch.cuda.synchronize()
            st = ctx.stats()
            if i > 0:
                ms.append(ev0.elapsed_time(ev1))
            del ox, oz
    finally:
        ctx.set_predictor(None)
        ctx.set_threshold(args.mode, args.delta1, args.delta2)
        pred.close()
    lm = sum(ms) / len(ms)
    log(f"[bench] learned thresholds {st['delta1']},{st['delta2']}: {lm:.2f} ms "
        f"(cost model {st_cost['delta1']},{st_cost['delta2']}: {cost_ms:.2f} ms)")
    held = None
    rep = os.path.join(ROOT, "paper_2002_12459_gb300", "predictor", "report.json")
    if os.path.exists(rep):
        with open(rep) as f:
            held = json.load(f)["summary"]
    return {"cost_model_ms": cost_ms, "learned_ms": lm, "learned_over_cost_model": lm / cost_ms,
            "cost_model_delta": [st_cost["delta1"], st_cost["delta2"]],
            "learned_delta": [st["delta1"], st["delta2"]],
            "out_count_equal": st["out_count"] == st_cost["out_count"],
            "held_out": None if held is None else {
                k: held[k] for k in ("relations", "learned_over_best_geomean",
                                     "cost_over_best_geomean", "train_relations")}}


# ----------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2002_12459_gb300 import build, jp

    torch.cuda.set_device(local_rank)
    build.build()
    rx, ry, wl = make_workload(args.workload)
    dx = torch.from_numpy(rx).cuda()
    dy = torch.from_numpy(ry).cuda()
    ctx = jp.Context(local_rank)
    tensor_peaks = ctx.measure_peaks()          # this GPU's FP8 tcgen05 and INT8 mma.sync rates
    log(f"[bench] measured tensor peaks: {tensor_peaks}")
    ctx.set_threshold(args.mode, args.delta1, args.delta2)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()

    # N > 1: rank r answers the x-range shard r of the one query (its tuples of R against
    # all of S) at the thresholds Algorithm 3 picks for the whole relation, found once
    # before the timed steps; every rank then makes the same partition (x and z degrees
    # are whole in each shard, y degrees come from S), and the ranks' outputs concatenated
    # in rank order are the query's sorted output
    bounds = None
    if world > 1:
        bounds, (qx, qy) = shard_plan(rx, ry, world, rank)
        dqx, dqy = torch.from_numpy(qx).cuda(), torch.from_numpy(qy).cuda()
        ox, oz = ctx.two_path(dx, dy)
        plan = ctx.stats()
        del ox, oz
        ctx.set_threshold("fixed", plan["delta1"], plan["delta2"])

        def query():
            return ctx.two_path(dqx, dqy, dx, dy)
    else:
        def query():
            return ctx.two_path(dx, dy)

    for i in range(args.warmup):
        ox, oz = query()
        del ox, oz
        torch.cuda.synchronize()
        log(f"[bench] warmup {i}: {ctx.stats()['ms_pass'][12]:.2f} ms")

    sampler = ClockSampler(local_rank)
    sampler.start()
    step_ms, stats, slot_ms = [], [], {}
    for i in range(args.steps):
        flush.fill_(i & 0xFF)                     # evict L2 (256 MiB > 129 MB)
        torch.cuda.synchronize()
        barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(ctx.stream)
        ox, oz = query()
        ev1.record(ctx.stream)
        torch.cuda.synchronize()
        barrier()
        ms = ev0.elapsed_time(ev1)
        st = ctx.stats()
        step_ms.append(ms)
        stats.append(st)
        for k, v in enumerate(st["ms_pass"]):
            slot_ms[k] = slot_ms.get(k, 0.0) + v / args.steps
        if i < args.steps - 1:
            del ox, oz
        log(f"[bench] step {i}: {ms:.2f} ms, OUT={st['out_count']}, launches={st['kernel_launches']}")
    clocks = sampler.stop()
    st = stats[-1]
    out = st["out_count"]
    mean_ms = sum(step_ms) / len(step_ms)
    max_ms = reduce_over_ranks(mean_ms, "max", world)
    total_out = int(reduce_over_ranks(out, "sum", world))

    # end to end through the C-ABI with host buffers, right after the timed
    # steps (same workspace and allocator state as the steps it is compared with)
    e2e = None
    if world == 1 and not args.no_e2e:
        # host input columns in, the result written by the output kernel straight into
        # pinned host columns (jp_two_path_into): every byte crosses the host link
        hrx = torch.from_numpy(rx).pin_memory()
        hry = torch.from_numpy(ry).pin_memory()
        cols = [torch.empty(out + 1, dtype=torch.int32, pin_memory=True) for _ in range(2)]
        times = []
        n = 0
        for i in range(1 + args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n = ctx.two_path_into(hrx, hry, cols[0], cols[1])
            torch.cuda.synchronize()
            if i > 0:
                times.append(time.perf_counter() - t0)
        k = len(times)
        e2e = {"value": out / (sum(times) / k), "unit": UNIT, "api": "jp_two_path_into",
               "h2d_bytes_per_step": int(8 * len(rx)), "d2h_bytes_per_step": int(8 * out),
               "ms_per_step": 1e3 * sum(times) / k, "count_equal": n == out}
        # the same through jp_two_path + jp_result_to_host (a device result, then copied)
        times, split = [], {}
        for i in range(1 + args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            gx, gz = ctx.two_path_host(hrx, hry, cols, timings=split if i > 0 else None)
            torch.cuda.synchronize()
            if i > 0:
                times.append(time.perf_counter() - t0)
            del gx, gz
        e2e["via_device_result"] = {"ms_per_step": 1e3 * sum(times) / len(times),
                                    "ms_split": {nm: round(1e3 * v / len(times), 2)
                                                 for nm, v in split.items()}}
        del cols, hrx, hry

    # the same query at the learned thresholds (the shipped predictor), timed
    # the same way, against the cost-model thresholds above
    learned = None
    if world == 1 and not args.no_learned and args.mode == "cost_model":
        learned = learned_vs_cost_model(ctx, dx, dy, flush, mean_ms, st, args)

    # sampled bit-exact check of the last result against the per-row oracle
    parity = None
    if rank == 0:
        import oracle
        oracle.build()
        srt = oracle.SortedS(rx, ry)
        hx = ox.cpu().numpy()
        hz = oz.cpu().numpy()
        ux = np.unique(rx)
        rng = np.random.default_rng(0)
        ux_c, cand = candidate_counts(rx, ry)
        if bounds is not None:           # rows of this rank's shard only
            keep = (ux >= bounds[rank]) & (ux < bounds[rank + 1])
            keep_c = (ux_c >= bounds[rank]) & (ux_c < bounds[rank + 1])
            ux, ux_c, cand = ux[keep], ux_c[keep_c], cand[keep_c]
        sample = list(rng.choice(ux, min(24, len(ux)), replace=False)) + list(ux_c[np.argsort(-cand)[:4]])
        ok = True
        for a in sample:
            s, e = np.searchsorted(hx, a, "left"), np.searchsorted(hx, a, "right")
            want = oracle.two_path_row(ry[rx == a], srt)
            ok &= bool(np.array_equal(hz[s:e], want))
        parity = {"rows_checked": len(sample), "bit_exact": ok}
        del hx, hz
    del ox, oz

    base = None
    if rank == 0 and world == 1 and not args.no_cpu:
        base = cpu_baseline(rx, ry, args.cpu_cand, full=args.cpu_full)

    peaks, kind = load_peaks()
    peaks.update(tensor_peaks)
    rl, rl_all = roofline(st, peaks, kind, slot_ms, args.workload)
    launches = sum(s["kernel_launches"] for s in stats)
    product = None
    if (world == 1 and not args.no_extra and args.workload == "two_path_powerlaw_10m"
            and args.mode == "cost_model"):
        product = product_record(ctx, dx, dy, flush, args, peaks, kind)
    ctx.close()
    if rank != 0:
        return None
    extra = None
    if world == 1 and not args.no_extra:
        extra = {}
        for name, fn in (("two_path_uniform_20k", lambda: run_uniform(args)),
                         ("star3_2m", lambda: run_star(args, "star3_2m"))):
            try:
                extra[name] = fn()
            except Exception as e:     # reported, never hidden
                extra[name] = {"error": f"{type(e).__name__}: {e}"}
        if "star3_2m" in extra and "metric" in extra["star3_2m"]:
            r = extra["star3_2m"]
            extra["star3_2m"] = {k: r[k] for k in ("value", "unit", "ms_per_step", "steps", "config",
                                                   "roofline", "kernel_rooflines", "cpu_baseline",
                                                   "parity", "gpu_launches")}
    return {
        "metric": METRIC, "value": total_out / (max_ms * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms,
        "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": args.workload, "n_tuples": wl["n"], "dom_x": wl["dom_x"],
                   "gamma_x": wl["gamma_x"], "dom_y": wl["dom_y"], "gamma_y": wl["gamma_y"],
                   "seed": wl["seed"], "query": "two-path self-join Q(x,z)=R(x,y),R(z,y)",
                   "threshold_mode": args.mode, "delta1": st["delta1"], "delta2": st["delta2"],
                   "u": st["u"], "v": st["v"], "w": st["w"], "out_count": total_out,
                   "light_candidates": st["light_candidates"], "out_join": st["out_join"],
                   "heavy_gemm": "tcgen05 kind::f8f6f4, E4M3 0/1 operands, exact FP32 accumulate",
                   "parallelism": (f"x-range shards of one query on {world} ranks, no collective on "
                                   "the data path" if world > 1 else "single GPU"),
                   "l2": "256 MiB flush written before every step",
                   "pass_ms": {k: round(v, 3) for k, v in slot_ms.items() if v > 0}},
        "roofline": rl, "kernel_rooflines": rl_all, "cpu_baseline": base, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "parity": parity, "learned_vs_cost_model": learned,
        "heavy_product_at_fixed_thresholds": product,
        "extra_workloads": extra,
    }


# ----------------------------------------------------------------- star workload
def run_star(args, workload=None):
    """Star Q*_3 on the 3 x 2M workload (single GPU, rank 0)."""
    import torch
    from paper_2002_12459_gb300 import build, jp
    from paper_2002_12459_gb300 import workloads as W

    build.build()
    workload = workload or args.workload
    t = time.time()
    rels = W.make(workload)
    wl = W.WORKLOADS[workload]
    log(f"[bench] workload {workload}: {len(rels)} x {len(rels[0][0])} tuples in {time.time() - t:.1f}s")
    drels = [(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()) for x, y in rels]
    ctx = jp.Context(0)
    tensor_peaks = ctx.measure_peaks()
    ctx.set_threshold(args.mode, args.delta1, args.delta2)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for i in range(args.warmup):
        cols = ctx.star(drels)
        del cols
        torch.cuda.synchronize()
        log(f"[bench] warmup {i}: {ctx.stats()['ms_pass'][12]:.2f} ms")
    sampler = ClockSampler(0)
    sampler.start()
    step_ms, stats, slot_ms = [], [], {}
    cols = None
    for i in range(args.steps):
        cols = None
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(ctx.stream)
        cols = ctx.star(drels)
        ev1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        st = ctx.stats()
        step_ms.append(ms)
        stats.append(st)
        for k, v in enumerate(st["ms_pass"]):
            slot_ms[k] = slot_ms.get(k, 0.0) + v / args.steps
        log(f"[bench] step {i}: {ms:.2f} ms, OUT={st['out_count']}, launches={st['kernel_launches']}")
    clocks = sampler.stop()
    st = dict(stats[-1])
    st["k"] = 3
    out = st["out_count"]
    mean_ms = sum(step_ms) / len(step_ms)

    # sampled bit-exact check: every output tuple whose x1 lies in a small range
    import oracle
    oracle.build()
    x1 = np.unique(rels[0][0])
    lo, hi = int(x1[len(x1) // 3]), int(x1[len(x1) // 3 + 15])
    want = oracle.star(rels, x_lo=lo, x_hi=hi)
    b = torch.searchsorted(cols[0], torch.tensor([lo, hi + 1], dtype=torch.int32, device="cuda"))
    s, e = int(b[0]), int(b[1])
    got = [c[s:e].cpu().numpy() for c in cols]
    ok = all(np.array_equal(g, w) for g, w in zip(got, want))
    parity = {"x1_range": [lo, hi], "tuples_checked": int(e - s), "bit_exact": bool(ok)}
    del cols

    base = None
    if not args.no_cpu:
        t = time.perf_counter()
        lo2, hi2 = int(x1[0]), int(x1[min(len(x1) - 1, 1000)])
        n = len(oracle.star(rels, x_lo=lo2, x_hi=hi2)[0])
        secs = time.perf_counter() - t
        base = {"value": n / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": (f"x1 values {lo2}..{hi2} (1001 of {len(x1)}), single-threaded C oracle "
                           f"incl. its sort of the three relations; {n} distinct triples in {secs:.2f}s")}
    peaks, kind = load_peaks()
    peaks.update(tensor_peaks)
    rl, rl_all = roofline(st, peaks, kind, slot_ms, workload)
    launches = sum(s_["kernel_launches"] for s_ in stats)
    ctx.close()
    return {
        "metric": METRIC, "value": out / (mean_ms * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": workload, "n_tuples_per_relation": wl["n"], "k": 3,
                   "dom_x": wl["dom_x"], "dom_y": wl["dom_y"], "gamma_y": wl["gamma_y"],
                   "seed": wl["seed"], "query": "star Q*_3(x1,x2,x3)=R1(x1,y),R2(x2,y),R3(x3,y)",
                   "threshold_mode": args.mode, "delta1": st["delta1"], "delta2": st["delta2"],
                   "heavy_pairs_u": st["u"], "v": st["v"], "w": st["w"], "out_count": out,
                   "out_join": st["out_join"], "l2": "256 MiB flush written before every step",
                   "pass_ms": {k: round(v, 3) for k, v in slot_ms.items() if v > 0}},
        "roofline": rl, "kernel_rooflines": rl_all, "cpu_baseline": base,
        "e2e": None, "e2e_note": "not measured: the result is 144 GB, beyond a host copy per step",
        "gpu_launches": launches, "clocks": clocks, "parity": parity,
    }


def run_uniform(args, workload="two_path_uniform_20k", delta=141):
    """The small two-path workload at fixed thresholds floor(sqrt(N)): timed on the GPU, the
    whole output compared with the oracle, and the oracle timed on one host core."""
    import torch
    from paper_2002_12459_gb300 import build, jp
    import oracle

    build.build()
    rx, ry, wl = make_workload(workload)
    dx, dy = torch.from_numpy(rx).cuda(), torch.from_numpy(ry).cuda()
    ctx = jp.Context(0)
    ctx.set_threshold("fixed", delta, delta)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        ox, oz = ctx.two_path(dx, dy)
        torch.cuda.synchronize()
    steps = max(args.steps, 20)
    ms = []
    for i in range(steps):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(ctx.stream)
        ox, oz = ctx.two_path(dx, dy)
        ev1.record(ctx.stream)
        torch.cuda.synchronize()
        ms.append(ev0.elapsed_time(ev1))
    st = ctx.stats()
    ctx.close()
    oracle.build()
    t = time.perf_counter()
    wx, wz = oracle.two_path(rx, ry)
    secs = time.perf_counter() - t
    ok = np.array_equal(ox.cpu().numpy(), wx) and np.array_equal(oz.cpu().numpy(), wz)
    mean_ms = sum(ms) / len(ms)
    out = st["out_count"]
    return {"workload": workload, "value": out / (mean_ms * 1e-3), "unit": UNIT,
            "ms_per_step": mean_ms, "steps": steps,
            "config": {"n_tuples": wl["n"], "dom_x": wl["dom_x"], "dom_y": wl["dom_y"],
                       "seed": wl["seed"], "threshold_mode": "fixed", "delta1": delta,
                       "delta2": delta, "u": st["u"], "v": st["v"], "out_count": out,
                       "light_candidates": st["light_candidates"],
                       "pass_ms": {k: round(v, 4) for k, v in enumerate(st["ms_pass"]) if v > 0}},
            "parity": {"pairs_checked": int(len(wx)), "bit_exact": bool(ok)},
            "cpu_baseline": {"value": len(wx) / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"the whole relation, single-threaded C oracle: {len(wx)} "
                                       f"distinct pairs in {secs:.3f}s"},
            "note": "a tiny query: the time is the pipeline's launches and host synchronisations"}


# ----------------------------------------------------------------- set similarity join
def ssj_rooflines(st, peaks, ms, cand, distinct_light):
    """Phases of jp_two_path_counts against their rooflines (algorithmic work per step).

    counting product: 2 u v w flops; candidate fill: per candidate an id read (4 B) and a key
    written (8 B); sort and run lengths: per candidate the key read once (8 B), per distinct light
    pair a key and a count written (12 B); heavy rows, merge and output: per output pair 12 B
    written, per distinct pair 12 B read.
    """
    hbm = peaks["hbm_gbs"]
    out = st["out_count"]
    res = {}
    if ms.get(4, 0) > 0 and st["u"] > 0:
        f8 = peaks.get("fp8_tcgen05_tflops") or 2.0 * peaks["bf16_tflops"]
        ach = 2.0 * st["u"] * st["v"] * st["w"] / (ms[4] * 1e-3) / 1e12
        res["heavy_gemm_kernel<true>"] = {"ms": ms[4], "bound": "tensor", "achieved": ach,
                                          "peak": f8, "unit": "TFLOP/s", "frac": ach / f8,
                                          "traffic": None}
    work = {13: ("cand_fill_kernel", 12.0 * cand),
            14: ("radix sort + run lengths", 8.0 * cand + 12.0 * distinct_light),
            15: ("heavy rows, merge, output", 12.0 * out + 12.0 * distinct_light)}
    for slot, (name, byts) in work.items():
        if ms.get(slot, 0) > 0:
            ach = byts / (ms[slot] * 1e-3) / 1e9
            res[name] = {"ms": ms[slot], "bound": "hbm", "achieved": ach, "peak": hbm,
                         "unit": "GB/s", "frac": ach / hbm, "traffic": None}
    top = max(res, key=lambda k: res[k]["ms"])
    return dict(res[top], kernel=top), res


def run_ssj(args):
    """Ordered set similarity join (pairs sharing >= c_min y, by decreasing count)."""
    import torch
    from paper_2002_12459_gb300 import build, jp
    from paper_2002_12459_gb300 import workloads as W

    build.build()
    wl = W.WORKLOADS[args.workload]
    c_min = wl["c_min"]
    t = time.time()
    rx, ry = W.make(args.workload)
    log(f"[bench] workload {args.workload}: {len(rx)} tuples in {time.time() - t:.1f}s")
    dx, dy = torch.from_numpy(rx).cuda(), torch.from_numpy(ry).cuda()
    ctx = jp.Context(0)
    tensor_peaks = ctx.measure_peaks()
    ctx.set_threshold(args.mode, args.delta1, args.delta2)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for i in range(args.warmup):
        cols = ctx.two_path_counts(dx, dy, c_min=c_min, order="count")
        del cols
        torch.cuda.synchronize()
        log(f"[bench] warmup {i}: {ctx.stats()['ms_pass'][12]:.2f} ms")
    sampler = ClockSampler(0)
    sampler.start()
    step_ms, slot_ms, st = [], {}, None
    cols = None
    for i in range(args.steps):
        cols = None
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(ctx.stream)
        cols = ctx.two_path_counts(dx, dy, c_min=c_min, order="count")
        ev1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        st = ctx.stats()
        step_ms.append(ms)
        for k, v in enumerate(st["ms_pass"]):
            slot_ms[k] = slot_ms.get(k, 0.0) + v / args.steps
        log(f"[bench] step {i}: {ms:.2f} ms, OUT={st['out_count']}, ranges={st['count_ranges']}, "
            f"launches={st['kernel_launches']}")
    clocks = sampler.stop()
    mean_ms = sum(step_ms) / len(step_ms)
    out = st["out_count"]

    # sampled bit-exact check: the pairs of an x range (taken out of the count order and
    # sorted by (x, z) on the device) against the oracle's counts
    import oracle
    oracle.build()
    ox, oz, oc = cols
    vals, cnts = np.unique(rx, return_counts=True)
    hub = int(vals[np.argmax(cnts)])
    checked, ok = 0, True
    for lo, hi in [(hub, hub), (int(vals[len(vals) // 2]), int(vals[len(vals) // 2 + 300]))]:
        sel = (ox >= lo) & (ox <= hi)
        gx, gz, gc = ox[sel].long(), oz[sel].long(), oc[sel]
        perm = torch.argsort(gx * (1 << 32) + (gz + (1 << 31)))
        wx, wz, wc = oracle.two_path(rx, ry, x_lo=lo, x_hi=hi, with_counts=True)
        keep = wc >= c_min
        ok &= (np.array_equal(gx[perm].cpu().numpy(), wx[keep])
               and np.array_equal(gz[perm].cpu().numpy(), wz[keep])
               and np.array_equal(gc[perm].cpu().numpy(), wc[keep]))
        checked += int(keep.sum())
    ok &= bool((oc[1:] <= oc[:-1]).all())
    parity = {"x_ranges": "the largest-degree x, and 301 x values mid-domain", "pairs_checked": checked,
              "count_order_nonincreasing": bool((oc[1:] <= oc[:-1]).all()), "bit_exact": bool(ok)}
    del cols, ox, oz, oc, sel, gx, gz, gc

    base = None
    if not args.no_cpu:
        lo, hi, k, c, nx, ctot = cpu_sample(rx, ry, 1.0e7)
        t = time.perf_counter()
        wx, wz, wc = oracle.two_path(rx, ry, x_lo=lo, x_hi=hi, with_counts=True)
        n = int((wc >= c_min).sum())
        secs = time.perf_counter() - t
        base = {"value": n / secs, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                "sample": (f"x values {lo}..{hi} ({k} of {nx} x values, {c:.3g} of {ctot:.3g} join "
                           f"candidates), single-threaded C oracle with witness counts, filtered "
                           f">= {c_min}; {n} pairs in {secs:.2f}s")}
    peaks, kind = load_peaks()
    peaks.update(tensor_peaks)
    rl, rl_all = ssj_rooflines(st, peaks, slot_ms, st["light_candidates"], st["count_light_pairs"])
    ctx.close()
    return {
        "metric": "ssj_pairs_per_sec", "value": out / (mean_ms * 1e-3), "unit": "pairs/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": args.workload, "n_tuples": wl["n"], "c_min": c_min,
                   "order": "count descending, ties in (x, z) order",
                   "query": "SSJ: (a, c, |R[a] ∩ R[c]|) with |R[a] ∩ R[c]| >= c_min",
                   "threshold_mode": args.mode, "delta1": st["delta1"], "delta2": st["delta2"],
                   "u": st["u"], "v": st["v"], "w": st["w"], "out_count": out,
                   "light_candidates": st["light_candidates"], "x_ranges": st["count_ranges"],
                   "light_pairs": st["count_light_pairs"], "heavy_pairs": st["heavy_pairs"],
                   "l2": "256 MiB flush written before every step",
                   "pass_ms": {k: round(v, 3) for k, v in slot_ms.items() if v > 0}},
        "roofline": rl, "kernel_rooflines": rl_all, "cpu_baseline": base,
        "e2e": None, "e2e_note": "not measured for this workload",
        "gpu_launches": st["kernel_launches"] * args.steps, "clocks": clocks, "parity": parity,
    }


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle on all host cores, each step a stratified sample of the workload's rows."""
    rx, ry, wl = make_workload(args.workload)
    procs = os.cpu_count() or 1
    orc = OracleRows(rx, ry, procs)
    try:
        rows, k = stratified_rows(orc.cand, args.ref_cand)
        for _ in range(args.warmup):
            orc.run(rows)
        times, n = [], 0
        for _ in range(args.steps):
            n, secs = orc.run(rows)
            times.append(secs)
    finally:
        orc.close()
    secs = sum(times) / len(times)
    value = n / secs
    c = float(orc.cand[rows].sum())
    sample = (f"every {k}-th x in decreasing candidate order ({len(rows)} of {len(orc.ux)} x values, "
              f"{c:.3g} of {orc.cand.sum():.3g} join candidates) per step; C oracle on {procs} "
              f"processes, S sorted and R grouped once before timing; {n} distinct pairs")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": args.workload, "n_tuples": wl["n"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="two_path_powerlaw_10m")
    ap.add_argument("--mode", default="cost_model", choices=["fixed", "closed_form", "cost_model"])
    ap.add_argument("--delta1", type=int, default=1)
    ap.add_argument("--delta2", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the uniform 20k and star k = 3 workloads reported beside the main one")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip timing the query at the shipped predictor's thresholds")
    ap.add_argument("--ref-cand", type=float, default=4.0e8,
                    help="join candidates per step of the reference arm (all host cores)")
    ap.add_argument("--cpu-cand", type=float, default=3.0e8,
                    help="join candidates of the single-core oracle sample (x cores for all cores)")
    ap.add_argument("--cpu-full", action="store_true",
                    help="time the all-cores oracle over every row of the relation")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    from paper_2002_12459_gb300 import workloads as W
    if W.WORKLOADS[args.workload]["kind"] == "star":
        res = run_star(args) if rank == 0 else None
    elif W.WORKLOADS[args.workload]["kind"] == "ssj":
        res = run_ssj(args) if rank == 0 else None
    else:
        res = run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
