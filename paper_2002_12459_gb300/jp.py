"""Python binding of the C-ABI library ``libjp.so`` (argument marshalling only).

Every step of the query runs in the library's CUDA kernels; this module only
converts torch tensors to pointers, hands PyTorch's caching allocator to the
library, and wraps the result columns as torch tensors without copying.

There is no fallback: if ``libjp.so`` is missing, or no sm_103 GPU is
present, the calls raise.

Functions mirror the C names: ``jp_two_path`` -> ``Context.two_path``,
``jp_star`` -> ``Context.star``, ``jp_set_threshold`` ->
``Context.set_threshold``, ``jp_get_stats`` -> ``Context.stats``.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libjp.so")

JP_OK, JP_EINVAL, JP_ENOMEM, JP_ECUDA, JP_EOVERFLOW, JP_ETIMEOUT, JP_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
JP_FIXED, JP_CLOSED_FORM, JP_COST_MODEL = 0, 1, 2
_MODES = {"fixed": JP_FIXED, "closed_form": JP_CLOSED_FORM, "cost_model": JP_COST_MODEL}
_CODES = {JP_EINVAL: "JP_EINVAL", JP_ENOMEM: "JP_ENOMEM", JP_ECUDA: "JP_ECUDA",
          JP_EOVERFLOW: "JP_EOVERFLOW", JP_ETIMEOUT: "JP_ETIMEOUT",
          JP_EUNSUPPORTED: "JP_EUNSUPPORTED"}


class JPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class jp_rel(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("n", ctypes.c_int64)]


class jp_result(ctypes.Structure):
    _fields_ = [("col", ctypes.c_void_p * 8), ("count", ctypes.c_int64), ("k", ctypes.c_int32),
                ("_block", ctypes.c_void_p), ("_bytes", ctypes.c_size_t)]


class jp_stats(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int64), ("n_s", ctypes.c_int64), ("dom_x", ctypes.c_int64),
                ("dom_y", ctypes.c_int64), ("dom_z", ctypes.c_int64),
                ("out_join", ctypes.c_double), ("out_estimate", ctypes.c_double),
                ("delta1", ctypes.c_int64), ("delta2", ctypes.c_int64),
                ("threshold_mode", ctypes.c_int32), ("u", ctypes.c_int64),
                ("v", ctypes.c_int64), ("w", ctypes.c_int64),
                ("light_candidates", ctypes.c_int64), ("out_count", ctypes.c_int64),
                ("heavy_pairs", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("light_x", ctypes.c_int64 * 8), ("light_cand", ctypes.c_int64 * 8),
                ("light_deg", ctypes.c_int64 * 8),
                ("ms_total", ctypes.c_double),
                ("ms_pass", ctypes.c_double * 16), ("learned_judged", ctypes.c_int64),
                ("filter_pairs", ctypes.c_int64), ("filter_query_out", ctypes.c_int64),
                ("count_ranges", ctypes.c_int64), ("count_light_pairs", ctypes.c_int64),
                ("gemm_tile", ctypes.c_int64)]


class jp_cost_model(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("T_I", "T_m", "T_s", "mm_rate", "mm_fixed", "eps", "wcoj_factor", "judge")]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_lib_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libjp.so; raises if it has not been built."""
    global _lib
    with _lib_lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with "
                                   "python -m paper_2002_12459_gb300.build")
            lib = ctypes.CDLL(path)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            lib.jp_create.argtypes = [ctypes.POINTER(vp), i32, vp, ALLOC_FN, FREE_FN, vp]
            lib.jp_create.restype = i32
            lib.jp_destroy.argtypes = [vp]
            lib.jp_destroy.restype = None
            lib.jp_set_threshold.argtypes = [vp, i32, i64, i64]
            lib.jp_set_threshold.restype = i32
            lib.jp_set_cost_model.argtypes = [vp, ctypes.POINTER(jp_cost_model)]
            lib.jp_set_cost_model.restype = i32
            lib.jp_get_cost_model.argtypes = [vp, ctypes.POINTER(jp_cost_model)]
            lib.jp_get_cost_model.restype = i32
            lib.jp_set_gemm_tile.argtypes = [vp, i32, i64]
            lib.jp_set_gemm_tile.restype = i32
            lib.jp_get_gemm_tile.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)]
            lib.jp_get_gemm_tile.restype = i32
            lib.jp_set_stream.argtypes = [vp, vp]
            lib.jp_set_stream.restype = i32
            lib.jp_two_path.argtypes = [vp, ctypes.POINTER(jp_rel), ctypes.POINTER(jp_rel),
                                        ctypes.POINTER(jp_result)]
            lib.jp_two_path.restype = i32
            lib.jp_two_path_into.argtypes = [vp, ctypes.POINTER(jp_rel), ctypes.POINTER(jp_rel), vp,
                                             vp, i64, ctypes.POINTER(ctypes.c_int64)]
            lib.jp_two_path_into.restype = i32
            lib.jp_two_path_batch.argtypes = [vp, ctypes.POINTER(jp_rel), ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(jp_result),
                                              ctypes.POINTER(ctypes.c_int64)]
            lib.jp_two_path_batch.restype = i32
            lib.jp_two_path_filter.argtypes = [vp, ctypes.POINTER(jp_rel), ctypes.POINTER(jp_rel),
                                               ctypes.POINTER(jp_rel), ctypes.POINTER(jp_result)]
            lib.jp_two_path_filter.restype = i32
            lib.jp_two_path_counts.argtypes = [vp, ctypes.POINTER(jp_rel), ctypes.POINTER(jp_rel),
                                               i64, i32, ctypes.POINTER(jp_result)]
            lib.jp_two_path_counts.restype = i32
            lib.jp_set_count_chunk.argtypes = [vp, i64]
            lib.jp_set_count_chunk.restype = i32
            lib.jp_selftest_wait.argtypes = [vp, i64]
            lib.jp_selftest_wait.restype = i32
            dp = ctypes.POINTER(ctypes.c_double)
            lib.jp_measure_peaks.argtypes = [vp, dp, dp]
            lib.jp_measure_peaks.restype = i32
            lib.jp_star_batch.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(jp_rel),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(jp_result),
                                          ctypes.POINTER(ctypes.c_int64)]
            lib.jp_star_batch.restype = i32
            lib.jp_star.argtypes = [vp, i32, ctypes.POINTER(jp_rel), ctypes.POINTER(jp_result)]
            lib.jp_star.restype = i32
            lib.jp_get_stats.argtypes = [vp, ctypes.POINTER(jp_stats)]
            lib.jp_get_stats.restype = i32
            lib.jp_result_to_host.argtypes = [vp, ctypes.POINTER(jp_result),
                                              ctypes.POINTER(ctypes.c_void_p)]
            lib.jp_result_to_host.restype = i32
            lib.jp_result_free.argtypes = [vp, ctypes.POINTER(jp_result)]
            lib.jp_result_free.restype = None
            lib.jp_last_error.argtypes = [vp]
            lib.jp_last_error.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def _rel_of(x, y) -> jp_rel:
    import torch
    for t in (x, y):
        if t.dtype != torch.int32 or not t.is_contiguous():
            raise TypeError("relation columns must be contiguous int32 tensors")
    if x.numel() != y.numel():
        raise ValueError("relation columns differ in length")
    return jp_rel(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.numel())


class Context:
    """One jp_ctx on one CUDA device, issuing work on one stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self._torch = torch
        self.lib = load()
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._live = {}

        def _alloc(nbytes, _stream, _user):
            try:
                t = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
            except RuntimeError:
                return None
            p = t.data_ptr()
            self._live[p] = t
            return p

        def _free(ptr, _nbytes, _stream, _user):
            self._live.pop(ptr, None)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            rc = self.lib.jp_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream),
                                    self._alloc_cb, self._free_cb, None)
        if rc != JP_OK:
            raise JPError(rc, "jp_create failed")
        self.h = h
        table = os.path.join(PKG, "predictor", "gemm_tiles.json")
        if os.path.exists(table):     # the tile autotuner's crossover (tune.py)
            import json
            with open(table) as f:
                self.set_gemm_tile(0, int(json.load(f)["auto_max_tiles"]))

    def close(self):
        if getattr(self, "h", None):
            with self._torch.cuda.stream(self.stream):
                self.lib.jp_destroy(self.h)
            self.h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != JP_OK:
            raise JPError(rc, self.lib.jp_last_error(self.h).decode())

    def set_threshold(self, mode="closed_form", delta1: int = 1, delta2: int = 1):
        m = _MODES[mode] if isinstance(mode, str) else int(mode)
        self._check(self.lib.jp_set_threshold(self.h, m, int(delta1), int(delta2)))

    def set_cost_model(self, **consts):
        """Replace Algorithm 3's constants (jp_set_cost_model); no argument restores the
        defaults, keyword arguments change the named constants of the current set."""
        if not consts:
            self._check(self.lib.jp_set_cost_model(self.h, None))
            return
        m = jp_cost_model()
        self._check(self.lib.jp_get_cost_model(self.h, ctypes.byref(m)))
        for k, v in consts.items():
            if k not in dict(jp_cost_model._fields_):
                raise KeyError(k)
            setattr(m, k, float(v))
        self._check(self.lib.jp_set_cost_model(self.h, ctypes.byref(m)))

    def set_gemm_tile(self, width: int = 0, auto_max_tiles: int = 32):
        """jp_set_gemm_tile: product tile width 128 or 256, or 0 (auto: 128 up to
        auto_max_tiles tiles of 128 x 256)."""
        self._check(self.lib.jp_set_gemm_tile(self.h, int(width), int(auto_max_tiles)))

    def gemm_tile(self):
        w, t = ctypes.c_int(), ctypes.c_int64()
        self._check(self.lib.jp_get_gemm_tile(self.h, ctypes.byref(w), ctypes.byref(t)))
        return w.value, t.value

    def cost_model(self) -> dict:
        """The context's current Algorithm 3 constants (jp_get_cost_model)."""
        m = jp_cost_model()
        self._check(self.lib.jp_get_cost_model(self.h, ctypes.byref(m)))
        return {k: getattr(m, k) for k, _ in jp_cost_model._fields_}

    def _take(self, res: jp_result):
        """Wrap result columns as int32 tensors viewing the library's block."""
        torch = self._torch
        k, n = res.k, res.count
        if n == 0:
            self.lib.jp_result_free(self.h, ctypes.byref(res))
            return tuple(torch.empty(0, dtype=torch.int32, device=self.device) for _ in range(k))
        blk = self._live.get(res._block)
        if blk is None:
            raise RuntimeError("result block was not allocated through this context")
        cols = []
        for i in range(k):
            off = res.col[i] - res._block
            cols.append(blk[off:off + 4 * n].view(torch.int32))
        self.lib.jp_result_free(self.h, ctypes.byref(res))   # the views keep the storage
        return tuple(cols)

    def two_path(self, rx, ry, sz=None, sy=None):
        """Sorted distinct (x, z) of Q(x,z) = R(x,y), S(z,y); S defaults to R."""
        R = _rel_of(rx, ry)
        S = _rel_of(sz, sy) if sz is not None else None
        res = jp_result()
        with self._torch.cuda.stream(self.stream):
            rc = self.lib.jp_two_path(self.h, ctypes.byref(R), ctypes.byref(S) if S else None,
                                      ctypes.byref(res))
        self._check(rc)
        return self._take(res)

    def two_path_into(self, rx, ry, out_x, out_z, sz=None, sy=None) -> int:
        """jp_two_path_into: the sorted distinct pairs written into out_x / out_z (int32
        tensors on this device, or pinned CPU tensors written directly over the host link).
        Returns the pair count; raises JPError(JP_EOVERFLOW) with ``.count`` set when the
        buffers are too small."""
        for t in (out_x, out_z):
            if t.dtype != self._torch.int32 or not t.is_contiguous():
                raise TypeError("output columns must be contiguous int32 tensors")
        R = _rel_of(rx, ry)
        S = _rel_of(sz, sy) if sz is not None else None
        cnt = ctypes.c_int64(0)
        cap = min(out_x.numel(), out_z.numel())
        with self._torch.cuda.stream(self.stream):
            rc = self.lib.jp_two_path_into(self.h, ctypes.byref(R), ctypes.byref(S) if S else None,
                                           ctypes.c_void_p(out_x.data_ptr()),
                                           ctypes.c_void_p(out_z.data_ptr()), cap, ctypes.byref(cnt))
        if rc != JP_OK:
            err = JPError(rc, self.lib.jp_last_error(self.h).decode())
            err.count = cnt.value
            raise err
        return cnt.value

    def two_path_filter(self, tx, tz, rx, ry, sz=None, sy=None):
        """Pairs (a, b) of T = (tx, tz) with R(a, y), S(b, y) for some y: sorted, distinct."""
        R = _rel_of(rx, ry)
        S = _rel_of(sz, sy) if sz is not None else None
        T = _rel_of(tx, tz)
        res = jp_result()
        with self._torch.cuda.stream(self.stream):
            rc = self.lib.jp_two_path_filter(self.h, ctypes.byref(R),
                                             ctypes.byref(S) if S else None, ctypes.byref(T),
                                             ctypes.byref(res))
        self._check(rc)
        return self._take(res)

    def two_path_counts(self, rx, ry, sz=None, sy=None, c_min: int = 1, order: str = "pairs"):
        """Pairs (a, c) sharing at least c_min y, with the count: (x, z, count) columns.

        ``order`` is "pairs" ((x, z) ascending) or "count" (count descending, ties in
        (x, z) order).
        """
        R = _rel_of(rx, ry)
        S = _rel_of(sz, sy) if sz is not None else None
        o = {"pairs": 0, "count": 1}[order]
        res = jp_result()
        with self._torch.cuda.stream(self.stream):
            rc = self.lib.jp_two_path_counts(self.h, ctypes.byref(R),
                                             ctypes.byref(S) if S else None, int(c_min), o,
                                             ctypes.byref(res))
        self._check(rc)
        return self._take(res)

    def set_count_chunk(self, candidates: int):
        self._check(self.lib.jp_set_count_chunk(self.h, int(candidates)))

    def measure_peaks(self) -> dict:
        """Measured dense tensor rates (TFLOP/s): tcgen05 FP8 and INT8 mma.sync."""
        f8, i8 = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.jp_measure_peaks(self.h, ctypes.byref(f8), ctypes.byref(i8)))
        return {"fp8_tcgen05_tflops": f8.value, "int8_mma_sync_tflops": i8.value}

    def selftest_wait(self, wait_ns: int) -> int:
        """Run the bounded-wait self-test; returns the library's code (JP_ETIMEOUT expected)."""
        rc = self.lib.jp_selftest_wait(self.h, int(wait_ns))
        self._torch.cuda.synchronize(self.device)
        return rc

    def two_path_batch(self, x, y, qoff):
        """Batch of self-joins: query q is tuples [qoff[q], qoff[q+1]) of (x, y).

        Returns (ox, oz, out_off): the queries' sorted distinct pairs one after
        another and, as a numpy int64 array of nq + 1 entries, where each
        query's pairs start.
        """
        import numpy as np
        qoff = np.ascontiguousarray(qoff, dtype=np.int64)
        nq = len(qoff) - 1
        out_off = np.zeros(nq + 1, np.int64)
        R = _rel_of(x, y)
        res = jp_result()
        i64p = ctypes.POINTER(ctypes.c_int64)
        with self._torch.cuda.stream(self.stream):
            rc = self.lib.jp_two_path_batch(self.h, ctypes.byref(R), nq,
                                            qoff.ctypes.data_as(i64p), ctypes.byref(res),
                                            out_off.ctypes.data_as(i64p))
        self._check(rc)
        ox, oz = self._take(res)
        return ox, oz, out_off

    def star(self, rels):
        """Sorted distinct k-tuples of Q*_k over ``rels = [(x1, y1), ...]``."""
        k = len(rels)
        arr = (jp_rel * k)(*[_rel_of(x, y) for x, y in rels])
        res = jp_result()
        with self._torch.cuda.stream(self.stream):
            rc = self.lib.jp_star(self.h, k, arr, ctypes.byref(res))
        self._check(rc)
        return self._take(res)

    def star_batch(self, queries):
        """jp_star_batch: ``queries`` is a list of star queries, each three relations
        ``[(x1, y1), (x2, y2), (x3, y3)]`` of int32 tensors (all on this device, or all on the
        host).  Returns (c0, c1, c2, out_off): the queries' sorted distinct triples one after
        another and, as a numpy int64 array of nq + 1 entries, where each query's start."""
        import numpy as np
        torch = self._torch
        nq = len(queries)
        qoff = np.zeros((3, nq + 1), np.int64)
        cols = []
        for i in range(3):
            xs = [q[i][0] for q in queries]
            ys = [q[i][1] for q in queries]
            qoff[i, 1:] = np.cumsum([x.numel() for x in xs])
            cols.append((torch.cat(xs).contiguous(), torch.cat(ys).contiguous()))
        rels = (jp_rel * 3)(*[_rel_of(x, y) for x, y in cols])
        out_off = np.zeros(nq + 1, np.int64)
        res = jp_result()
        i64p = ctypes.POINTER(ctypes.c_int64)
        with torch.cuda.stream(self.stream):
            rc = self.lib.jp_star_batch(self.h, nq, rels, qoff.ctypes.data_as(i64p),
                                        ctypes.byref(res), out_off.ctypes.data_as(i64p))
        self._check(rc)
        if res.count == 0:
            self.lib.jp_result_free(self.h, ctypes.byref(res))
            e = torch.empty(0, dtype=torch.int32, device=self.device)
            return e, e.clone(), e.clone(), out_off
        c0, c1, c2 = self._take(res)
        return c0, c1, c2, out_off

    def two_path_host(self, rx, ry, out_cols=None, timings=None):
        """End-to-end call with HOST input columns (pinned torch CPU tensors).

        The library copies the inputs to the device; the result is copied
        back into pinned host tensors with jp_result_to_host.  If ``timings``
        is a dict it receives the wall seconds of the query call ("query"),
        the copy to host ("to_host") and the release ("free").
        """
        import time
        torch = self._torch
        R = _rel_of(rx, ry)
        res = jp_result()
        t0 = time.perf_counter()
        with torch.cuda.stream(self.stream):
            self._check(self.lib.jp_two_path(self.h, ctypes.byref(R), None, ctypes.byref(res)))
        t1 = time.perf_counter()
        n = res.count
        if out_cols is None or out_cols[0].numel() < n:
            out_cols = [torch.empty(max(n, 1), dtype=torch.int32, pin_memory=True) for _ in range(2)]
        ptrs = (ctypes.c_void_p * 2)(out_cols[0].data_ptr(), out_cols[1].data_ptr())
        t2 = t1
        try:
            self._check(self.lib.jp_result_to_host(self.h, ctypes.byref(res), ptrs))
            t2 = time.perf_counter()
        finally:
            self.lib.jp_result_free(self.h, ctypes.byref(res))
        if timings is not None:
            t3 = time.perf_counter()
            timings["query"] = timings.get("query", 0.0) + (t1 - t0)
            timings["to_host"] = timings.get("to_host", 0.0) + (t2 - t1)
            timings["free"] = timings.get("free", 0.0) + (t3 - t2)
        return out_cols[0][:n], out_cols[1][:n]

    def stats(self) -> dict:
        s = jp_stats()
        self._check(self.lib.jp_get_stats(self.h, ctypes.byref(s)))
        arrays = ("ms_pass", "light_x", "light_cand", "light_deg")
        d = {name: getattr(s, name) for name, _ in jp_stats._fields_ if name not in arrays}
        for name in arrays:
            d[name] = list(getattr(s, name))
        return d


# ------------------------------------------------------------------ predictor
JP_LEARNED = 3
JP_MLP_PARAMS = 99330
JP_MLP_MAX_BATCH = 1024
_MODES["learned"] = JP_LEARNED


def _bind_predictor(lib):
    if getattr(lib, "_pred_bound", False):
        return lib
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    fp = ctypes.POINTER(ctypes.c_float)
    lib.jp_features.argtypes = [vp, ctypes.POINTER(jp_rel), ctypes.POINTER(jp_rel), fp]
    lib.jp_features.restype = i32
    lib.jp_set_predictor.argtypes = [vp, vp]
    lib.jp_set_predictor.restype = i32
    lib.jp_mlp_create.argtypes = [ctypes.POINTER(vp), i32, vp]
    lib.jp_mlp_create.restype = i32
    lib.jp_mlp_destroy.argtypes = [vp]
    lib.jp_mlp_destroy.restype = None
    lib.jp_mlp_set_params.argtypes = [vp, fp, i64]
    lib.jp_mlp_set_params.restype = i32
    lib.jp_mlp_get_params.argtypes = [vp, fp, i64]
    lib.jp_mlp_get_params.restype = i32
    lib.jp_mlp_forward.argtypes = [vp, fp, i32, fp]
    lib.jp_mlp_forward.restype = i32
    lib.jp_mlp_gradients.argtypes = [vp, fp, fp, i32, fp, fp]
    lib.jp_mlp_gradients.restype = i32
    lib.jp_mlp_train_step.argtypes = [vp, fp, fp, i32, ctypes.c_float, fp]
    lib.jp_mlp_train_step.restype = i32
    lib._pred_bound = True
    return lib


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Predictor:
    """The learned threshold predictor (jp_mlp_*): features -> (ln D1, ln D2)."""

    def __init__(self, device: int = 0, stream=None):
        import numpy as np
        import torch
        self._np = np
        self.lib = _bind_predictor(load())
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        rc = self.lib.jp_mlp_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream))
        if rc != JP_OK:
            raise JPError(rc, "jp_mlp_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.jp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != JP_OK:
            raise JPError(rc, what)

    @classmethod
    def trained(cls, device: int = 0, stream=None):
        """A predictor holding the shipped parameters (predictor/params.npy,
        written by ``python -m paper_2002_12459_gb300.learn --out``)."""
        import numpy as np
        p = cls(device, stream)
        p.set_params(np.load(os.path.join(PKG, "predictor", "params.npy")))
        return p

    def set_params(self, params):
        p = self._np.ascontiguousarray(params, dtype=self._np.float32).ravel()
        self._check(self.lib.jp_mlp_set_params(self.h, _fptr(p), p.size), "jp_mlp_set_params")

    def get_params(self):
        p = self._np.empty(JP_MLP_PARAMS, self._np.float32)
        self._check(self.lib.jp_mlp_get_params(self.h, _fptr(p), p.size), "jp_mlp_get_params")
        return p

    def forward(self, X):
        X = self._np.ascontiguousarray(X, dtype=self._np.float32)
        Y = self._np.empty((X.shape[0], 2), self._np.float32)
        self._check(self.lib.jp_mlp_forward(self.h, _fptr(X), X.shape[0], _fptr(Y)), "jp_mlp_forward")
        return Y

    def gradients(self, X, T):
        X = self._np.ascontiguousarray(X, dtype=self._np.float32)
        T = self._np.ascontiguousarray(T, dtype=self._np.float32)
        g = self._np.empty(JP_MLP_PARAMS, self._np.float32)
        loss = self._np.zeros(1, self._np.float32)
        self._check(self.lib.jp_mlp_gradients(self.h, _fptr(X), _fptr(T), X.shape[0], _fptr(g),
                                              _fptr(loss)), "jp_mlp_gradients")
        return g, float(loss[0])

    def train_step(self, X, T, lr):
        X = self._np.ascontiguousarray(X, dtype=self._np.float32)
        T = self._np.ascontiguousarray(T, dtype=self._np.float32)
        loss = self._np.zeros(1, self._np.float32)
        self._check(self.lib.jp_mlp_train_step(self.h, _fptr(X), _fptr(T), X.shape[0],
                                               ctypes.c_float(lr), _fptr(loss)), "jp_mlp_train_step")
        return float(loss[0])


def _context_features(self, rx, ry, sz=None, sy=None):
    """The 128 predictor features of the query on R (and S)."""
    import numpy as np
    _bind_predictor(self.lib)
    R = _rel_of(rx, ry)
    S = _rel_of(sz, sy) if sz is not None else None
    out = np.empty(128, np.float32)
    with self._torch.cuda.stream(self.stream):
        rc = self.lib.jp_features(self.h, ctypes.byref(R), ctypes.byref(S) if S else None, _fptr(out))
    self._check(rc)
    return out


def _context_set_predictor(self, pred):
    _bind_predictor(self.lib)
    self._predictor = pred
    self._check(self.lib.jp_set_predictor(self.h, pred.h if pred is not None else None))


Context.features = _context_features
Context.set_predictor = _context_set_predictor
