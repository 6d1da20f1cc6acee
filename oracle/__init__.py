"""CPU oracle for the join-project path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and its ``--impl reference`` arm) may import this
package.  The product library never calls it and shares no code with it; the
two meet only in the seeded input generators of
``paper_2002_12459_gb300.workloads``, which hold none of the method's
arithmetic.

Contents:

* ``two_path`` / ``star`` / ``two_path_row`` / ``two_path_rows``: the plain definition of the
  queries (Section 2.1) in C (``jp_oracle.c``): sort-based hash join on y,
  projection, sort and unique.  Exact, integer only.
* ``brute_two_path`` / ``brute_star``: pure-Python triple loops over the
  active domain, for tiny inputs only (used to pin the C oracle).
* ``algorithm1``: Algorithm 1 step by step in the paper's order (partition,
  light join, heavy matrices, matrix product, union), used to pin the worked
  example's matrices and the heavy dimensions.
* ``bsi`` / ``brute_bsi``: the batch of boolean set intersection queries of
  Section 3.3, Q_batch(x,z) = R(x,y), S(z,y), T(x,z), as the three-way join
  followed by the projection on (x, z) (numpy), and as a pure-Python loop over
  T for tiny inputs.
* ``ssj`` / ``brute_ssj``: the set similarity join (Section 1) -- pairs whose
  sets share at least c values, with the count -- in (x, z) order or by
  decreasing count (Section 4, "Ordered SSJ"), from the C oracle's witness
  counts, and as pure-Python set intersections for tiny inputs.
* ``cost_model``: the threshold formulas (Section 3.1 closed forms, the
  Section 3.2 star cost, the Section 5 output estimate and Algorithm 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

__all__ = ["build", "two_path", "star", "two_path_row", "two_path_rows", "brute_two_path",
           "brute_star", "normalise", "bsi", "brute_bsi", "ssj", "brute_ssj"]


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (a checker, not the product)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.oracle_two_path.restype = ctypes.c_int64
            lib.oracle_two_path.argtypes = [i32p, i32p, ctypes.c_int64, i32p, i32p, ctypes.c_int64,
                                            ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p,
                                            ctypes.c_int64]
            lib.oracle_star.restype = ctypes.c_int64
            lib.oracle_star.argtypes = [ctypes.c_int, ctypes.POINTER(i32p), ctypes.POINTER(i32p),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                        ctypes.c_int32, ctypes.POINTER(i32p), ctypes.c_int64]
            lib.oracle_two_path_row.restype = ctypes.c_int64
            lib.oracle_two_path_row.argtypes = [i32p, ctypes.c_int64, i32p, i32p, ctypes.c_int64,
                                                i32p, ctypes.c_int64]
            lib.oracle_two_path_rows.restype = ctypes.c_int64
            lib.oracle_two_path_rows.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                                                 i32p, i32p, i32p, ctypes.c_int64, i32p,
                                                 ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
            lib.oracle_sort_by_y.restype = ctypes.c_int64
            lib.oracle_sort_by_y.argtypes = [i32p, i32p, ctypes.c_int64, i32p, i32p]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


I32_MIN = -(1 << 31)
I32_MAX = (1 << 31) - 1


def two_path(rx, ry, sz=None, sy=None, x_lo: int = I32_MIN, x_hi: int = I32_MAX,
             with_counts: bool = False):
    """Sorted distinct (x, z) of Q(x,z) = R(x,y), S(z,y) with x in [x_lo, x_hi].

    ``sz/sy`` default to R (self-join).  With ``with_counts`` also returns the
    number of distinct witnesses y of every pair.
    """
    lib = _load()
    rx, ry = _i32(rx), _i32(ry)
    if sz is None:
        sz, sy = rx, ry
    sz, sy = _i32(sz), _i32(sy)
    cap = 1 << 16
    while True:
        ox = np.empty(cap, np.int32)
        oz = np.empty(cap, np.int32)
        oc = np.empty(cap, np.int32) if with_counts else None
        n = lib.oracle_two_path(_p(rx), _p(ry), len(rx), _p(sz), _p(sy), len(sz),
                                x_lo, x_hi, _p(ox), _p(oz),
                                _p(oc) if with_counts else None, cap)
        if n < 0:
            raise MemoryError("oracle_two_path ran out of memory")
        if n <= cap:
            out = (ox[:n], oz[:n])
            return out + (oc[:n],) if with_counts else out
        cap = int(n)


def star(rels, x_lo: int = I32_MIN, x_hi: int = I32_MAX):
    """Sorted distinct tuples of Q*_k over ``rels = [(x1, y1), ..., (xk, yk)]``."""
    lib = _load()
    k = len(rels)
    xs = [_i32(r[0]) for r in rels]
    ys = [_i32(r[1]) for r in rels]
    i32p = ctypes.POINTER(ctypes.c_int32)
    XA = (i32p * k)(*[_p(a) for a in xs])
    YA = (i32p * k)(*[_p(a) for a in ys])
    NA = (ctypes.c_int64 * k)(*[len(a) for a in xs])
    cap = 1 << 16
    while True:
        outs = [np.empty(cap, np.int32) for _ in range(k)]
        OA = (i32p * k)(*[_p(a) for a in outs])
        n = lib.oracle_star(k, XA, YA, NA, x_lo, x_hi, OA, cap)
        if n < 0:
            raise MemoryError("oracle_star failed")
        if n <= cap:
            return tuple(o[:n] for o in outs)
        cap = int(n)


class SortedS:
    """S deduplicated and sorted by (y, z), for per-row oracle queries."""

    def __init__(self, sz, sy):
        lib = _load()
        sz, sy = _i32(sz), _i32(sy)
        oy = np.empty(len(sz), np.int32)
        oz = np.empty(len(sz), np.int32)
        m = lib.oracle_sort_by_y(_p(sz), _p(sy), len(sz), _p(oy), _p(oz))
        if m < 0:
            raise MemoryError
        self.y = np.ascontiguousarray(oy[:m])
        self.z = np.ascontiguousarray(oz[:m])


def two_path_row(r_y_of_a, s_sorted: SortedS) -> np.ndarray:
    """Sorted distinct z with (a, y) in R and (z, y) in S, given a's y values."""
    lib = _load()
    ya = _i32(r_y_of_a)
    cap = 1 << 12
    while True:
        out = np.empty(cap, np.int32)
        n = lib.oracle_two_path_row(_p(ya), len(ya), _p(s_sorted.y), _p(s_sorted.z),
                                    len(s_sorted.y), _p(out), cap)
        if n < 0:
            raise MemoryError
        if n <= cap:
            return out[:n]
        cap = int(n)


def two_path_rows(r_off, r_y, s_sorted: SortedS, cap_hint: int = 0):
    """Sorted distinct z of several rows (row i's y values are r_y[r_off[i]:r_off[i+1]]).

    Returns (z values of all rows one after another, int64 count per row).
    """
    lib = _load()
    r_off = np.ascontiguousarray(r_off, dtype=np.int64)
    r_y = _i32(r_y)
    nrows = len(r_off) - 1
    cnt = np.zeros(max(nrows, 1), np.int64)
    cap = max(int(cap_hint), 1 << 12)
    i64p = ctypes.POINTER(ctypes.c_int64)
    while True:
        out = np.empty(cap, np.int32)
        n = lib.oracle_two_path_rows(r_off.ctypes.data_as(i64p), nrows, _p(r_y),
                                     _p(s_sorted.y), _p(s_sorted.z), len(s_sorted.y), _p(out),
                                     cap, cnt.ctypes.data_as(i64p))
        if n < 0:
            raise MemoryError
        if n <= cap:
            return out[:n], cnt[:nrows]
        cap = int(n)


def brute_two_path(rx, ry, sz=None, sy=None):
    """Pure-Python triple loop over (a, c, b): tiny inputs only."""
    if sz is None:
        sz, sy = rx, ry
    R = set(zip(map(int, rx), map(int, ry)))
    S = set(zip(map(int, sz), map(int, sy)))
    xs = sorted({a for a, _ in R})
    zs = sorted({c for c, _ in S})
    bs = sorted({b for _, b in R} | {b for _, b in S})
    out = []
    for a in xs:
        for c in zs:
            for b in bs:
                if (a, b) in R and (c, b) in S:
                    out.append((a, c))
                    break
    return out


def brute_star(rels):
    """Pure-Python enumeration over the active domains: tiny inputs only."""
    import itertools
    sets = [set(zip(map(int, r[0]), map(int, r[1]))) for r in rels]
    doms = [sorted({a for a, _ in s}) for s in sets]
    bs = sorted(set().union(*[{b for _, b in s} for s in sets]))
    out = []
    for t in itertools.product(*doms):
        for b in bs:
            if all((t[i], b) in sets[i] for i in range(len(sets))):
                out.append(t)
                break
    return out


def normalise(x, y):
    """Distinct (x, y) tuples of a relation, sorted; plus per-value degrees."""
    x = np.asarray(x, np.int64)
    y = np.asarray(y, np.int64)
    key = np.unique((x << 32) | (y & 0xFFFFFFFF))
    ux = (key >> 32).astype(np.int32)
    uy = (key & 0xFFFFFFFF).astype(np.uint32).astype(np.int32)
    return ux, uy


def _pair_keys(a, b) -> np.ndarray:
    """int64 keys ordering pairs of int32 lexicographically (signed)."""
    return (np.asarray(a, np.int64) << 32) | (np.asarray(b, np.int64) - I32_MIN)


def bsi(rx, ry, tx, tz, sz=None, sy=None):
    """Sorted distinct (a, b) of Q_batch(x,z) = R(x,y), S(z,y), T(x,z) (Section 3.3).

    The join of T with R on x gives the triples (a, b, y); those whose (b, y)
    is a tuple of S survive; the result is their projection on (a, b).
    """
    if sz is None:
        sz, sy = rx, ry
    rx, ry = normalise(rx, ry)
    sz, sy = normalise(sz, sy)
    tk = np.unique(_pair_keys(tx, tz))
    ta = (tk >> 32).astype(np.int32)
    tb = ((tk & 0xFFFFFFFF) + I32_MIN).astype(np.int32)
    if len(tk) == 0 or len(rx) == 0 or len(sz) == 0:
        return np.empty(0, np.int32), np.empty(0, np.int32)
    # T join R on x: R is sorted by x, so a's tuples are one range
    lo = np.searchsorted(rx, ta, "left")
    hi = np.searchsorted(rx, ta, "right")
    deg = hi - lo
    pair = np.repeat(np.arange(len(tk)), deg)
    start = np.repeat(lo - np.concatenate(([0], np.cumsum(deg)[:-1])), deg)
    y = ry[np.arange(len(pair)) + start]
    # semi-join of the triples with S on (z, y)
    skeys = np.sort(_pair_keys(sz, sy))
    k = _pair_keys(tb[pair], y)
    at = np.minimum(np.searchsorted(skeys, k), len(skeys) - 1)
    hit = np.unique(pair[skeys[at] == k])
    return ta[hit], tb[hit]


def brute_bsi(rx, ry, tx, tz, sz=None, sy=None):
    """Pure-Python loop over the distinct pairs of T: tiny inputs only."""
    if sz is None:
        sz, sy = rx, ry
    R = set(zip(map(int, rx), map(int, ry)))
    S = set(zip(map(int, sz), map(int, sy)))
    out = []
    for a, b in sorted(set(zip(map(int, tx), map(int, tz)))):
        ya = {y for x, y in R if x == a}
        yb = {y for z, y in S if z == b}
        if ya & yb:
            out.append((a, b))
    return out


def ssj(rx, ry, c_min: int = 1, sz=None, sy=None, order: str = "pairs"):
    """(x, z, count) of the pairs whose sets share at least ``c_min`` y values.

    ``order`` "pairs": (x, z) ascending; "count": count descending, equal
    counts in (x, z) order.
    """
    ox, oz, oc = two_path(rx, ry, sz, sy, with_counts=True)
    keep = oc >= c_min
    ox, oz, oc = ox[keep], oz[keep], oc[keep]
    if order == "count":
        perm = np.lexsort((oz, ox, -oc.astype(np.int64)))
        ox, oz, oc = ox[perm], oz[perm], oc[perm]
    return ox, oz, oc


def brute_ssj(rx, ry, c_min: int = 1, sz=None, sy=None):
    """Pure-Python set intersections over every pair of sets: tiny inputs only."""
    if sz is None:
        sz, sy = rx, ry
    A = {}
    for a, b in zip(map(int, rx), map(int, ry)):
        A.setdefault(a, set()).add(b)
    B = {}
    for c, b in zip(map(int, sz), map(int, sy)):
        B.setdefault(c, set()).add(b)
    out = []
    for a in sorted(A):
        for c in sorted(B):
            k = len(A[a] & B[c])
            if k >= c_min:
                out.append((a, c, k))
    return out
