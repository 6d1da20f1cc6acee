"""The C-ABI library loads and exports every symbol include/jp.h declares.

No compute call is made: this runs without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "jp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(jp_[a-z_0-9]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def lib():
    from paper_2002_12459_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("jp_two_path", "jp_star", "jp_set_threshold", "jp_create", "jp_destroy",
              "jp_get_stats", "jp_result_free", "jp_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_null_arguments_are_rejected_without_gpu(lib):
    lib.jp_two_path.restype = ctypes.c_int
    lib.jp_two_path.argtypes = [ctypes.c_void_p] * 4
    assert lib.jp_two_path(None, None, None, None) == -1          # JP_EINVAL
    lib.jp_set_threshold.restype = ctypes.c_int
    lib.jp_set_threshold.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64]
    assert lib.jp_set_threshold(None, 0, 1, 1) == -1
    lib.jp_two_path_batch.restype = ctypes.c_int
    lib.jp_two_path_batch.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.jp_two_path_batch(None, None, 1, None, None, None) == -1
    lib.jp_two_path_filter.restype = ctypes.c_int
    lib.jp_two_path_filter.argtypes = [ctypes.c_void_p] * 5
    assert lib.jp_two_path_filter(None, None, None, None, None) == -1
    lib.jp_two_path_counts.restype = ctypes.c_int
    lib.jp_two_path_counts.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
    assert lib.jp_two_path_counts(None, None, None, 1, 0, None) == -1
    lib.jp_set_count_chunk.restype = ctypes.c_int
    lib.jp_set_count_chunk.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    assert lib.jp_set_count_chunk(None, 1 << 20) == -1
    lib.jp_selftest_wait.restype = ctypes.c_int
    lib.jp_selftest_wait.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    assert lib.jp_selftest_wait(None, 1000) == -1
    lib.jp_measure_peaks.restype = ctypes.c_int
    lib.jp_measure_peaks.argtypes = [ctypes.c_void_p] * 3
    assert lib.jp_measure_peaks(None, None, None) == -1
    lib.jp_set_cost_model.restype = ctypes.c_int
    lib.jp_set_cost_model.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.jp_set_cost_model(None, None) == -1
    lib.jp_get_cost_model.restype = ctypes.c_int
    lib.jp_get_cost_model.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.jp_get_cost_model(None, None) == -1
    lib.jp_last_error.restype = ctypes.c_char_p
    lib.jp_last_error.argtypes = [ctypes.c_void_p]
    assert lib.jp_last_error(None) == b"NULL context"


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2002_12459_gb300 import jp
    monkeypatch.setattr(jp, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        jp.load(str(tmp_path / "missing.so"))
