"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU,
exports every function declared in include/kohler.h, and the binding refuses to
run when the library is missing (there is no fallback)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kohler.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|int32_t|const char\s*\*)\s+(kohler_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1707_05062_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("kohler_curve", "kohler_curve_batch", "kohler_thresholds", "kohler_submit", "kohler_poll",
                     "kohler_analyze_batch", "kohler_analyze_host", "kohler_server_create", "kohler_server_destroy",
                     "kohler_strerror", "kohler_stream_status", "kohler_segment", "kohler_autotune",
                     "kohler_tune_save", "kohler_tune_load", "kohler_tune_clear", "kohler_tune_count"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_strerror_without_gpu(lib_path):
    L = ctypes.CDLL(lib_path)
    L.kohler_strerror.restype = ctypes.c_char_p
    L.kohler_strerror.argtypes = [ctypes.c_int]
    assert L.kohler_strerror(0) == b"ok"
    assert L.kohler_strerror(-3) == b"pixel value >= M"
    assert L.kohler_strerror(12345) == b"unknown status"


def test_argument_errors_without_gpu(lib_path):
    # argument checks run before any CUDA call
    L = ctypes.CDLL(lib_path)
    L.kohler_curve.restype = ctypes.c_int
    p, i64, i32, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
    L.kohler_curve.argtypes = [p, i, i64, i64, i64, i32, i, p, p, p, p]
    assert L.kohler_curve(None, 1, 8, 8, 8, 256, 4, None, None, None, None) == -1
    assert L.kohler_curve(1024, 1, 8, 8, 8, 256, 5, None, None, None, None) == -2  # no 5-neighbourhood: unsupported
    assert L.kohler_curve(1024, 1, 8, 8, 8, 257, 4, None, None, None, None) == -1
    assert L.kohler_curve(1024, 2, 8, 8, 15, 4096, 4, None, None, None, None) == -1
    L.kohler_server_create.restype = ctypes.c_int
    L.kohler_server_create.argtypes = [p, i32, i32, ctypes.c_size_t, i32]
    assert L.kohler_server_create(None, 256, 4, 0, 0) == -1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_1707_05062_gb300 as k

    monkeypatch.setattr(k, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(k, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        k.lib()


def test_segment_argument_errors_without_gpu(lib_path):
    L = ctypes.CDLL(lib_path)
    L.kohler_segment.restype = ctypes.c_int
    p, i64, i32, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
    L.kohler_segment.argtypes = [p, i, i64, i64, i64, i32, p, p, i32, p, i64, p]
    assert L.kohler_segment(None, 1, 8, 8, 8, 256, None, None, 0, 4096, 8, None) == -1   # no image
    assert L.kohler_segment(1024, 1, 8, 8, 8, 256, None, None, 0, None, 8, None) == -1   # no output
    assert L.kohler_segment(1024, 1, 8, 8, 8, 300, None, None, 0, 4096, 8, None) == -1   # M > 256 for uint8
    assert L.kohler_segment(1024, 1, 8, 8, 4, 256, None, None, 0, 4096, 8, None) == -1   # pitch < width
    assert L.kohler_segment(1024, 1, 8, 8, 8, 256, None, None, 3, 4096, 8, None) == -1   # thresholds missing
