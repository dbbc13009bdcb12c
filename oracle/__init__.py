"""CPU oracle for the Köhler contrast curve — test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it (see ``kohler_oracle.c`` for what each function computes
and which part of the paper it follows).

The C source is compiled with the system C compiler into ``oracle/_build/`` the
first time it is needed (or by :func:`build`), and called through ctypes on
numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kohler_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_RANGE = 0, -1, -3


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile ``kohler_oracle.c`` (gcc -O2 -fopenmp) unless an up-to-date build exists."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = [os.environ.get("CC", "gcc"), "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p, i64, i32, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
            for name in ("oracle_curve", "oracle_curve_n4", "oracle_curve_alg1", "oracle_curve_n8",
                         "oracle_curve_n8half", "oracle_curve_n8_alg1", "oracle_curve_n6", "oracle_curve_n6half",
                         "oracle_curve_n6_alg1"):
                f = getattr(lib, name)
                f.argtypes = [p, i, i64, i64, i64, i32, p, p]
                f.restype = i
            lib.oracle_curve_at.argtypes = [p, i, i64, i64, i64, i32, p, i32, p, p]
            lib.oracle_curve_at.restype = i
            lib.oracle_normalise.argtypes = [p, p, i32, p]
            lib.oracle_normalise.restype = None
            lib.oracle_thresholds.argtypes = [p, p, i32, i32, p, p, p]
            lib.oracle_thresholds.restype = i
            _lib = lib
    return _lib


def _image_args(img: np.ndarray):
    if img.ndim != 2 or img.dtype not in (np.uint8, np.uint16):
        raise ValueError("image must be a 2-D uint8 or uint16 array")
    if img.strides[1] != img.itemsize or img.strides[0] < img.shape[1] * img.itemsize:
        img = np.ascontiguousarray(img)
    h, w = img.shape
    return img, img.itemsize, w, h, img.strides[0]


def _check(rc: int):
    if rc == ERR_RANGE:
        raise OracleError("pixel value >= M")
    if rc != OK:
        raise OracleError(f"oracle returned {rc}")


def _curve_fn(name: str, img: np.ndarray, M: int):
    img, es, w, h, pitch = _image_args(img)
    card = np.zeros(M, np.uint64)
    sumc = np.zeros(M, np.uint64)
    _check(getattr(_load(), name)(img.ctypes.data, es, w, h, pitch, M, card.ctypes.data, sumc.ctypes.data))
    return card, sumc


def curve(img: np.ndarray, M: int):
    """(card, sumc) over N4* pairs, one threshold at a time (Eq. 1-3 with Eq. 9)."""
    return _curve_fn("oracle_curve", img, M)


def curve_n4(img: np.ndarray, M: int):
    """(card, sumc) over ordered pairs of the full 4-neighbourhood (Eq. 1-2 literally)."""
    return _curve_fn("oracle_curve_n4", img, M)


def curve_alg1(img: np.ndarray, M: int):
    """(card, sumc) by Algorithm 1 with per-thread accumulators (Sections 3.1, 3.3)."""
    return _curve_fn("oracle_curve_alg1", img, M)


def curve_n8(img: np.ndarray, M: int):
    """(card, sumc) over ordered pairs of the full 8-neighbourhood (Eq. 1-2 with N8)."""
    return _curve_fn("oracle_curve_n8", img, M)


def curve_n8half(img: np.ndarray, M: int):
    """(card, sumc) over the half 8-neighbourhood N8* (right, down, down-right, down-left)."""
    return _curve_fn("oracle_curve_n8half", img, M)


def curve_n8_alg1(img: np.ndarray, M: int):
    """(card, sumc) by Algorithm 1 over the four N8* translations."""
    return _curve_fn("oracle_curve_n8_alg1", img, M)


def curve_n6(img: np.ndarray, M: int):
    """(card, sumc) over ordered pairs of the full hexagonal 6-neighbourhood (odd rows
    shifted half a pixel right)."""
    return _curve_fn("oracle_curve_n6", img, M)


def curve_n6half(img: np.ndarray, M: int):
    """(card, sumc) over the half 6-neighbourhood N6* (right, down, and down-left on
    even rows or down-right on odd rows)."""
    return _curve_fn("oracle_curve_n6half", img, M)


def curve_n6_alg1(img: np.ndarray, M: int):
    """(card, sumc) by Algorithm 1 over the three N6* translations."""
    return _curve_fn("oracle_curve_n6_alg1", img, M)


def curve_at(img: np.ndarray, M: int, ts):
    """(card, sumc) at the listed thresholds only (N4* pairs)."""
    img, es, w, h, pitch = _image_args(img)
    ts = np.ascontiguousarray(np.asarray(ts, dtype=np.int32))
    card = np.zeros(ts.size, np.uint64)
    sumc = np.zeros(ts.size, np.uint64)
    _check(_load().oracle_curve_at(img.ctypes.data, es, w, h, pitch, M, ts.ctypes.data, ts.size,
                                   card.ctypes.data, sumc.ctypes.data))
    return card, sumc


def normalise(card: np.ndarray, sumc: np.ndarray) -> np.ndarray:
    """C(t) = sumc(t) / card(t) as IEEE doubles, 0.0 where card(t) = 0."""
    card = np.ascontiguousarray(card, dtype=np.uint64)
    sumc = np.ascontiguousarray(sumc, dtype=np.uint64)
    out = np.zeros(card.size, np.float64)
    _load().oracle_normalise(card.ctypes.data, sumc.ctypes.data, card.size, out.ctypes.data)
    return out


def thresholds(card: np.ndarray, sumc: np.ndarray, max_k: int):
    """(ranked local maxima padded with -1 to max_k, total count, t0)."""
    card = np.ascontiguousarray(card, dtype=np.uint64)
    sumc = np.ascontiguousarray(sumc, dtype=np.uint64)
    out_t = np.full(max(max_k, 1), -1, np.int32)
    cnt = ctypes.c_int32(0)
    t0 = ctypes.c_int32(0)
    _check(_load().oracle_thresholds(card.ctypes.data, sumc.ctypes.data, card.size, max_k,
                                     out_t.ctypes.data, ctypes.byref(cnt), ctypes.byref(t0)))
    return out_t[:max_k].copy(), int(cnt.value), int(t0.value)


def analyze(img: np.ndarray, M: int, max_k: int, method: str = "alg1", nbhd: int = 4):
    """Whole path on the CPU: card, sumc, C(t), ranked thresholds, count, t0
    (nbhd 4, 6 or 8: the 4-, hexagonal 6- or 8-neighbourhood)."""
    if nbhd == 8:
        fn = {"alg1": curve_n8_alg1, "def": curve_n8half, "n8": curve_n8}[method]
    elif nbhd == 6:
        fn = {"alg1": curve_n6_alg1, "def": curve_n6half, "n6": curve_n6}[method]
    else:
        fn = {"alg1": curve_alg1, "def": curve, "n4": curve_n4}[method]
    card, sumc = fn(img, M)
    c = normalise(card, sumc)
    ts, cnt, t0 = thresholds(card, sumc, max_k)
    return card, sumc, c, ts, cnt, t0


def segment(img: np.ndarray, M: int, thresholds) -> np.ndarray:
    """Segmentation of an image by a set of thresholds (Section 2.1: the classes
    C_0^t = {f <= t} and C_1^t = {f > t} of one threshold; Fig. 1 and its
    caption: several thresholds, each class shown as the mean value of its
    pixels; Section 4: two-class segmentation of video frames).

    The thresholds in [0, M[ (others dropped), sorted and without repeats,
    t_1 < ... < t_k, cut the grey levels into k + 1 classes: C_0 = {f <= t_1},
    C_i = {t_i < f <= t_{i+1}}, C_k = {f > t_k}; the class of a pixel is the
    number of thresholds strictly below its value.  Every pixel takes the mean
    value of its class, rounded half up to an integer: floor((2 S + n) / (2 n))
    for a class of n pixels whose values sum to S.  Returns an array of the
    image's shape and dtype.  A pixel >= M raises OracleError (range)."""
    f = np.asarray(img)
    if f.ndim != 2 or f.dtype not in (np.uint8, np.uint16):
        raise OracleError("image must be a 2-D uint8/uint16 array")
    if f.size and int(f.max()) >= M:
        raise OracleError(f"oracle returned {ERR_RANGE}")
    ts = sorted({int(t) for t in thresholds if 0 <= int(t) < M})
    v = f.astype(np.int64)
    cls = np.zeros(f.shape, np.int64)
    for t in ts:
        cls += v > t
    out = np.zeros_like(f)
    for c in range(len(ts) + 1):
        mask = cls == c
        n = int(mask.sum())
        if n:
            s = int(v[mask].sum())
            out[mask] = (2 * s + n) // (2 * n)
    return out
