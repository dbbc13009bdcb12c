"""Python binding of libkohler: Köhler's boundary-contrast curve and thresholds on GB300.

A thin ctypes layer over the C ABI declared in ``include/kohler.h``: it only
marshals arguments.  Every step of the computation runs in the library's CUDA
kernels; PyTorch provides device memory and streams.  There is no CPU fallback:
if ``libkohler.so`` has not been built, every call raises.

Images are 2-D tensors (row-major, unit stride along a row) of dtype
``torch.uint8`` or 16-bit (``torch.uint16`` or ``torch.int16``, read as unsigned).
Curves come back as int64 tensors holding the exact uint64 counts (all values
here stay below 2^63) and a float64 curve.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkohler.so")

KOHLER_U8, KOHLER_U16 = 1, 2
KOHLER_N4 = 4
KOHLER_N6 = 6
KOHLER_N8 = 8
OK, PENDING = 0, 1
ERR_ARG, ERR_UNSUPPORTED, ERR_RANGE, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_BUSY = -1, -2, -3, -4, -5, -6, -7

_lock = threading.Lock()
_lib = None


class KohlerError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = lib().kohler_strerror(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


class KohlerImage(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("width", ctypes.c_int64), ("height", ctypes.c_int64),
                ("pitch_bytes", ctypes.c_int64)]


class KohlerResult(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_int32), ("count", ctypes.c_int32), ("thresholds", ctypes.c_void_p),
                ("latency_s", ctypes.c_double), ("width", ctypes.c_int64), ("height", ctypes.c_int64)]


class KohlerFrame(ctypes.Structure):
    _fields_ = [("host_frame", ctypes.c_void_p), ("width", ctypes.c_int64), ("height", ctypes.c_int64),
                ("pitch_bytes", ctypes.c_int64)]


def lib():
    """The loaded libkohler (raises if it is missing: no fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libkohler.so is not built ({LIB_PATH}); run paper_1707_05062_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            p, i32, i64, i = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int
            L.kohler_curve.argtypes = [p, i, i64, i64, i64, i32, i, p, p, p, p]
            L.kohler_curve_batch.argtypes = [p, i32, i, i32, i, p, p, p, p]
            L.kohler_thresholds.argtypes = [p, p, i32, i32, i32, p, p, p, p]
            L.kohler_analyze_batch.argtypes = [p, i32, i, i32, i, i32, p, p, p, p, p, p, p]
            L.kohler_analyze_host.argtypes = [p, i, i64, i64, i64, i32, i, i32, p, p, p, p, p, p]
            L.kohler_stream_status.argtypes = [p]
            L.kohler_stream_overlap.argtypes = [p, i32]
            L.kohler_band_histograms.argtypes = [p, i64, i64, i, i64, i64, i64, i64, i64, i32, i, p, p]
            L.kohler_histograms_curve.argtypes = [p, i, i64, i64, i32, i32, p, p, p, p, p, p, p, p]
            L.kohler_test_inject.argtypes = [i32, i32]
            L.kohler_segment.argtypes = [p, i, i64, i64, i64, i32, p, p, i32, p, i64, p]
            if hasattr(L, "kohler_analyze_noalloc"):
                L.kohler_analyze_noalloc.argtypes = [p, i, i64, i64, i64, i32, i, i32, p, p, p, p, p, p, p, p]
                L.kohler_analyze_noalloc.restype = i
            L.kohler_autotune.argtypes = [p, i32, i, i32, i, i32, p, ctypes.c_char_p, i64]
            L.kohler_tune_save.argtypes = [ctypes.c_char_p]
            L.kohler_tune_load.argtypes = [ctypes.c_char_p]
            L.kohler_tune_clear.argtypes = []
            L.kohler_tune_count.argtypes = []
            for name in ("kohler_autotune", "kohler_tune_save", "kohler_tune_load", "kohler_tune_clear",
                         "kohler_tune_count"):
                getattr(L, name).restype = i
            L.kohler_release.argtypes = []
            L.kohler_strerror.argtypes = [i]
            L.kohler_strerror.restype = ctypes.c_char_p
            for name in ("kohler_curve", "kohler_curve_batch", "kohler_thresholds", "kohler_analyze_batch",
                         "kohler_analyze_host", "kohler_stream_status", "kohler_release", "kohler_segment",
                         "kohler_stream_overlap", "kohler_test_inject", "kohler_band_histograms",
                         "kohler_histograms_curve"):
                getattr(L, name).restype = i
            if hasattr(L, "kohler_server_create"):
                L.kohler_server_create.argtypes = [p, i32, i32, ctypes.c_size_t, i32]
                L.kohler_server_create_ex.argtypes = [p, i32, i32, ctypes.c_size_t, i32, ctypes.c_size_t]
                L.kohler_submit.argtypes = [p, p, i, i64, i64, i64, p]
                L.kohler_submit_segment.argtypes = [p, p, i, i64, i64, i64, p, i64, p]
                L.kohler_submit_borrowed.argtypes = [p, p, i, i64, i64, i64, p]
                L.kohler_submit_borrowed_many.argtypes = [p, p, i32, i, p, p]
                L.kohler_poll_many.argtypes = [p, p, i32, p, p, i64]
                L.kohler_poll.argtypes = [p, ctypes.c_uint64, p, i64]
                L.kohler_server_curve.argtypes = [p, ctypes.c_uint64, p]
                L.kohler_server_stats.argtypes = [p, p, p, p, p]
                L.kohler_server_destroy.argtypes = [p]
                for name in ("kohler_server_create", "kohler_server_create_ex", "kohler_submit", "kohler_submit_segment",
                             "kohler_submit_borrowed", "kohler_submit_borrowed_many", "kohler_poll_many",
                             "kohler_poll",
                             "kohler_server_curve",
                             "kohler_server_stats", "kohler_server_destroy"):
                    getattr(L, name).restype = i
            _lib = L
    return _lib


FAULT_ALLOC, FAULT_RING_WAIT = 1, 2


def stream_overlap(stream=None, enable: bool = True, pipeline: bool = False):
    """Lets the first kernel of each later call on `stream` start before the
    stream's previous kernel ends (kohler_stream_overlap mode 1), and with
    `pipeline` also runs consecutive one-image uint8 calls side by side on half
    the GPU each (mode 2): only for streams whose kernel before each call does
    not write that call's images."""
    mode = (2 if pipeline else 1) if enable else 0
    _check(lib().kohler_stream_overlap(_stream(stream), mode), "kohler_stream_overlap")


def test_inject(kind: int, count: int):
    """Test hook (kohler_test_inject): host-side injected allocation failures
    (FAULT_ALLOC) or ring-wait failures of the strip pass (FAULT_RING_WAIT)."""
    _check(lib().kohler_test_inject(kind, count), "kohler_test_inject")


HIST_WORDS = 1024  # uint64 words of the histograms of a uint8 image: H_lo, H_hi (256 each), H_s (512)


def row_bands(height: int, n: int):
    """[y0, y1) of n bands of rows covering [0, height), in order (empty bands
    when n > height)."""
    return [(height * k // n, height * (k + 1) // n) for k in range(n)]


def band_rows(height: int, y0: int, y1: int):
    """The rows a band [y0, y1) must hold: three above it, the band, one below."""
    return max(0, y0 - 3), min(height, y1 + 1)


def band_histograms(rows: torch.Tensor, first_row: int, height: int, y0: int, y1: int, M: int,
                    hist: torch.Tensor = None, stream=None) -> torch.Tensor:
    """Adds the histograms of the pairs band [y0, y1) owns to `hist` (int64[1024]
    on the device; allocated and zeroed if None) and returns it.  `rows` holds
    image rows first_row .. first_row + rows.shape[0] - 1 (kohler_band_histograms)."""
    if hist is None:
        hist = torch.zeros(HIST_WORDS, dtype=torch.int64, device=rows.device)
    ptr, w, n, pitch = _image(rows)
    _check(lib().kohler_band_histograms(ptr, first_row, n, _dtype_code(rows), w, height, pitch, y0, y1, M, KOHLER_N4,
                                        hist.data_ptr(), _stream(stream)), "kohler_band_histograms")
    return hist


def histograms_curve(hist: torch.Tensor, width: int, height: int, M: int, max_k: int, *, stream=None):
    """(card, sumc, curve, out_t, count, t0) from summed band histograms
    (kohler_histograms_curve); clears `hist`."""
    dev = hist.device
    card = torch.empty(M, dtype=torch.int64, device=dev)
    sumc = torch.empty(M, dtype=torch.int64, device=dev)
    c = torch.empty(M, dtype=torch.float64, device=dev)
    out_t = torch.empty(max(max_k, 1), dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int32, device=dev)
    t0 = torch.empty(1, dtype=torch.int32, device=dev)
    _check(lib().kohler_histograms_curve(hist.data_ptr(), KOHLER_U8, width, height, M, max_k, card.data_ptr(),
                                         sumc.data_ptr(), c.data_ptr(), out_t.data_ptr(), cnt.data_ptr(),
                                         t0.data_ptr(), None, _stream(stream)), "kohler_histograms_curve")
    return card, sumc, c, out_t[:max_k], cnt, t0


def analyze_row_band(rows: torch.Tensor, first_row: int, width: int, height: int, band, M: int, max_k: int,
                     group=None, stream=None):
    """One rank's part of the row-band split of one image over the ranks of
    `group` (torch.distributed, one band per rank, for instance `row_bands(height,
    world)[rank]`): this band's histograms, one sum over the ranks (the only
    exchange: 1024 int64), then the curve and thresholds, on every rank."""
    hist = band_histograms(rows, first_row, height, band[0], band[1], M, stream=stream)
    reduce_histograms(hist, group)
    return histograms_curve(hist, width, height, M, max_k, stream=stream)


def reduce_histograms(hist: torch.Tensor, group=None) -> torch.Tensor:
    """Sums band histograms (or any per-band counts) over the ranks of `group`
    in place; a no-op without an initialised process group."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(hist, op=dist.ReduceOp.SUM, group=group)
    return hist


def _check(rc: int, what: str):
    if rc != OK:
        raise KohlerError(rc, what)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.uint8:
        return KOHLER_U8
    if t.dtype in (torch.int16, getattr(torch, "uint16", torch.int16)):
        return KOHLER_U16
    raise TypeError(f"image dtype must be uint8 or 16-bit, got {t.dtype}")


def _image(t: torch.Tensor):
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("image must be a 2-D tensor with unit stride along rows")
    return t.data_ptr(), t.shape[1], t.shape[0], t.stride(0) * t.element_size()


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream if hasattr(s, "cuda_stream") else int(s)


def _images(imgs: Sequence[torch.Tensor]):
    arr = (KohlerImage * max(1, len(imgs)))()
    codes = set()
    for k, t in enumerate(imgs):
        if not t.is_cuda:
            raise ValueError("images must be on the GPU")
        ptr, w, h, pitch = _image(t)
        arr[k] = KohlerImage(ptr, w, h, pitch)
        codes.add(_dtype_code(t))
    if len(codes) > 1:
        raise ValueError("all images of a batch must have one dtype")
    return arr, (codes.pop() if codes else KOHLER_U8)


def curve(img: torch.Tensor, M: int, *, with_curve: bool = True, stream=None, nbhd: int = KOHLER_N4):
    """(card, sumc, curve) of one device image: int64[M], int64[M], float64[M] (or None)."""
    dev = img.device
    card = torch.empty(M, dtype=torch.int64, device=dev)
    sumc = torch.empty(M, dtype=torch.int64, device=dev)
    c = torch.empty(M, dtype=torch.float64, device=dev) if with_curve else None
    ptr, w, h, pitch = _image(img)
    _check(lib().kohler_curve(ptr, _dtype_code(img), w, h, pitch, M, nbhd, card.data_ptr(), sumc.data_ptr(),
                              c.data_ptr() if c is not None else None, _stream(stream)), "kohler_curve")
    return card, sumc, c


def curve_batch(imgs: Sequence[torch.Tensor], M: int, *, with_curve: bool = True, stream=None,
                nbhd: int = KOHLER_N4):
    """(card, sumc, curve) of n device images: [n, M] each (curve may be None)."""
    n = len(imgs)
    dev = imgs[0].device if n else torch.device("cuda")
    arr, code = _images(imgs)
    card = torch.empty((n, M), dtype=torch.int64, device=dev)
    sumc = torch.empty((n, M), dtype=torch.int64, device=dev)
    c = torch.empty((n, M), dtype=torch.float64, device=dev) if with_curve else None
    _check(lib().kohler_curve_batch(arr, n, code, M, nbhd, card.data_ptr(), sumc.data_ptr(),
                                    c.data_ptr() if c is not None else None, _stream(stream)), "kohler_curve_batch")
    return card, sumc, c


def thresholds(card: torch.Tensor, sumc: torch.Tensor, max_k: int, *, stream=None):
    """(ranked maxima int32[n, max_k], count int32[n], t0 int32[n]) from exact curves."""
    if card.dim() == 1:
        card, sumc = card[None], sumc[None]
    card, sumc = card.contiguous(), sumc.contiguous()
    n, M = card.shape
    dev = card.device
    out_t = torch.empty((n, max(max_k, 1)), dtype=torch.int32, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    t0 = torch.empty(n, dtype=torch.int32, device=dev)
    _check(lib().kohler_thresholds(card.data_ptr(), sumc.data_ptr(), n, M, max_k, out_t.data_ptr(), cnt.data_ptr(),
                                   t0.data_ptr(), _stream(stream)), "kohler_thresholds")
    return out_t[:, :max_k], cnt, t0


def analyze_batch(imgs: Sequence[torch.Tensor], M: int, max_k: int, *, with_curve: bool = True, stream=None,
                  out=None, nbhd: int = KOHLER_N4):
    """Fused curves and thresholds of n device images (one launch per 128 images).
    Returns (card, sumc, curve, out_t, count, t0); `out` may supply these tensors."""
    n = len(imgs)
    dev = imgs[0].device
    arr, code = _images(imgs)
    if out is None:
        out = (torch.empty((n, M), dtype=torch.int64, device=dev), torch.empty((n, M), dtype=torch.int64, device=dev),
               torch.empty((n, M), dtype=torch.float64, device=dev) if with_curve else None,
               torch.empty((n, max(max_k, 1)), dtype=torch.int32, device=dev),
               torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n, dtype=torch.int32, device=dev))
    card, sumc, c, out_t, cnt, t0 = out
    _check(lib().kohler_analyze_batch(arr, n, code, M, nbhd, max_k, card.data_ptr(), sumc.data_ptr(),
                                      c.data_ptr() if c is not None else None, out_t.data_ptr(), cnt.data_ptr(),
                                      t0.data_ptr(), _stream(stream)), "kohler_analyze_batch")
    return card, sumc, c, out_t[:, :max_k], cnt, t0


def analyze_host(img, M: int, max_k: int, nbhd: int = KOHLER_N4, out=None):
    """Whole path from a host image (numpy array or CPU tensor, pinned is fastest) back
    to host results: (card, sumc, curve, thresholds, count, t0) as numpy arrays and ints.
    `out` (from host_outputs(M, max_k)) supplies the output arrays, for callers that
    repeat the call without allocating."""
    import numpy as np

    if isinstance(img, torch.Tensor):
        if img.is_cuda:
            raise ValueError("analyze_host takes a host image")
        code = _dtype_code(img)
        ptr, w, h, pitch = _image(img)
    else:
        a = np.asarray(img)
        if a.dtype not in (np.uint8, np.uint16) or a.ndim != 2 or a.strides[1] != a.itemsize:
            raise ValueError("host image must be a 2-D uint8/uint16 array with unit stride along rows")
        code = KOHLER_U8 if a.dtype == np.uint8 else KOHLER_U16
        ptr, w, h, pitch = a.ctypes.data, a.shape[1], a.shape[0], a.strides[0]
    if out is not None:
        card, sumc, c, ts, cnt, t0 = out[0], out[1], out[2], out[3], out[4], out[5]
        if (card.shape != (M,) or sumc.shape != (M,) or c.shape != (M,) or ts.size < max_k
                or card.dtype != np.uint64 or sumc.dtype != np.uint64 or c.dtype != np.float64
                or ts.dtype != np.int32 or not isinstance(cnt, np.ndarray) or not isinstance(t0, np.ndarray)):
            raise ValueError("out must come from host_outputs(M, max_k) with the call's M and max_k")
    else:
        card = np.empty(M, np.uint64)
        sumc = np.empty(M, np.uint64)
        c = np.empty(M, np.float64)
        ts = np.empty(max(max_k, 1), np.int32)
        cnt = np.zeros(1, np.int32)
        t0 = np.zeros(1, np.int32)
    _check(lib().kohler_analyze_host(ptr, code, w, h, pitch, M, nbhd, max_k, card.ctypes.data,
                                     sumc.ctypes.data, c.ctypes.data, ts.ctypes.data, cnt.ctypes.data,
                                     t0.ctypes.data), "kohler_analyze_host")
    return card, sumc, c, ts[:max_k], int(cnt[0]), int(t0[0])


def host_outputs(M: int, max_k: int):
    """Output arrays for analyze_host(..., out=...): card, sumc (uint64[M]), curve
    (float64[M]), thresholds (int32[max(max_k, 1)]), count and t0 (int32[1])."""
    import numpy as np

    return (np.empty(M, np.uint64), np.empty(M, np.uint64), np.empty(M, np.float64),
            np.empty(max(max_k, 1), np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32))


def segment(img: torch.Tensor, M: int, thresholds: torch.Tensor, count: torch.Tensor = None, *, out=None,
            stream=None) -> torch.Tensor:
    """The image segmented by `thresholds` (device int32 tensor, any order; entries outside
    [0, M[ ignored; `count`: device int32 scalar, use only its first entries): every pixel
    becomes the mean value of its class, rounded half up.  Returns `out` (same shape and
    dtype as `img`, allocated if not given).  A pixel >= M shows up in stream_status."""
    if not img.is_cuda:
        raise ValueError("image must be on the GPU")
    code = _dtype_code(img)
    ptr, w, h, pitch = _image(img)
    ts = thresholds.to(device=img.device, dtype=torch.int32).contiguous()
    if out is None:
        out = torch.empty_like(img)
    optr, ow, oh, opitch = _image(out)
    if (ow, oh) != (w, h) or out.dtype != img.dtype:
        raise ValueError("out must match the image's shape and dtype")
    cptr = None
    if count is not None:
        count = count.to(device=img.device, dtype=torch.int32)
        cptr = count.data_ptr()
    _check(lib().kohler_segment(ptr, code, w, h, pitch, M, ts.data_ptr() if ts.numel() else None, cptr, ts.numel(),
                                optr, opitch, _stream(stream)), "kohler_segment")
    return out


def stream_status(stream=None) -> int:
    """Deferred status of the calls on a stream (waits for it): OK or ERR_RANGE/ERR_CUDA."""
    return lib().kohler_stream_status(_stream(stream))


def autotune(imgs: Sequence[torch.Tensor], M: int, *, nbhd: int = KOHLER_N4, reps: int = 20, stream=None) -> dict:
    """Times every launch configuration for these device images (up to 128), keeps
    the fastest for later launches of the same kind, and returns the tuner's
    report (per group of images: every candidate's time, exactness and the choice)."""
    import json

    arr, code = _images(imgs)
    buf = ctypes.create_string_buffer(1 << 20)
    _check(lib().kohler_autotune(arr, len(imgs), code, M, nbhd, reps, _stream(stream), buf, len(buf)),
           "kohler_autotune")
    return json.loads(buf.value.decode())


def tune_save(path: str) -> None:
    """Writes the tuned entries to a JSON file."""
    _check(lib().kohler_tune_save(os.fsencode(path)), "kohler_tune_save")


def tune_load(path: str) -> None:
    """Adds the entries of a JSON file written by tune_save."""
    _check(lib().kohler_tune_load(os.fsencode(path)), "kohler_tune_load")


def tune_clear() -> None:
    """Forgets every tuned entry."""
    _check(lib().kohler_tune_clear(), "kohler_tune_clear")


def tune_count() -> int:
    return lib().kohler_tune_count()


def release() -> None:
    _check(lib().kohler_release(), "kohler_release")
