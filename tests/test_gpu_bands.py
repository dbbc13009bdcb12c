"""Row-band split of one image (kohler_band_histograms + kohler_histograms_curve).

Each band is handed over in a buffer of its own that holds only the rows the
band needs (three above it, the band, one below it), as a rank of a multi-GPU
split would hold them; a read outside that buffer would see the tensor copy's
zero fill and change the result.  The summed histograms must give the oracle's
card, sumc, C(t) and thresholds exactly (tolerance zero), for any number of
bands, including empty ones and bands of one row.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
MAX_K = 16


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_05062_gb300 import build

    build.build()
    oracle.build()
    import paper_1707_05062_gb300 as K

    return K


def band_buffer(img: torch.Tensor, r0: int, r1: int, pad: int = 0) -> torch.Tensor:
    """Rows r0 .. r1 - 1 of img in a fresh buffer (row pitch widened by pad bytes)."""
    W = img.shape[1]
    buf = torch.full((r1 - r0, W + pad), 255, dtype=img.dtype, device=img.device)
    buf[:, :W] = img[r0:r1]
    return buf[:, :W]


def split_analyze(K, a: np.ndarray, M: int, n: int, stream, pad: int = 0):
    img = torch.from_numpy(a).cuda()
    H, W = a.shape
    hist = torch.zeros(K.HIST_WORDS, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(stream):
        for y0, y1 in K.row_bands(H, n):
            r0, r1 = K.band_rows(H, y0, y1)
            rows = band_buffer(img, r0, r1, pad)
            stream.synchronize()
            K.band_histograms(rows, r0, H, y0, y1, M, hist, stream=stream)
            stream.synchronize()  # the band's buffer is released before the next band
        out = K.histograms_curve(hist, W, H, M, MAX_K, stream=stream)
    stream.synchronize()
    assert K.stream_status(stream) == 0
    assert not hist.any(), "the histograms are cleared for reuse"
    return [x.cpu().numpy() for x in out]


def check(got, a, M, what):
    card, sumc, c, ts, cnt, t0 = oracle.analyze(a, M, MAX_K)
    assert np.array_equal(got[0].view(np.uint64), card), what
    assert np.array_equal(got[1].view(np.uint64), sumc), what
    assert np.array_equal(got[2], c), what
    assert np.array_equal(got[3], ts) and int(got[4][0]) == cnt and int(got[5][0]) == t0, what


CASES = [
    ("voronoi 1040x777", lambda: synth.voronoi_image(31, 1040, 777, 120, 4.0), 256),
    ("smooth 528x301, M=200", lambda: synth.smooth_image(32, 528, 301, 200), 200),
    ("random 272x64", lambda: synth.random_image(33, 272, 64, 256), 256),
    ("blobs 256x256", lambda: synth.blobs_image(), 256),
]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("name,make,M", CASES, ids=[c[0] for c in CASES])
def test_bands_sum_to_whole_image(K, name, make, M, n):
    a = make()
    got = split_analyze(K, a, M, n, torch.cuda.Stream())
    check(got, a, M, f"{name}, {n} bands")


def test_bands_of_one_row_and_empty_bands(K):
    a = synth.smooth_image(34, 48, 9, 256)
    s = torch.cuda.Stream()
    for n in (9, 13):  # one row per band; four empty bands
        check(split_analyze(K, a, 256, n, s), a, 256, f"{n} bands over 9 rows")
    b = synth.random_image(35, 64, 1, 256)  # a single row: right pairs only
    check(split_analyze(K, b, 256, 2, s), b, 256, "one row, two bands")


def test_bands_with_wider_pitch_and_uneven_split(K):
    a = synth.voronoi_image(36, 800, 450, 60, 3.0)
    s = torch.cuda.Stream()
    check(split_analyze(K, a, 256, 5, s, pad=48), a, 256, "pitch 848")
    # uneven bands given directly
    img = torch.from_numpy(a).cuda()
    H, W = a.shape
    hist = torch.zeros(K.HIST_WORDS, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(s):
        for y0, y1 in ((0, 1), (1, 4), (4, 200), (200, 201), (201, 450)):
            r0, r1 = K.band_rows(H, y0, y1)
            K.band_histograms(band_buffer(img, r0, r1), r0, H, y0, y1, 256, hist, stream=s)
            s.synchronize()
        out = K.histograms_curve(hist, W, H, 256, MAX_K, stream=s)
    s.synchronize()
    check([x.cpu().numpy() for x in out], a, 256, "uneven bands")


def test_band_range_error_and_refusals(K):
    a = synth.smooth_image(37, 64, 40, 100)
    a[25, 7] = 180  # a pixel >= M in the band [20, 30)
    img = torch.from_numpy(a).cuda()
    H, W = a.shape
    s = torch.cuda.Stream()
    hist = torch.zeros(K.HIST_WORDS, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(s):
        K.band_histograms(img[0:21], 0, H, 0, 20, 100, hist, stream=s)
        s.synchronize()
        assert K.stream_status(s) == 0  # the band that does not hold the pixel
        K.band_histograms(img[17:31], 17, H, 20, 30, 100, hist, stream=s)
        s.synchronize()
        assert K.stream_status(s) == K.ERR_RANGE
        assert K.stream_status(s) == 0  # reported once
    lib = K.lib()
    h = hist.data_ptr()
    st = s.cuda_stream
    base = img.data_ptr()
    # rows that do not hold the band's neighbours
    assert lib.kohler_band_histograms(base + 18 * W, 18, 13, 1, W, H, W, 20, 30, 100, 4, h, st) == K.ERR_ARG
    assert lib.kohler_band_histograms(base + 17 * W, 17, 13, 1, W, H, W, 20, 30, 100, 4, h, st) == K.ERR_ARG
    assert lib.kohler_band_histograms(base, 0, 10, 1, W, H, W, 5, 3, 100, 4, h, st) == K.ERR_ARG
    # outside the uint8 strip pass: 8-neighbourhood, width not a multiple of 16
    assert lib.kohler_band_histograms(base, 0, 40, 1, W, H, W, 0, 40, 100, 8, h, st) == K.ERR_UNSUPPORTED
    assert lib.kohler_band_histograms(base, 0, 40, 1, 60, H, W, 0, 40, 100, 4, h, st) == K.ERR_UNSUPPORTED
    assert lib.kohler_histograms_curve(h, 2, W, H, 100, 4, h, h, None, h, h, h, None, st) == K.ERR_UNSUPPORTED
