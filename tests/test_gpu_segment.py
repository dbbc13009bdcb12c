"""Parity of the CUDA segmentation (kohler_segment) with the oracle, element by
element and bit-exact: each output pixel is the mean value of its class, rounded
half up (Section 2.1 classes, Fig. 1 caption).  All calls go through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_05062_gb300 import build

    build.build()
    yield


def K():
    import paper_1707_05062_gb300 as k

    return k


def to_dev(img, pad_cols=0, offset=0):
    h, w = img.shape
    src = torch.from_numpy(img.view(np.int16).copy() if img.dtype == np.uint16 else img.copy())
    if pad_cols == 0 and offset == 0:
        return src.cuda()
    buf = torch.zeros(h * (w + pad_cols) + offset + 16, dtype=src.dtype, device="cuda")
    view = buf[offset: offset + h * (w + pad_cols)].view(h, w + pad_cols)[:, :w]
    view.copy_(src.cuda())
    return view


def host(t, dtype):
    a = t.cpu().numpy()
    return a.view(np.uint16) if dtype == np.uint16 else a


def seg_dev(img, M, ts, count=None, pad=0, offset=0, out_pad=0):
    d = to_dev(img, pad, offset)
    t = torch.tensor(ts, dtype=torch.int32, device="cuda")
    out = None
    if out_pad:
        out = torch.zeros((img.shape[0], img.shape[1] + out_pad), dtype=d.dtype, device="cuda")[:, : img.shape[1]]
    c = torch.tensor(count, dtype=torch.int32, device="cuda") if count is not None else None
    r = K().segment(d, M, t, c, out=out)
    torch.cuda.synchronize()
    assert K().stream_status() == K().OK
    return host(r, img.dtype)


SHAPES = [(1, 1), (1, 16), (3, 5), (17, 16), (33, 100), (64, 1000), (7, 2056), (300, 24), (129, 784)]


@pytest.mark.parametrize("h,w", SHAPES)
def test_u8_shapes(h, w):
    img = synth.smooth_image(h + 7 * w, w, h, 256)
    ts = [200, 40, 90, 130, 40, -1, -1]
    assert np.array_equal(seg_dev(img, 256, ts), oracle.segment(img, 256, ts)), f"{h}x{w}"


@pytest.mark.parametrize("pad,offset,out_pad", [(8, 0, 0), (3, 0, 5), (0, 1, 0), (5, 3, 16), (120, 8, 1)])
def test_u8_pitch_offset(pad, offset, out_pad):
    img = synth.smooth_image(77, 264, 37, 256)
    ts = [100, 60]
    assert np.array_equal(seg_dev(img, 256, ts, pad=pad, offset=offset, out_pad=out_pad), oracle.segment(img, 256, ts))


@pytest.mark.parametrize("ts", [[], [-1, -1], [0], [255], [254], [300, 5], [7, 7, 7, 3], list(range(0, 256, 3))])
def test_u8_threshold_sets(ts):
    img = synth.random_image(5, 96, 40, 256)
    assert np.array_equal(seg_dev(img, 256, ts), oracle.segment(img, 256, ts))


@pytest.mark.parametrize("M", [2, 7, 100])
def test_u8_small_M(M):
    img = synth.smooth_image(M, 96, 33, M)
    ts = [M // 2, M - 2, 0]
    assert np.array_equal(seg_dev(img, M, ts), oracle.segment(img, M, ts))


def test_count_limits_the_thresholds():
    img = synth.smooth_image(9, 128, 50, 256)
    ts = [60, 200, 120, 30]
    got = seg_dev(img, 256, ts, count=2)
    assert np.array_equal(got, oracle.segment(img, 256, ts[:2]))
    got0 = seg_dev(img, 256, ts, count=0)
    assert np.array_equal(got0, oracle.segment(img, 256, []))


@pytest.mark.parametrize("M,h,w", [(4096, 33, 132), (4096, 20, 131), (1000, 40, 64), (65536, 9, 37), (20000, 17, 40)])
def test_u16(M, h, w):
    img = synth.smooth_image(M + h, w, h, M, np.uint16)
    ts = [M // 3, M // 2, 2 * M // 3, M + 5, -3]
    assert np.array_equal(seg_dev(img, M, ts), oracle.segment(img, M, ts)), f"M={M} {h}x{w}"
    assert np.array_equal(seg_dev(img, M, ts, pad=3, offset=1), oracle.segment(img, M, ts))


def test_range_error_then_recovery():
    k = K()
    img = synth.smooth_image(3, 64, 16, 100)
    img[7, 33] = 150
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out = k.segment(to_dev(img), 100, torch.tensor([50], dtype=torch.int32, device="cuda"), stream=s)
    assert k.stream_status(s) == k.ERR_RANGE
    assert not out.cpu().any()
    good = synth.smooth_image(4, 64, 16, 100)
    with torch.cuda.stream(s):
        out = k.segment(to_dev(good), 100, torch.tensor([50], dtype=torch.int32, device="cuda"), stream=s)
    assert k.stream_status(s) == k.OK
    assert np.array_equal(out.cpu().numpy(), oracle.segment(good, 100, [50]))


def test_consecutive_calls_reuse_scratch():
    a = synth.smooth_image(1, 200, 90, 256)
    b = synth.random_image(2, 200, 90, 256)
    for _ in range(2):
        assert np.array_equal(seg_dev(a, 256, [100]), oracle.segment(a, 256, [100]))
        assert np.array_equal(seg_dev(b, 256, [30, 220]), oracle.segment(b, 256, [30, 220]))


def test_chained_after_analyze_on_18mp():
    # thresholds and their count stay on the device between the two calls
    k = K()
    img = synth.voronoi_18mp()
    d = torch.from_numpy(img).cuda()
    card, sumc, c, ts, cnt, t0 = k.analyze_batch([d], 256, 6)
    out = k.segment(d, 256, ts[0], cnt[0])
    torch.cuda.synchronize()
    assert k.stream_status() == k.OK
    ots = oracle.analyze(img, 256, 6)[3]
    assert np.array_equal(ts[0].cpu().numpy(), ots)
    assert np.array_equal(out.cpu().numpy(), oracle.segment(img, 256, [t for t in ots if t >= 0]))
