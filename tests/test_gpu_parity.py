"""Parity of the CUDA library with the CPU oracle, element by element.

card and sumc must be equal as integers, C(t) equal as doubles (tolerance 0:
both sides take the IEEE round-to-nearest quotient of the same two integers),
and the ranked thresholds, their count and t0 equal exactly.  All calls go
through the C ABI (the ctypes binding only marshals arguments).
"""
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

MAX_K = 16


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_05062_gb300 import build

    build.build()
    oracle.build()
    yield


def K():
    import paper_1707_05062_gb300 as k

    return k


def to_dev(img: np.ndarray, pad_cols: int = 0, offset: int = 0) -> torch.Tensor:
    """Device copy of a host image, optionally with a wider pitch and a start offset."""
    h, w = img.shape
    if img.dtype == np.uint16:
        src = torch.from_numpy(img.view(np.int16).copy())
        dt = torch.int16
    else:
        src = torch.from_numpy(img.copy())
        dt = torch.uint8
    if pad_cols == 0 and offset == 0:
        return src.cuda()
    buf = torch.zeros(h * (w + pad_cols) + offset + 16, dtype=dt, device="cuda")
    view = buf[offset: offset + h * (w + pad_cols)].view(h, w + pad_cols)[:, :w]
    view.copy_(src.cuda())
    return view


def u64(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def expect(img: np.ndarray, M: int, method: str = "alg1"):
    return oracle.analyze(img, M, MAX_K, method=method)


def assert_same(got, want, tag=""):
    card, sumc, c, ts, cnt, t0 = got
    ocard, osumc, oc, ots, ocnt, ot0 = want
    assert np.array_equal(card, ocard), f"{tag} card differs at {np.nonzero(card != ocard)[0][:8]}"
    assert np.array_equal(sumc, osumc), f"{tag} sumc differs at {np.nonzero(sumc != osumc)[0][:8]}"
    if c is not None:
        assert np.array_equal(c, oc), f"{tag} curve differs"
    if ts is not None:
        assert np.array_equal(ts, ots), f"{tag} thresholds {ts} != {ots}"
        assert cnt == ocnt and t0 == ot0, f"{tag} count/t0 {cnt},{t0} != {ocnt},{ot0}"


def run_analyze(imgs_dev, M):
    card, sumc, c, ts, cnt, t0 = K().analyze_batch(imgs_dev, M, MAX_K)
    torch.cuda.synchronize()
    out = []
    for i in range(len(imgs_dev)):
        out.append((u64(card[i]), u64(sumc[i]), c[i].cpu().numpy(), ts[i].cpu().numpy(), int(cnt[i]), int(t0[i])))
    return out


def run_curve(img_dev, M):
    card, sumc, c = K().curve(img_dev, M)
    torch.cuda.synchronize()
    return u64(card), u64(sumc), c.cpu().numpy()


# ------------------------------------------------------------------------ shapes and layouts
SHAPES = [(1, 1), (1, 8), (8, 1), (2, 3), (3, 7), (5, 8), (17, 16), (9, 255), (31, 256), (40, 257), (13, 520),
          (64, 1000), (7, 2056), (300, 24)]


@pytest.mark.parametrize("h,w", SHAPES)
@pytest.mark.parametrize("kind", ["smooth", "random"])
def test_u8_shapes(h, w, kind):
    seed = h * 1000 + w
    img = synth.smooth_image(seed, w, h, 256) if kind == "smooth" else synth.random_image(seed, w, h, 256)
    want = expect(img, 256)
    got = run_analyze([to_dev(img)], 256)[0]
    assert_same(got, want, f"{h}x{w}")
    card, sumc, c = run_curve(to_dev(img), 256)
    assert np.array_equal(card, want[0]) and np.array_equal(sumc, want[1]) and np.array_equal(c, want[2])


@pytest.mark.parametrize("pad,offset", [(8, 0), (3, 0), (0, 1), (5, 3), (120, 8)])
def test_u8_pitch_and_offset(pad, offset):
    img = synth.smooth_image(77, 264, 37, 256)
    want = expect(img, 256)
    got = run_analyze([to_dev(img, pad, offset)], 256)[0]
    assert_same(got, want)


@pytest.mark.parametrize("M", [2, 7, 100, 255])
def test_u8_small_M(M):
    img = synth.smooth_image(M, 96, 33, M)
    want = expect(img, M)
    assert_same(run_analyze([to_dev(img)], M)[0], want)
    img2 = synth.smooth_image(M + 1, 93, 21, M)  # generic pass (width not a multiple of 8)
    assert_same(run_analyze([to_dev(img2)], M)[0], expect(img2, M))


# Images whose base, pitch and width are multiples of 16 bytes take the uint8
# route that streams 256-column strips through bulk copies: widths that leave
# a ragged last strip (16 .. 240 columns), one-row and two-row images, pitches
# wider than the row, and M < 256 (range checked on the device).
U8H_SHAPES = [(1, 16), (2, 16), (1, 32), (3, 272), (5, 512), (50, 528), (129, 784), (33, 4112), (300, 5184), (2, 1296)]


@pytest.mark.parametrize("h,w", U8H_SHAPES)
@pytest.mark.parametrize("kind", ["smooth", "random"])
def test_u8_strip_route_shapes(h, w, kind):
    seed = 7 * h + w
    img = synth.smooth_image(seed, w, h, 256) if kind == "smooth" else synth.random_image(seed, w, h, 256)
    assert_same(run_analyze([to_dev(img)], 256)[0], expect(img, 256), f"{h}x{w}")


@pytest.mark.parametrize("M,pad", [(2, 16), (61, 0), (200, 48)])
def test_u8_strip_route_small_M_and_pitch(M, pad):
    img = synth.smooth_image(M + pad, 800, 45, M)
    assert_same(run_analyze([to_dev(img, pad)], M)[0], expect(img, M), f"M={M} pad={pad}")


def test_u8_strip_route_many_rounds():
    # 160 000 strip-rows: every block folds its lane copies more than once
    img = synth.smooth_image(5, 1024, 40000, 256)
    assert_same(run_analyze([to_dev(img)], 256)[0], expect(img, 256), "1024x40000")


@pytest.mark.parametrize("M,h,w", [(4096, 33, 132), (4096, 20, 131), (1000, 40, 64), (300, 17, 30), (65536, 9, 37),
                                   (8192, 12, 40)])
def test_u16(M, h, w):
    img = synth.smooth_image(M + w, w, h, M, np.uint16, noise_sd=24.0)
    want = expect(img, M)
    got = run_analyze([to_dev(img)], M)[0]
    assert_same(got, want, f"u16 M={M}")


def test_u16_pitch_offset():
    img = synth.smooth_image(5, 128, 25, 4096, np.uint16, noise_sd=30.0)
    want = expect(img, 4096)
    assert_same(run_analyze([to_dev(img, 4, 0)], 4096)[0], want)   # pitch 264 B: fast pass
    assert_same(run_analyze([to_dev(img, 3, 0)], 4096)[0], want)   # pitch 262 B: generic pass
    assert_same(run_analyze([to_dev(img, 0, 2)], 4096)[0], want)   # 4-byte offset: generic pass


# ------------------------------------------------------------------------ degenerate images
@pytest.mark.parametrize("shape", [(1, 1), (1, 16), (16, 1), (4, 8), (3, 5)])
def test_constant(shape):
    img = np.full(shape, 93, np.uint8)
    got = run_analyze([to_dev(img)], 256)[0]
    card, sumc, c, ts, cnt, t0 = got
    assert not card.any() and not sumc.any() and not c.any()
    assert cnt == 0 and t0 == -1 and (ts == -1).all()


def test_step_and_checkerboard():
    img = np.zeros((24, 64), np.uint8)
    img[:, 32:] = 201
    assert_same(run_analyze([to_dev(img)], 256)[0], expect(img, 256))
    yy, xx = np.mgrid[0:24, 0:64]
    cb = np.where((xx + yy) % 2 == 0, 3, 250).astype(np.uint8)
    assert_same(run_analyze([to_dev(cb)], 256)[0], expect(cb, 256))
    ramp = np.tile((2 * np.arange(64) % 256).astype(np.uint8), (5, 1))
    assert_same(run_analyze([to_dev(ramp)], 256)[0], expect(ramp, 256))


def test_range_error_u8():
    k = K()
    M = 100
    img = synth.smooth_image(3, 64, 16, M)
    img[7, 33] = 150  # one pixel out of range
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        card, sumc, c, ts, cnt, t0 = k.analyze_batch([to_dev(img)], M, MAX_K, stream=s)
    assert k.stream_status(s) == k.ERR_RANGE
    assert not card.cpu().any() and not sumc.cpu().any()
    assert k.stream_status(s) == k.OK  # the deferred status is consumed
    # a later good image on the same stream is unaffected
    good = synth.smooth_image(4, 64, 16, M)
    with torch.cuda.stream(s):
        out = k.analyze_batch([to_dev(good)], M, MAX_K, stream=s)
    assert k.stream_status(s) == k.OK
    torch.cuda.synchronize()
    assert np.array_equal(u64(out[0][0]), expect(good, M)[0])


@pytest.mark.parametrize("w", [64, 63])
def test_range_error_u16(w):
    k = K()
    img = synth.smooth_image(9, w, 10, 4096, np.uint16)
    img[3, 5] = 5000
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        card, *_ = k.analyze_batch([to_dev(img)], 4096, MAX_K, stream=s)
    assert k.stream_status(s) == k.ERR_RANGE
    assert not card.cpu().any()


def test_bad_arguments():
    k = K()
    img = to_dev(np.zeros((4, 8), np.uint8))
    card = torch.empty(256, dtype=torch.int64, device="cuda")
    L = k.lib()
    assert L.kohler_curve(img.data_ptr(), 1, 8, 4, 8, 1, 4, card.data_ptr(), card.data_ptr(), None, None) == k.ERR_ARG
    assert L.kohler_curve(img.data_ptr(), 1, 8, 4, 7, 256, 4, card.data_ptr(), card.data_ptr(), None, None) == k.ERR_ARG
    assert L.kohler_curve(img.data_ptr(), 1, 0, 4, 8, 256, 4, card.data_ptr(), card.data_ptr(), None, None) == k.ERR_ARG
    assert L.kohler_curve(img.data_ptr(), 1, 8, 4, 8, 300, 4, card.data_ptr(), card.data_ptr(), None, None) == k.ERR_ARG
    assert L.kohler_curve(img.data_ptr(), 1, 8, 4, 8, 256, 5, card.data_ptr(), card.data_ptr(), None, None) == k.ERR_UNSUPPORTED
    assert L.kohler_curve(None, 1, 8, 4, 8, 256, 4, card.data_ptr(), card.data_ptr(), None, None) == k.ERR_ARG
    assert L.kohler_curve(img.data_ptr(), 3, 8, 4, 8, 256, 4, card.data_ptr(), card.data_ptr(), None, None) == k.ERR_ARG


# ------------------------------------------------------------------------ thresholds entry point
def test_thresholds_entry_point():
    k = K()
    imgs = [synth.smooth_image(s, 80, 30, 256) for s in range(5)] + [synth.blobs_image()]
    curves = [oracle.curve(im, 256) for im in imgs]
    card = torch.from_numpy(np.stack([c for c, _ in curves]).view(np.int64)).cuda()
    sumc = torch.from_numpy(np.stack([s for _, s in curves]).view(np.int64)).cuda()
    for max_k in (0, 1, 6, 40):
        ts, cnt, t0 = k.thresholds(card, sumc, max_k)
        torch.cuda.synchronize()
        for i, (c, s) in enumerate(curves):
            ots, ocnt, ot0 = oracle.thresholds(c, s, max_k)
            assert np.array_equal(ts[i].cpu().numpy(), ots) and int(cnt[i]) == ocnt and int(t0[i]) == ot0


def test_thresholds_exact_ties():
    # curves chosen so that doubles cannot separate the values: exactness decides
    k = K()
    big = 2**60
    card = np.array([0, big, big + 1, 3, 999999999999999, 3, 0], np.uint64)
    sumc = np.array([0, big - 1, big, 1, 333333333333333, 1, 0], np.uint64)
    ts, cnt, t0 = k.thresholds(torch.from_numpy(card.view(np.int64)).cuda(), torch.from_numpy(sumc.view(np.int64)).cuda(), 4)
    ots, ocnt, ot0 = oracle.thresholds(card, sumc, 4)
    assert np.array_equal(ts[0].cpu().numpy(), ots) and int(cnt[0]) == ocnt and int(t0[0]) == ot0


# ------------------------------------------------------------------------ batches
@pytest.mark.parametrize("max_k", [0, 1, 5, 31, 32, 33, 100])
def test_many_maxima_every_max_k(max_k):
    # a noisy 12-bit field has hundreds of local maxima: the fused call (top-list
    # selection for max_k <= 32, ranking otherwise) and the standalone threshold
    # call must both give the oracle's ranked list, count and t0
    img = synth.cosine_u16(21, 256, 96)
    M = 4096
    card, sumc = oracle.curve_alg1(img, M)
    ots, ocnt, ot0 = oracle.thresholds(card, sumc, max_k)
    assert ocnt > 100
    k = K()
    out = k.analyze_batch([to_dev(img)], M, max_k)
    torch.cuda.synchronize()
    assert np.array_equal(u64(out[0][0]), card) and np.array_equal(u64(out[1][0]), sumc)
    assert int(out[4][0]) == ocnt and int(out[5][0]) == ot0
    assert np.array_equal(out[3][0].cpu().numpy()[:max_k], ots)
    ts, cnt, t0 = k.thresholds(torch.from_numpy(card.view(np.int64)).cuda(), torch.from_numpy(sumc.view(np.int64)).cuda(),
                               max_k)
    torch.cuda.synchronize()
    assert np.array_equal(ts[0].cpu().numpy()[:max_k], ots) and int(cnt[0]) == ocnt and int(t0[0]) == ot0


def test_batch_mixed_sizes_and_paths():
    imgs = [synth.smooth_image(100 + i, w, h, 256) for i, (w, h) in
            enumerate([(64, 48), (65, 48), (256, 7), (1, 30), (30, 1), (520, 33), (8, 8), (333, 101)])]
    want = [expect(im, 256) for im in imgs]
    got = run_analyze([to_dev(im) for im in imgs], 256)
    for i in range(len(imgs)):
        assert_same(got[i], want[i], f"image {i}")
    # permuted batch gives the same per-image results
    perm = [5, 2, 7, 0, 3, 1, 6, 4]
    got2 = run_analyze([to_dev(imgs[p]) for p in perm], 256)
    for j, p in enumerate(perm):
        assert_same(got2[j], want[p], f"perm {j}")


def test_batch_more_than_one_launch():
    # 130 images: two launches of at most 128 descriptors
    imgs = [synth.smooth_image(500 + i, 40 + 8 * (i % 5), 9 + i % 7, 256) for i in range(130)]
    got = run_analyze([to_dev(im) for im in imgs], 256)
    for i, im in enumerate(imgs):
        assert_same(got[i], expect(im, 256), f"image {i}")
    card, sumc, c = K().curve_batch([to_dev(im) for im in imgs], 256)
    torch.cuda.synchronize()
    for i, im in enumerate(imgs):
        oc, os_ = oracle.curve_alg1(im, 256)
        assert np.array_equal(u64(card[i]), oc) and np.array_equal(u64(sumc[i]), os_)


def test_two_streams_concurrently():
    k = K()
    a = synth.smooth_image(1, 512, 300, 256)
    b = synth.smooth_image(2, 512, 300, 256)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    da, db = to_dev(a), to_dev(b)
    torch.cuda.synchronize()
    outs = []
    for _ in range(5):
        with torch.cuda.stream(s1):
            oa = k.analyze_batch([da], 256, MAX_K, stream=s1)
        with torch.cuda.stream(s2):
            ob = k.analyze_batch([db], 256, MAX_K, stream=s2)
        outs.append((oa, ob))
    torch.cuda.synchronize()
    wa, wb = expect(a, 256), expect(b, 256)
    for oa, ob in outs:
        assert np.array_equal(u64(oa[0][0]), wa[0]) and np.array_equal(u64(ob[0][0]), wb[0])
        assert np.array_equal(u64(oa[1][0]), wa[1]) and np.array_equal(u64(ob[1][0]), wb[1])


# ------------------------------------------------------------------------ host-buffer path
@pytest.mark.parametrize("shape", [(1, 1), (37, 100), (600, 1032), (600, 1024)])
def test_analyze_host(shape):
    k = K()
    img = synth.smooth_image(shape[0] + shape[1], shape[1], shape[0], 256)
    card, sumc, c, ts, cnt, t0 = k.analyze_host(img, 256, MAX_K)
    assert_same((card, sumc, c, ts, cnt, t0), expect(img, 256))
    pinned = torch.from_numpy(img).pin_memory()
    got = k.analyze_host(pinned, 256, MAX_K)
    assert_same(got, expect(img, 256))
    out = k.host_outputs(256, MAX_K)
    for _ in range(2):  # the caller's arrays, reused
        assert_same(k.analyze_host(pinned, 256, MAX_K, out=out), expect(img, 256))
    with pytest.raises(ValueError):
        k.analyze_host(pinned, 256, MAX_K, out=k.host_outputs(255, MAX_K))


@pytest.mark.parametrize("dtype,w,h,M", [(np.uint8, 1000, 600, 256), (np.uint8, 333, 101, 200), (np.uint16, 516, 130, 4096)])
def test_analyze_host_pinned(dtype, w, h, M):
    # pinned host memory: the banded copies run asynchronously
    img = synth.smooth_image(91, w, h, M, dtype)
    src = torch.from_numpy(img.view(np.int16) if dtype == np.uint16 else img).pin_memory()
    got = K().analyze_host(src, M, MAX_K)
    assert_same((got[0], got[1], got[2], got[3], got[4], got[5]), expect(img, M), f"pinned {w}x{h}")


def test_analyze_host_u16_and_range():
    k = K()
    img = synth.smooth_image(8, 200, 150, 4096, np.uint16, noise_sd=25.0)
    assert_same(k.analyze_host(img, 4096, MAX_K), expect(img, 4096))
    bad = img.copy()
    bad[10, 10] = 4096
    with pytest.raises(k.KohlerError) as e:
        k.analyze_host(bad, 4096, MAX_K)
    assert e.value.status == k.ERR_RANGE
    # the error is reported once: the next call on a clean image succeeds
    assert_same(k.analyze_host(img, 4096, MAX_K), expect(img, 4096))


def test_analyze_host_in_bands():
    # images of more than 8 MB are copied and reduced in row bands (one per 8 MB,
    # at most 4): 36 Mpx pinned and packed (4 bands), and 18 Mpx from a wider
    # array (rows copied to a padded device pitch, 2 bands)
    k = K()
    big = synth.random_image(12, 6016, 6000, 256)
    got = k.analyze_host(torch.from_numpy(big).pin_memory(), 256, MAX_K)
    assert_same(got, expect(big, 256), "36 Mpx")
    wide = np.zeros((3456, 5200), np.uint8)
    wide[:, :5184] = synth.voronoi_18mp()
    view = wide[:, :5184]
    assert_same(k.analyze_host(view, 256, MAX_K), expect(np.ascontiguousarray(view), 256), "18 Mpx, pitch 5200")


def test_analyze_host_recorded_replays():
    # from pinned memory the host path is recorded as one CUDA graph on a
    # geometry's second call and replayed afterwards with the new image's
    # address: every call must give that image's own exact result, across
    # geometries (banded and not), a pageable call in between, a range error
    # and a workspace that grows in the middle (which invalidates the recordings)
    k = K()
    shapes = [(3456, 5184, 256), (600, 1024, 256), (300, 1000, 200)]
    for rnd in range(3):
        for si, (h, w, M) in enumerate(shapes):
            imgs = [synth.random_image(1000 * rnd + 10 * si + j, w, h, M) for j in range(3)]
            wants = [expect(a, M) for a in imgs]
            pins = [torch.from_numpy(a).pin_memory() for a in imgs]
            for j in (0, 1, 2, 1, 0):
                assert_same(k.analyze_host(pins[j], M, MAX_K), wants[j], f"round {rnd} {w}x{h} image {j}")
            assert_same(k.analyze_host(imgs[2], M, MAX_K), wants[2], "pageable between replays")
            if M < 256:  # a pixel >= M (M = 256 cannot be exceeded in uint8)
                bad = imgs[0].copy()
                bad[h // 2, w // 3] = M
                with pytest.raises(k.KohlerError) as e:
                    k.analyze_host(torch.from_numpy(bad).pin_memory(), M, MAX_K)
                assert e.value.status == k.ERR_RANGE
                assert_same(k.analyze_host(pins[1], M, MAX_K), wants[1], "after a range error")
        if rnd == 1:  # a larger M grows the host path's workspace
            u = synth.smooth_image(77, 516, 130, 4096, np.uint16)
            assert_same(k.analyze_host(torch.from_numpy(u.view(np.int16)).pin_memory(), 4096, MAX_K), expect(u, 4096))


# ------------------------------------------------------------------------ workloads at full size
def test_blobs_256():
    img = synth.blobs_image()
    assert_same(run_analyze([to_dev(img)], 256)[0], expect(img, 256))


@pytest.mark.slow
def test_voronoi_18mp_full():
    img = synth.voronoi_18mp()
    want = expect(img, 256)
    assert_same(run_analyze([to_dev(img)], 256)[0], want, "18 Mpx")
    # the definitional oracle at sampled thresholds agrees too
    ts = np.array([0, int(img.min()), 50, 120, 200, int(img.max()) - 1, 255], np.int32)
    c, s = oracle.curve_at(img, 256, ts)
    assert np.array_equal(c, want[0][ts]) and np.array_equal(s, want[1][ts])


@pytest.mark.slow
def test_voronoi_batch96_full():
    specs = synth.batch96_specs()
    imgs = synth.voronoi_batch(specs, workers=os.cpu_count() or 1)
    got = run_analyze([to_dev(im) for im in imgs], 256)
    for i, im in enumerate(imgs):
        assert_same(got[i], expect(im, 256), f"image {i} {im.shape}")


@pytest.mark.slow
def test_cosine_u16_batch16_full():
    imgs = synth.cosine_u16_batch()
    got = run_analyze([to_dev(im) for im in imgs], 4096)
    for i, im in enumerate(imgs):
        assert_same(got[i], expect(im, 4096), f"image {i}")
