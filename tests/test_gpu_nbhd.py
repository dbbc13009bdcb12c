"""Parity of the CUDA library with the oracle for the 8-neighbourhood (KOHLER_N8:
Eq. 1-3 with the diagonal neighbours) and the hexagonal 6-neighbourhood
(KOHLER_N6: odd rows shifted half a pixel right), element by element: card and
sumc equal as integers, C(t) equal as doubles, thresholds, count and t0 equal.
All calls go through the C ABI."""
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


def to_dev(img, pad_cols=0, offset=0):
    h, w = img.shape
    src = torch.from_numpy(img.view(np.int16).copy() if img.dtype == np.uint16 else img.copy())
    if pad_cols == 0 and offset == 0:
        return src.cuda()
    buf = torch.zeros(h * (w + pad_cols) + offset + 16, dtype=src.dtype, device="cuda")
    view = buf[offset: offset + h * (w + pad_cols)].view(h, w + pad_cols)[:, :w]
    view.copy_(src.cuda())
    return view


def got_of(out, i):
    card, sumc, c, ts, cnt, t0 = out
    return (card[i].cpu().numpy().view(np.uint64), sumc[i].cpu().numpy().view(np.uint64), c[i].cpu().numpy(),
            ts[i].cpu().numpy(), int(cnt[i]), int(t0[i]))


def assert_same(got, want, tag=""):
    for k, name in enumerate(("card", "sumc", "curve", "thresholds")):
        assert np.array_equal(got[k], want[k]), f"{tag} {name} differs"
    assert got[4] == want[4] and got[5] == want[5], f"{tag} count/t0"


def run(imgs_np, M, nb, **kw):
    out = K().analyze_batch([to_dev(im, **kw) for im in imgs_np], M, MAX_K, nbhd=nb)
    torch.cuda.synchronize()
    assert K().stream_status() == K().OK
    return [got_of(out, i) for i in range(len(imgs_np))]


SHAPES = [(1, 1), (1, 9), (9, 1), (2, 2), (3, 7), (17, 16), (33, 40), (64, 257), (7, 2056)]
NBS = pytest.mark.parametrize("nb", [8, 6])


@NBS
@pytest.mark.parametrize("h,w", SHAPES)
@pytest.mark.parametrize("kind", ["smooth", "random"])
def test_u8_shapes(h, w, kind, nb):
    img = synth.smooth_image(h * 3 + w, w, h, 256) if kind == "smooth" else synth.random_image(h + w, w, h, 256)
    assert_same(run([img], 256, nb)[0], oracle.analyze(img, 256, MAX_K, nbhd=nb), f"{h}x{w}")


@pytest.mark.parametrize("nb,method", [(8, "n8"), (6, "n6")])
def test_definitional_route_agrees(nb, method):
    img = synth.random_image(3, 30, 20, 64)
    want = oracle.analyze(img, 64, MAX_K, method=method, nbhd=nb)
    assert_same(run([img], 64, nb)[0], want)


@NBS
@pytest.mark.parametrize("pad,offset", [(8, 0), (3, 1), (120, 5)])
def test_pitch_offset(pad, offset, nb):
    img = synth.smooth_image(11, 100, 37, 256)
    assert_same(run([img], 256, nb, pad_cols=pad, offset=offset)[0], oracle.analyze(img, 256, MAX_K, nbhd=nb))


@NBS
@pytest.mark.parametrize("M,dtype,h,w", [(7, np.uint8, 30, 41), (4096, np.uint16, 33, 132), (65536, np.uint16, 9, 37)])
def test_M_and_uint16(M, dtype, h, w, nb):
    img = synth.smooth_image(M + w, w, h, M, dtype)
    assert_same(run([img], M, nb)[0], oracle.analyze(img, M, MAX_K, nbhd=nb), f"M={M}")


@NBS
def test_batch_of_mixed_sizes(nb):
    imgs = [synth.smooth_image(k, w, h, 256) for k, (h, w) in enumerate([(40, 64), (1, 300), (123, 77), (300, 512)])]
    got = run(imgs, 256, nb)
    for i, im in enumerate(imgs):
        assert_same(got[i], oracle.analyze(im, 256, MAX_K, nbhd=nb), f"image {i}")


@NBS
def test_differs_from_n4_where_it_should(nb):
    # a diagonal boundary: the 8- and 6-neighbourhoods see pairs across it that N4 does not
    img = np.fromfunction(lambda y, x: np.where(x > y, 200, 10), (20, 20), dtype=int).astype(np.uint8)
    got = run([img], 256, nb)[0]
    n4 = K().analyze_batch([to_dev(img)], 256, MAX_K)
    torch.cuda.synchronize()
    assert not np.array_equal(got[0], n4[0][0].cpu().numpy().view(np.uint64))
    assert_same(got, oracle.analyze(img, 256, MAX_K, nbhd=nb))


def test_n6_row_parity_comes_from_the_image_row():
    # the same pixels seen from row 1 on: the row shift flips, so the curve must
    # follow the oracle on the cropped image, not on the original's rows
    img = synth.random_image(5, 40, 31, 256)
    full = run([img], 256, 6)[0]
    crop = run([img[1:]], 256, 6)[0]
    assert_same(full, oracle.analyze(img, 256, MAX_K, nbhd=6))
    assert_same(crop, oracle.analyze(np.ascontiguousarray(img[1:]), 256, MAX_K, nbhd=6))


# 16-byte aligned uint8 rows with W % 16 == 0 take the strip pass (tensor copies
# with left and right halos): ragged last strips, 1- and 2-row images, M < 256
STRIP_SHAPES = [(1, 16), (2, 16), (3, 32), (3, 272), (5, 512), (50, 528), (129, 784), (33, 4112), (2, 1296)]


@NBS
@pytest.mark.parametrize("h,w", STRIP_SHAPES)
@pytest.mark.parametrize("kind", ["smooth", "random"])
def test_strip_route_shapes(h, w, kind, nb):
    seed = 5 * h + w
    img = synth.smooth_image(seed, w, h, 256) if kind == "smooth" else synth.random_image(seed, w, h, 256)
    assert_same(run([img], 256, nb)[0], oracle.analyze(img, 256, MAX_K, nbhd=nb), f"{h}x{w}")


@NBS
@pytest.mark.parametrize("M", [2, 61, 200])
def test_strip_route_small_M(M, nb):
    img = synth.smooth_image(M + 3, 528, 45, M)
    assert_same(run([img], M, nb)[0], oracle.analyze(img, M, MAX_K, nbhd=nb), f"M={M}")


@NBS
def test_strip_route_batch_and_crop(nb):
    # several strip images in one launch (one tensor map each), and a crop that
    # starts one row lower (the N6 row parity follows the image's own rows)
    imgs = [synth.random_image(k, w, h, 256) for k, (h, w) in enumerate([(64, 256), (3, 528), (77, 1024)])]
    imgs.append(np.ascontiguousarray(imgs[2][1:]))
    got = run(imgs, 256, nb)
    for i, im in enumerate(imgs):
        assert_same(got[i], oracle.analyze(im, 256, MAX_K, nbhd=nb), f"image {i}")


@NBS
def test_host_path_and_curve_api(nb):
    k = K()
    img = synth.smooth_image(21, 256, 90, 256)
    want = oracle.analyze(img, 256, MAX_K, nbhd=nb)
    got = k.analyze_host(img, 256, MAX_K, nbhd=nb)
    assert_same(got, want)
    card, sumc, c = k.curve(to_dev(img), 256, nbhd=nb)
    torch.cuda.synchronize()
    assert np.array_equal(card.cpu().numpy().view(np.uint64), want[0])
    assert np.array_equal(c.cpu().numpy(), want[2])


@NBS
def test_host_path_in_bands(nb):
    # an image large enough to be copied in several bands (band edges inside the image)
    k = K()
    img = synth.voronoi_18mp()
    got = k.analyze_host(img, 256, MAX_K, nbhd=nb)
    assert_same(got, oracle.analyze(img, 256, MAX_K, nbhd=nb))


@NBS
def test_voronoi_18mp(nb):
    img = synth.voronoi_18mp()
    assert_same(run([img], 256, nb)[0], oracle.analyze(img, 256, MAX_K, nbhd=nb), "18 Mpx")
