"""Parity of the CUDA library with the oracle for the 8-neighbourhood
(KOHLER_N8: Eq. 1-3 with the diagonal neighbours), element by element: card
and sumc equal as integers, C(t) equal as doubles, thresholds, count and t0
equal.  All calls go through the C ABI."""
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


def run(imgs_np, M, **kw):
    out = K().analyze_batch([to_dev(im, **kw) for im in imgs_np], M, MAX_K, nbhd=K().KOHLER_N8)
    torch.cuda.synchronize()
    assert K().stream_status() == K().OK
    return [got_of(out, i) for i in range(len(imgs_np))]


SHAPES = [(1, 1), (1, 9), (9, 1), (2, 2), (3, 7), (17, 16), (33, 40), (64, 257), (7, 2056)]


@pytest.mark.parametrize("h,w", SHAPES)
@pytest.mark.parametrize("kind", ["smooth", "random"])
def test_u8_shapes(h, w, kind):
    img = synth.smooth_image(h * 3 + w, w, h, 256) if kind == "smooth" else synth.random_image(h + w, w, h, 256)
    assert_same(run([img], 256)[0], oracle.analyze(img, 256, MAX_K, nbhd=8), f"{h}x{w}")


def test_definitional_route_agrees():
    img = synth.random_image(3, 30, 20, 64)
    want = oracle.analyze(img, 64, MAX_K, method="n8", nbhd=8)
    assert_same(run([img], 64)[0], want)


@pytest.mark.parametrize("pad,offset", [(8, 0), (3, 1), (120, 5)])
def test_pitch_offset(pad, offset):
    img = synth.smooth_image(11, 100, 37, 256)
    assert_same(run([img], 256, pad_cols=pad, offset=offset)[0], oracle.analyze(img, 256, MAX_K, nbhd=8))


@pytest.mark.parametrize("M,dtype,h,w", [(7, np.uint8, 30, 41), (4096, np.uint16, 33, 132), (65536, np.uint16, 9, 37)])
def test_M_and_uint16(M, dtype, h, w):
    img = synth.smooth_image(M + w, w, h, M, dtype)
    assert_same(run([img], M)[0], oracle.analyze(img, M, MAX_K, nbhd=8), f"M={M}")


def test_batch_of_mixed_sizes():
    imgs = [synth.smooth_image(k, w, h, 256) for k, (h, w) in enumerate([(40, 64), (1, 300), (123, 77), (300, 512)])]
    got = run(imgs, 256)
    for i, im in enumerate(imgs):
        assert_same(got[i], oracle.analyze(im, 256, MAX_K, nbhd=8), f"image {i}")


def test_n8_differs_from_n4_where_it_should():
    # a diagonal boundary: the 8-neighbourhood sees the diagonal pairs across it
    img = np.fromfunction(lambda y, x: np.where(x > y, 200, 10), (20, 20), dtype=int).astype(np.uint8)
    n8 = run([img], 256)[0]
    n4 = K().analyze_batch([to_dev(img)], 256, MAX_K)
    torch.cuda.synchronize()
    assert not np.array_equal(n8[0], n4[0][0].cpu().numpy().view(np.uint64))
    assert_same(n8, oracle.analyze(img, 256, MAX_K, nbhd=8))


def test_host_path_and_curve_api():
    k = K()
    img = synth.smooth_image(21, 256, 90, 256)
    want = oracle.analyze(img, 256, MAX_K, nbhd=8)
    got = k.analyze_host(img, 256, MAX_K, nbhd=k.KOHLER_N8)
    assert_same(got, want)
    card, sumc, c = k.curve(to_dev(img), 256, nbhd=k.KOHLER_N8)
    torch.cuda.synchronize()
    assert np.array_equal(card.cpu().numpy().view(np.uint64), want[0])
    assert np.array_equal(c.cpu().numpy(), want[2])


def test_voronoi_18mp_n8():
    img = synth.voronoi_18mp()
    assert_same(run([img], 256)[0], oracle.analyze(img, 256, MAX_K, nbhd=8), "18 Mpx")
