"""Pins of the CPU oracle against facts that do not come from the oracle itself.

- hand-worked fixtures in tests/golden (derived from Eq. 1-4 by hand),
- a brute-force construction of the classes and of B(t) as explicit sets (Eq. 1-3),
- closed forms for images whose boundary can be written down,
- invariants of the definition (sums over t, support, symmetries, additivity),
- agreement of the three oracle formulations (full ordered N4 of Eq. 1, the N4*
  half neighbourhood of Eq. 9 and Algorithm 1).
The final tests plant mistakes in copies of the computation and check that the
pins catch each of them.
"""
import glob
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import brute
import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def parse_golden(path):
    d = {"rows": []}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        if k == "row":
            d["rows"].append([int(x) for x in v])
        elif k == "W":
            d["W"], d["H"] = int(v[0]), int(v[2])
        else:
            d[k] = [int(x) for x in v]
    img = np.array(d["rows"], dtype=np.uint8)
    assert img.shape == (d["H"], d["W"])
    return img, d


GOLDEN_FILES = sorted(glob.glob(os.path.join(GOLDEN, "example_*.txt")))


@pytest.mark.parametrize("path", GOLDEN_FILES, ids=os.path.basename)
def test_golden_fixture(path):
    img, d = parse_golden(path)
    M = d["M"][0]
    for fn in (oracle.curve, oracle.curve_n4, oracle.curve_alg1):
        card, sumc = fn(img, M)
        assert card.tolist() == d["card"]
        assert sumc.tolist() == d["sumc"]
    ts, cnt, t0 = oracle.thresholds(np.array(d["card"], np.uint64), np.array(d["sumc"], np.uint64), M)
    assert cnt == d["count"][0]
    assert t0 == d["t0"][0]
    assert ts[:cnt].tolist() == d["thresholds"]
    assert (ts[cnt:] == -1).all()
    c = oracle.normalise(np.array(d["card"], np.uint64), np.array(d["sumc"], np.uint64))
    for t in range(M):
        want = d["sumc"][t] / d["card"][t] if d["card"][t] else 0.0
        assert c[t] == want


def test_golden_brute_agrees():
    # the fixtures themselves are consistent with the literal set construction
    for path in GOLDEN_FILES:
        img, d = parse_golden(path)
        card, sumc = brute.curve(img, d["M"][0])
        assert card == d["card"] and sumc == d["sumc"]


# ------------------------------------------------------------------ brute force
def _random_small(seed):
    g = np.random.default_rng(seed)
    h, w = int(g.integers(1, 7)), int(g.integers(1, 7))
    M = int(g.integers(2, 13))
    return g.integers(0, M, size=(h, w)).astype(np.uint8), M


@pytest.mark.parametrize("seed", range(150))
def test_oracle_vs_brute_sets(seed):
    img, M = _random_small(seed)
    bc, bs = brute.curve(img, M)
    for fn in (oracle.curve, oracle.curve_n4, oracle.curve_alg1):
        card, sumc = fn(img, M)
        assert card.tolist() == bc
        assert sumc.tolist() == bs
    for max_k in (0, 1, 3, M):
        ts, cnt, t0 = oracle.thresholds(np.array(bc, np.uint64), np.array(bs, np.uint64), max_k)
        bts, bcnt, bt0 = brute.thresholds(bc, bs, max_k)
        assert (ts.tolist(), cnt, t0) == (bts, bcnt, bt0)


def _exhaustive(h, w, M):
    vals = np.array(list(itertools.product(range(M), repeat=h * w)), dtype=np.uint8)
    return vals.reshape(-1, h, w)


@pytest.mark.parametrize("h,w,M", [(1, 4, 4), (4, 1, 4), (2, 2, 5), (2, 3, 3), (3, 2, 3), (3, 3, 3)])
def test_oracle_exhaustive_tiny(h, w, M):
    imgs = _exhaustive(h, w, M)
    bc, bs = brute.curve_batch_numpy(imgs, M)
    for i in range(imgs.shape[0]):
        card, sumc = oracle.curve(imgs[i], M)
        assert np.array_equal(card.astype(np.int64), bc[i]), (imgs[i], card, bc[i])
        assert np.array_equal(sumc.astype(np.int64), bs[i])
    # the other two formulations on a spread of the same images
    for i in range(0, imgs.shape[0], max(1, imgs.shape[0] // 400)):
        for fn in (oracle.curve_n4, oracle.curve_alg1):
            card, sumc = fn(imgs[i], M)
            assert np.array_equal(card.astype(np.int64), bc[i])
            assert np.array_equal(sumc.astype(np.int64), bs[i])


def test_exhaustive_thresholds_3x3():
    imgs = _exhaustive(3, 3, 3)
    bc, bs = brute.curve_batch_numpy(imgs, 3)
    for i in range(0, imgs.shape[0], 7):
        ts, cnt, t0 = oracle.thresholds(bc[i].astype(np.uint64), bs[i].astype(np.uint64), 3)
        assert (ts.tolist(), cnt, t0) == brute.thresholds(bc[i].tolist(), bs[i].tolist(), 3)


# ------------------------------------------------------------------ closed forms
@pytest.mark.parametrize("a,b,w,h", [(0, 3, 4, 3), (10, 20, 6, 5), (0, 255, 2, 1), (7, 8, 3, 3), (100, 131, 9, 2)])
def test_two_level_step(a, b, w, h):
    # left half a, right half b (a < b): every row has exactly one crossing pair,
    # card(t) = H and C(t) = min(t - a, b - t) on [a, b[, both 0 elsewhere.
    img = np.full((h, w), a, np.uint8)
    img[:, w // 2:] = b
    M = 256
    card, sumc = oracle.curve(img, M)
    for t in range(M):
        if a <= t < b:
            assert card[t] == h and sumc[t] == h * min(t - a, b - t)
        else:
            assert card[t] == 0 and sumc[t] == 0
    ts, cnt, t0 = oracle.thresholds(card, sumc, 4)
    # single maximum at floor((a + b) / 2): a two-point plateau when b - a is odd
    assert cnt == 1 and t0 == (a + b) // 2 and ts[0] == (a + b) // 2


@pytest.mark.parametrize("a,b,w,h", [(2, 9, 5, 4), (0, 1, 3, 3), (50, 200, 7, 6)])
def test_checkerboard(a, b, w, h):
    yy, xx = np.mgrid[0:h, 0:w]
    img = np.where((xx + yy) % 2 == 0, a, b).astype(np.uint8)
    n_pairs = 2 * w * h - w - h
    card, sumc = oracle.curve(img, 256)
    for t in range(256):
        inside = a <= t < b
        assert card[t] == (n_pairs if inside else 0)
        assert sumc[t] == (n_pairs * min(t - a, b - t) if inside else 0)


def test_horizontal_ramps():
    w, h = 9, 4
    img = np.tile(np.arange(w, dtype=np.uint8), (h, 1))
    card, sumc = oracle.curve(img, 16)
    assert card.tolist() == [h] * (w - 1) + [0] * (16 - w + 1)
    assert sumc.tolist() == [0] * 16
    ts, cnt, t0 = oracle.thresholds(card, sumc, 3)
    assert cnt == 1 and t0 == 0  # C = 0 over the whole support: one plateau
    img2 = (2 * img).astype(np.uint8)
    card, sumc = oracle.curve(img2, 32)
    top = 2 * (w - 1)
    assert card.tolist() == [h if t < top else 0 for t in range(32)]
    assert sumc.tolist() == [h * (t % 2) if t < top else 0 for t in range(32)]
    ts, cnt, t0 = oracle.thresholds(card, sumc, 32)
    assert cnt == w - 1 and t0 == 1
    assert ts[:cnt].tolist() == list(range(1, top, 2))


@pytest.mark.parametrize("shape", [(1, 1), (1, 5), (5, 1), (4, 4)])
def test_constant_image(shape):
    img = np.full(shape, 7, np.uint8)
    card, sumc = oracle.curve(img, 10)
    assert not card.any() and not sumc.any()
    ts, cnt, t0 = oracle.thresholds(card, sumc, 5)
    assert cnt == 0 and t0 == -1 and (ts == -1).all()
    assert not oracle.normalise(card, sumc).any()


def test_uint16_values():
    img = np.array([[0, 4095, 100], [4000, 1, 2]], np.uint16)
    card, sumc = oracle.curve(img, 4096)
    # compare with the vectorised definition (exact for any value range)
    nc, ns = brute.curve_batch_numpy(img[None].astype(np.int64), 4096)
    assert np.array_equal(card.astype(np.int64), nc[0]) and np.array_equal(sumc.astype(np.int64), ns[0])


def test_range_error():
    img = np.array([[0, 5]], np.uint8)
    with pytest.raises(oracle.OracleError):
        oracle.curve(img, 5)
    with pytest.raises(oracle.OracleError):
        oracle.curve_alg1(img, 4)


# ------------------------------------------------------------------ invariants
def _pairs(img):
    img = img.astype(np.int64)
    a = np.concatenate([img[:, :-1].ravel(), img[:-1, :].ravel()])
    b = np.concatenate([img[:, 1:].ravel(), img[1:, :].ravel()])
    return a, b


INV_CASES = [
    ("u8-smooth", lambda: synth.smooth_image(11, 37, 23, 256)),
    ("u8-random", lambda: synth.random_image(12, 19, 17, 256)),
    ("u8-M40", lambda: synth.smooth_image(13, 31, 29, 40)),
    ("u16-12bit", lambda: synth.smooth_image(14, 23, 19, 4096, np.uint16, noise_sd=40.0)),
    ("blobs-crop", lambda: synth.blobs_image()[:40, :50].copy()),
]


@pytest.mark.parametrize("name,make", INV_CASES, ids=[c[0] for c in INV_CASES])
def test_invariants(name, make):
    img = make()
    M = 4096 if img.dtype == np.uint16 else (40 if name == "u8-M40" else 256)
    card, sumc = oracle.curve(img, M)
    a, b = _pairs(img)
    d = np.abs(a - b)
    # sum over t of card = sum of |f0 - f1|; of sumc = sum of floor(d^2 / 4)
    assert int(card.sum()) == int(d.sum())
    assert int(sumc.sum()) == int((d * d // 4).sum())
    # support: card(t) > 0 exactly on [min f, max f[ (the grid is connected)
    lo, hi = int(img.min()), int(img.max())
    assert [t for t in range(M) if card[t] > 0] == list(range(lo, hi))
    if hi > lo:
        assert sumc[lo] == 0
        assert sumc[hi - 1] <= card[hi - 1]
    # the three formulations agree
    c2, s2 = oracle.curve_n4(img, M)
    c3, s3 = oracle.curve_alg1(img, M)
    assert np.array_equal(card, c2) and np.array_equal(sumc, s2)
    assert np.array_equal(card, c3) and np.array_equal(sumc, s3)
    # symmetries of the grid
    for tr in (img.T, img[::-1], img[:, ::-1], img[::-1, ::-1]):
        ct, st = oracle.curve(np.ascontiguousarray(tr), M)
        assert np.array_equal(card, ct) and np.array_equal(sumc, st)
    # shift by a constant shifts both curves
    if hi + 3 < M:
        cs, ss = oracle.curve((img + 3).astype(img.dtype), M)
        assert np.array_equal(cs[3:], card[:-3]) and np.array_equal(ss[3:], sumc[:-3])
        assert not cs[:3].any()
    # complement f -> M-1-f maps card(t) to card(M-2-t)
    cc, _ = oracle.curve((M - 1 - img.astype(np.int64)).astype(img.dtype), M)
    assert np.array_equal(cc[: M - 1], card[M - 2:: -1]) and cc[M - 1] == 0
    # row bands overlapping by one row add up (inclusion-exclusion of the shared row)
    r = img.shape[0] // 2
    if r >= 1:
        ca, sa = oracle.curve(img[: r + 1], M)
        cb, sb = oracle.curve(img[r:], M)
        cr, sr = oracle.curve(img[r: r + 1], M)
        assert np.array_equal(ca + cb - cr, card) and np.array_equal(sa + sb - sr, sumc)
    # the per-threshold entry point gives the same values
    ts = np.array(sorted({0, lo, (lo + hi) // 2, max(hi - 1, 0), M - 1}), np.int32)
    ca, sa = oracle.curve_at(img, M, ts)
    assert np.array_equal(ca, card[ts]) and np.array_equal(sa, sumc[ts])


def test_strided_view():
    # a pitched view (pitch > width) gives the same curve as its compact copy
    big = synth.smooth_image(21, 40, 12, 256)
    view = big[:, 3:29]
    assert view.strides[0] == 40
    c1, s1 = oracle.curve(view, 256)
    c2, s2 = oracle.curve(np.ascontiguousarray(view), 256)
    assert np.array_equal(c1, c2) and np.array_equal(s1, s2)


def test_normalise_rounding():
    # C(t) is the round-to-nearest double quotient of the two integers
    card = np.array([3, 7, 0, 2**53 + 1, 10**12], np.uint64)
    sumc = np.array([1, 22, 0, 2**54, 3 * 10**12 + 1], np.uint64)
    c = oracle.normalise(card, sumc)
    assert c[0] == 1 / 3 and c[1] == 22 / 7 and c[2] == 0.0
    assert c[3] == float(2**54) / float(2**53 + 1)
    assert c[4] == float(3 * 10**12 + 1) / float(10**12)


def test_threshold_rules():
    # plateaus, endpoints, ties and truncation of the ranked list
    card = np.array([0, 1, 1, 1, 1, 2, 2, 0, 3, 0], np.uint64)
    sumc = np.array([0, 1, 1, 0, 2, 4, 2, 0, 6, 0], np.uint64)
    # C:             -  1  1  0  2  2  1  -  2  -
    ts, cnt, t0 = oracle.thresholds(card, sumc, 2)
    assert cnt == 3 and t0 == 4 and ts.tolist() == [4, 8]
    ts, cnt, t0 = oracle.thresholds(card, sumc, 5)
    assert ts.tolist() == [4, 8, 1, -1, -1]
    assert (ts.tolist(), cnt, t0) == brute.thresholds(card.tolist(), sumc.tolist(), 5)
    # exact comparison: 1/3 vs 333333333333333/999999999999999 are equal rationals
    card = np.array([3, 999999999999999, 3], np.uint64)
    sumc = np.array([1, 333333333333333, 1], np.uint64)
    ts, cnt, t0 = oracle.thresholds(card, sumc, 3)
    assert cnt == 1 and t0 == 0 and ts.tolist() == [0, -1, -1]
    # two quotients equal as doubles but different as rationals
    big = 2**60
    card = np.array([big, big + 1], np.uint64)
    sumc = np.array([big - 1, big], np.uint64)
    assert float(big - 1) / float(big) == float(big) / float(big + 1)
    ts, cnt, t0 = oracle.thresholds(card, sumc, 2)
    assert Fraction(big, big + 1) > Fraction(big - 1, big)
    assert cnt == 1 and t0 == 1


# ------------------------------------------------------------------ pin sensitivity
def _pin_suite(curve_fn):
    """Run closed forms, brute force and invariants against curve_fn(img, M) ->
    (card, sumc); return the list of failed checks."""
    fails = []
    img = np.full((3, 4), 0, np.uint8)
    img[:, 2:] = 5
    card, sumc = curve_fn(img, 8)
    exp_c = [3 if 0 <= t < 5 else 0 for t in range(8)]
    exp_s = [3 * min(t, 5 - t) if t < 5 else 0 for t in range(8)]
    if list(card) != exp_c or list(sumc) != exp_s:
        fails.append("step")
    for seed in range(20):
        im, M = _random_small(1000 + seed)
        bc, bs = brute.curve(im, M)
        c, s = curve_fn(im, M)
        if list(c) != bc or list(s) != bs:
            fails.append(f"brute{seed}")
            break
    im = synth.smooth_image(3, 13, 11, 64)
    c, s = curve_fn(im, 64)
    a, b = _pairs(im)
    d = np.abs(a - b)
    if int(np.sum(c)) != int(d.sum()) or int(np.sum(s)) != int((d * d // 4).sum()):
        fails.append("sums")
    return fails


def _mutant(kind):
    def fn(img, M):
        img = img.astype(np.int64)
        h, w = img.shape
        card = [0] * M
        sumc = [0] * M
        pairs = []
        for y in range(h):
            for x in range(w):
                if x + 1 < w:
                    pairs.append((img[y, x], img[y, x + 1]))
                if y + 1 < h and kind != "no_down":
                    pairs.append((img[y, x], img[y + 1, x]))
        for t in range(M):
            for f0, f1 in pairs:
                lo, hi = min(f0, f1), max(f0, f1)
                if kind == "ordered_only":
                    lo, hi = f0, f1
                cond = (lo < t < hi) if kind == "strict_lo" else (lo <= t <= hi) if kind == "closed_hi" else (lo <= t < hi)
                if cond:
                    card[t] += 1
                    if kind == "max_not_min":
                        sumc[t] += max(hi - t, t - lo)
                    elif kind == "one_sided":
                        sumc[t] += t - lo
                    else:
                        sumc[t] += min(hi - t, t - lo)
        return card, sumc
    return fn


@pytest.mark.parametrize("kind", ["no_down", "ordered_only", "strict_lo", "closed_hi", "max_not_min", "one_sided"])
def test_pins_catch_planted_mistakes(kind):
    assert _pin_suite(_mutant(kind)), f"mutation {kind} was not caught"


def test_pins_pass_on_oracle():
    assert _pin_suite(lambda img, M: tuple(x.tolist() for x in oracle.curve(img, M))) == []
    assert _pin_suite(_mutant("none")) == []
