"""Pins of the oracle's hexagonal 6-neighbourhood curves against facts that do not
come from the oracle itself (Section 2 names the 6-neighbourhood beside the 8- as
giving insignificant differences; Eq. 1-3 carry over with N6).

The grid is stored row by row with every odd row (0-based) shifted half a pixel to
the right.  The pins:
- a hand-worked 2 x 2 example, whose one diagonal pair fixes that reading,
- a brute force that finds neighbours from the pixel centres' positions and builds
  B(t) as an explicit list of ordered pairs,
- closed forms: vertical and horizontal steps (2H - 1 and 2W - 1 boundary pairs),
  a checkerboard (its shifted pairs join equal values, so N6 gives the N4 curve),
  a constant image,
- invariants: sums over t, agreement of the three routes (ordered N6, half
  neighbourhood N6*, Algorithm 1 over N6*).
Planted mistakes (the shift on the wrong rows, a missing shifted pair) must fail.
"""
import numpy as np
import pytest

import brute
import oracle
import synth


def _n6star_pairs(img):
    """Unordered pairs right, down, and down-left (even rows) / down-right (odd rows)."""
    v = img.astype(np.int64)
    h, w = v.shape
    a = [v[:, :-1].ravel(), v[:-1, :].ravel()]
    b = [v[:, 1:].ravel(), v[1:, :].ravel()]
    for y in range(h - 1):
        if y % 2 == 0:
            a.append(v[y, 1:])
            b.append(v[y + 1, :-1])
        else:
            a.append(v[y, :-1])
            b.append(v[y + 1, 1:])
    return np.concatenate(a), np.concatenate(b)


# Hand-worked: rows (0 4) and (6 9).  Row 0 is even, so its pixel 4 at x = 1 touches
# the pixel 6 at x = 0 of row 1 (shifted right by half a pixel); 0 and 9 are not
# neighbours.  Unordered pairs (lo, hi): (0,4) (6,9) right, (0,6) (4,9) down, (4,6).
# Per t, the pairs with lo <= t < hi and their min(hi - t, t - lo):
#   t=0: (0,4):0 (0,6):0          t=5: (0,6):1 (4,9):1 (4,6):1
#   t=1: (0,4):1 (0,6):1          t=6: (6,9):0 (4,9):2
#   t=2: (0,4):2 (0,6):2          t=7: (6,9):1 (4,9):2
#   t=3: (0,4):1 (0,6):3          t=8: (6,9):1 (4,9):1
#   t=4: (0,6):2 (4,9):0 (4,6):0  t=9: none
HAND_IMG = np.array([[0, 4], [6, 9]], np.uint8)
HAND_CARD = [2, 2, 2, 2, 3, 3, 2, 2, 2, 0]
HAND_SUMC = [0, 2, 4, 4, 2, 3, 2, 3, 2, 0]


def _n6_suite(curve_fn):
    fails = []
    card, sumc = curve_fn(HAND_IMG, 10)
    if list(card) != HAND_CARD or list(sumc) != HAND_SUMC:
        fails.append("hand2x2")
    a_, b_ = 20, 29
    for H, W, vertical in ((5, 6, True), (4, 9, False), (6, 3, True), (1, 4, True), (6, 1, False), (3, 7, False)):
        img = np.full((H, W), a_, np.uint8)
        if vertical:
            img[:, W // 2:] = b_
        else:
            img[H // 2:, :] = b_
        n = (2 * H - 1) if vertical else (2 * W - 1)
        card, sumc = curve_fn(img, 32)
        exp_c = [n if a_ <= t < b_ else 0 for t in range(32)]
        exp_s = [n * min(t - a_, b_ - t) if a_ <= t < b_ else 0 for t in range(32)]
        if list(card) != exp_c or list(sumc) != exp_s:
            fails.append(f"step{H}x{W}")
    cb = np.fromfunction(lambda y, x: np.where((x + y) % 2 == 0, 3, 11), (7, 6), dtype=int).astype(np.uint8)
    if [list(x) for x in curve_fn(cb, 16)] != [list(x) for x in oracle.curve(cb, 16)]:
        fails.append("checkerboard")
    if any(np.any(np.asarray(x)) for x in curve_fn(np.full((4, 5), 9, np.uint8), 16)):
        fails.append("constant")
    rng = np.random.default_rng(6)
    for trial in range(25):
        M = int(rng.integers(2, 14))
        img = rng.integers(0, M, size=(int(rng.integers(1, 6)), int(rng.integers(1, 6)))).astype(np.uint8)
        if [list(x) for x in curve_fn(img, M)] != list(brute.curve(img, M, nbhd=6)):
            fails.append(f"brute{trial}")
            break
    img = synth.smooth_image(4, 23, 17, 64)
    card, sumc = curve_fn(img, 64)
    a, b = _n6star_pairs(img)
    d = np.abs(a - b)
    if int(np.sum(card)) != int(d.sum()) or int(np.sum(sumc)) != int((d * d // 4).sum()):
        fails.append("sums")
    return fails


def test_brute_force_agrees_with_the_hand_example():
    card, sumc = brute.curve(HAND_IMG, 10, nbhd=6)
    assert card == HAND_CARD and sumc == HAND_SUMC


def test_brute_neighbourhood_is_symmetric_with_six_inner_neighbours():
    w, h = 6, 5
    for y in range(h):
        for x in range(w):
            nb = list(brute.n6(x, y, w, h))
            if 0 < x < w - 1 and 0 < y < h - 1:
                assert len(nb) == 6
            assert all((x, y) in brute.n6(xx, yy, w, h) for xx, yy in nb)


@pytest.mark.parametrize("route", ["n6", "n6half", "n6_alg1"])
def test_n6_routes_pass_the_pins(route):
    fn = {"n6": oracle.curve_n6, "n6half": oracle.curve_n6half, "n6_alg1": oracle.curve_n6_alg1}[route]
    assert _n6_suite(fn) == []


def test_n6_routes_agree_on_uint16():
    img = synth.smooth_image(2, 30, 21, 4096, np.uint16)
    a = oracle.curve_n6(img, 4096)
    b = oracle.curve_n6half(img, 4096)
    c = oracle.curve_n6_alg1(img, 4096)
    assert all(np.array_equal(a[i], b[i]) and np.array_equal(a[i], c[i]) for i in range(2))


def test_n6_analyze_thresholds():
    img = synth.smooth_image(7, 40, 30, 256)
    card, sumc, c, ts, cnt, t0 = oracle.analyze(img, 256, 8, nbhd=6)
    bc, bs = oracle.curve_n6(img, 256)
    assert np.array_equal(card, bc) and np.array_equal(sumc, bs)
    assert cnt >= 1 and t0 == ts[0]


def _pairs_curve(pairs_fn):
    def curve(img, M):
        a, b = pairs_fn(img)
        card = [0] * M
        sumc = [0] * M
        for f0, f1 in zip(a.tolist(), b.tolist()):
            lo, hi = min(f0, f1), max(f0, f1)
            for t in range(lo, hi):
                card[t] += 1
                sumc[t] += min(hi - t, t - lo)
        return card, sumc
    return curve


def test_pins_pass_on_a_clean_pair_list():
    assert _n6_suite(_pairs_curve(_n6star_pairs)) == []
    assert _n6_suite(_pairs_curve(lambda img: _n6star_pairs_parity(img, 1))) == []


def test_pins_catch_the_shift_on_the_wrong_rows():
    assert _n6_suite(_pairs_curve(lambda img: _n6star_pairs_parity(img, 0)))


def test_pins_catch_a_missing_shifted_pair():
    def no_shift(img):
        v = img.astype(np.int64)
        return (np.concatenate([v[:, :-1].ravel(), v[:-1, :].ravel()]),
                np.concatenate([v[:, 1:].ravel(), v[1:, :].ravel()]))
    assert _n6_suite(_pairs_curve(no_shift))


def _n6star_pairs_parity(img, shifted_parity):
    """N6* pairs with the half-pixel shift on rows of the given parity."""
    v = img.astype(np.int64)
    h, w = v.shape
    a = [v[:, :-1].ravel(), v[:-1, :].ravel()]
    b = [v[:, 1:].ravel(), v[1:, :].ravel()]
    for y in range(h - 1):
        if y % 2 != shifted_parity:  # row y unshifted, row y + 1 shifted right
            a.append(v[y, 1:])
            b.append(v[y + 1, :-1])
        else:
            a.append(v[y, :-1])
            b.append(v[y + 1, 1:])
    return np.concatenate(a), np.concatenate(b)
