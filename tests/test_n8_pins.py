"""Pins of the oracle's 8-neighbourhood curves against facts that do not come
from the oracle itself (the paper states the method for N4 and notes that the 8-
or 6-neighbourhood gives insignificant differences; Eq. 1-3 carry over with N8).

- a hand-worked 2 x 2 example with both diagonal pairs,
- a brute force that builds B(t) as an explicit list of ordered 8-neighbour pairs,
- closed forms: vertical and horizontal steps (3H - 2 and 3W - 2 boundary pairs),
  a checkerboard (its diagonal pairs are equal, so N8 gives the N4 curve),
  a constant image,
- invariants: sums over t, agreement of the three routes (ordered N8, half
  neighbourhood N8*, Algorithm 1 over N8*).
A planted mistake (a half neighbourhood missing one diagonal) must fail a pin.
"""
import numpy as np
import pytest

import brute
import oracle
import synth


def _n8star_pairs(img):
    v = img.astype(np.int64)
    h, w = v.shape
    a = [v[:, :-1].ravel(), v[:-1, :].ravel(), v[:-1, :-1].ravel(), v[:-1, 1:].ravel()]
    b = [v[:, 1:].ravel(), v[1:, :].ravel(), v[1:, 1:].ravel(), v[1:, :-1].ravel()]
    return np.concatenate(a), np.concatenate(b)


# Hand-worked: rows (0 4) and (6 9).  Unordered N8* pairs (lo, hi): (0,4) (6,9)
# right, (0,6) (4,9) down, (0,9) down-right, (4,6) down-left.  Per t, the pairs
# with lo <= t < hi and their min(hi - t, t - lo):
#   t=0: (0,4):0 (0,6):0 (0,9):0                 t=5: (0,6):1 (4,9):1 (4,6):1 (0,9):4
#   t=1: (0,4):1 (0,6):1 (0,9):1                 t=6: (6,9):0 (4,9):2 (0,9):3
#   t=2: (0,4):2 (0,6):2 (0,9):2                 t=7: (6,9):1 (4,9):2 (0,9):2
#   t=3: (0,4):1 (0,6):3 (0,9):3                 t=8: (6,9):1 (4,9):1 (0,9):1
#   t=4: (0,6):2 (4,9):0 (4,6):0 (0,9):4         t=9: none
HAND_IMG = np.array([[0, 4], [6, 9]], np.uint8)
HAND_CARD = [3, 3, 3, 3, 4, 4, 3, 3, 3, 0]
HAND_SUMC = [0, 3, 6, 7, 6, 7, 5, 5, 3, 0]


def _n8_suite(curve_fn):
    fails = []
    card, sumc = curve_fn(HAND_IMG, 10)
    if list(card) != HAND_CARD or list(sumc) != HAND_SUMC:
        fails.append("hand2x2")
    a_, b_ = 20, 29
    for H, W, vertical in ((5, 6, True), (4, 9, False), (1, 4, True), (6, 1, False)):
        img = np.full((H, W), a_, np.uint8)
        if vertical:
            img[:, W // 2:] = b_
        else:
            img[H // 2:, :] = b_
        n = (3 * H - 2) if vertical else (3 * W - 2)
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
    rng = np.random.default_rng(8)
    for trial in range(25):
        M = int(rng.integers(2, 14))
        img = rng.integers(0, M, size=(int(rng.integers(1, 6)), int(rng.integers(1, 6)))).astype(np.uint8)
        if [list(x) for x in curve_fn(img, M)] != list(brute.curve(img, M, nbhd=8)):
            fails.append(f"brute{trial}")
            break
    img = synth.smooth_image(4, 23, 17, 64)
    card, sumc = curve_fn(img, 64)
    a, b = _n8star_pairs(img)
    d = np.abs(a - b)
    if int(np.sum(card)) != int(d.sum()) or int(np.sum(sumc)) != int((d * d // 4).sum()):
        fails.append("sums")
    return fails


def test_brute_force_agrees_with_the_hand_example():
    card, sumc = brute.curve(HAND_IMG, 10, nbhd=8)
    assert card == HAND_CARD and sumc == HAND_SUMC


@pytest.mark.parametrize("route", ["n8", "n8half", "n8_alg1"])
def test_n8_routes_pass_the_pins(route):
    fn = {"n8": oracle.curve_n8, "n8half": oracle.curve_n8half, "n8_alg1": oracle.curve_n8_alg1}[route]
    assert _n8_suite(fn) == []


def test_n8_routes_agree_on_uint16():
    img = synth.smooth_image(2, 30, 20, 4096, np.uint16)
    a = oracle.curve_n8(img, 4096)
    b = oracle.curve_n8half(img, 4096)
    c = oracle.curve_n8_alg1(img, 4096)
    assert all(np.array_equal(a[i], b[i]) and np.array_equal(a[i], c[i]) for i in range(2))


def test_n8_analyze_thresholds():
    img = synth.smooth_image(7, 40, 30, 256)
    card, sumc, c, ts, cnt, t0 = oracle.analyze(img, 256, 8, nbhd=8)
    bc, bs = oracle.curve_n8(img, 256)
    assert np.array_equal(card, bc) and np.array_equal(sumc, bs)
    assert cnt >= 1 and t0 == ts[0]


def test_pins_catch_a_missing_diagonal():
    def three_directions(img, M):
        v = img.astype(np.int64)
        card = [0] * M
        sumc = [0] * M
        pairs = list(zip(v[:, :-1].ravel(), v[:, 1:].ravel())) + list(zip(v[:-1, :].ravel(), v[1:, :].ravel())) + \
            list(zip(v[:-1, :-1].ravel(), v[1:, 1:].ravel()))
        for t in range(M):
            for f0, f1 in pairs:
                lo, hi = min(f0, f1), max(f0, f1)
                if lo <= t < hi:
                    card[t] += 1
                    sumc[t] += min(hi - t, t - lo)
        return card, sumc

    assert _n8_suite(three_directions)
