"""Pins of the oracle's segmentation (thresholds -> quantised image) against facts
that do not come from the oracle itself.

The classes are those of Section 2.1 (C_0^t = {f <= t}, C_1^t = {f > t}) cut by
several thresholds, and every pixel shows the mean value of its class (Fig. 1
and its caption; Section 4 for two classes).  The pins:

- a hand-worked fixture in tests/golden/*.seg,
- a brute force that builds each class as an explicit set by comparing every
  pixel with every threshold and takes the exact mean with fractions,
- closed forms (step images, a constant image, no thresholds),
- invariants (order preserved, at most k + 1 output values, each output inside
  its class's range).
The last tests plant mistakes in copies of the computation and check that the
pins catch each of them.
"""
import glob
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def parse_seg(path):
    d = {"rows": [], "out": []}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        if k in ("row", "out"):
            d["rows" if k == "row" else "out"].append([int(x) for x in v])
        elif k == "W":
            d["W"], d["H"] = int(v[0]), int(v[2])
        else:
            d[k] = [int(x) for x in v]
    return (np.array(d["rows"], np.uint8), d["M"][0], d["thresholds"], np.array(d["out"], np.uint8))


def brute_segment(img, M, thresholds):
    """Classes as explicit sets: pixel x is in C_i when exactly i of the distinct
    thresholds t in [0, M[ satisfy t < f(x) (so f(x) <= t for the others); its output
    is the exact mean of its class rounded half up (floor(mean + 1/2))."""
    ts = set(int(t) for t in thresholds if 0 <= int(t) < M)
    h, w = img.shape
    members = {}
    for y in range(h):
        for x in range(w):
            i = sum(1 for t in ts if int(img[y, x]) > t)
            members.setdefault(i, []).append((y, x))
    out = np.zeros_like(img)
    for i, px in members.items():
        mean = Fraction(sum(int(img[y, x]) for y, x in px), len(px))
        val = math.floor(mean + Fraction(1, 2))
        for y, x in px:
            out[y, x] = val
    return out


def _seg_pin_suite(seg):
    """Closed forms, brute force, invariants and the fixture against seg(img, M, ts);
    returns the failed checks."""
    fails = []
    # step: levels a | b, any threshold in [a, b[ keeps the image; a threshold below a
    # or at/above b leaves one class, the rounded mean
    a, b = 30, 90
    step = np.full((4, 6), a, np.uint8)
    step[:, 3:] = b
    for t in (a, (a + b) // 2, b - 1):
        if not np.array_equal(seg(step, 256, [t]), step):
            fails.append(f"step{t}")
    one = seg(step, 256, [b])
    if not np.all(one == (a + b + 1) // 2):  # n equal halves: mean (a + b) / 2 exactly = 60
        fails.append("step_one_class")
    # pixels equal to a threshold belong to the lower class
    eq = np.array([[5, 5, 6, 6]], np.uint8)
    if seg(eq, 8, [5]).tolist() != [[5, 5, 6, 6]]:
        fails.append("equal_goes_low")
    # exact half rounds up: class {2, 3} has mean 2.5 -> 3
    half = np.array([[2, 3, 9, 9]], np.uint8)
    if seg(half, 16, [3]).tolist() != [[3, 3, 9, 9]]:
        fails.append("half_up")
    # no thresholds, constant image
    c = np.full((3, 3), 7, np.uint8)
    if not np.array_equal(seg(c, 8, []), c):
        fails.append("constant")
    # brute force on random tiny images and threshold sets (unsorted, with repeats
    # and out-of-range entries such as the -1 padding of a ranked list)
    rng = np.random.default_rng(42)
    for trial in range(30):
        M = int(rng.integers(2, 40))
        img = rng.integers(0, M, size=(int(rng.integers(1, 6)), int(rng.integers(1, 7)))).astype(np.uint8)
        ts = [int(t) for t in rng.integers(-2, M + 2, size=int(rng.integers(0, 6)))]
        if not np.array_equal(seg(img, M, ts), brute_segment(img, M, ts)):
            fails.append(f"brute{trial}")
            break
    # invariants on a smooth image
    img = synth.smooth_image(11, 40, 30, 256)
    ts = [40, 200, 90, 130]
    out = seg(img, 256, ts)
    f, o = img.astype(np.int64).ravel(), out.astype(np.int64).ravel()
    order = np.argsort(f, kind="stable")
    if np.any(np.diff(o[order]) < 0):
        fails.append("monotone")
    if len(np.unique(o)) > len(ts) + 1:
        fails.append("levels")
    bounds = [-1] + sorted(ts) + [256]
    for i in range(len(bounds) - 1):
        m = (f > bounds[i]) & (f <= bounds[i + 1])
        if m.any() and not (f[m].min() <= o[m].min() and o[m].max() <= f[m].max()):
            fails.append(f"range{i}")
    # the hand-worked fixture
    for path in sorted(glob.glob(os.path.join(GOLDEN, "*.seg"))):
        gi, gM, gts, gout = parse_seg(path)
        if not np.array_equal(seg(gi, gM, gts), gout):
            fails.append(os.path.basename(path))
    return fails


def test_golden_fixture_exists():
    assert glob.glob(os.path.join(GOLDEN, "*.seg"))


def test_segment_pins_pass_on_oracle():
    assert _seg_pin_suite(oracle.segment) == []


def test_segment_oracle_dtypes_and_range():
    img = synth.smooth_image(3, 20, 9, 4096, np.uint16)
    out = oracle.segment(img, 4096, [1000, 3000])
    assert out.dtype == np.uint16 and out.shape == img.shape
    assert np.array_equal(out, brute_segment(img, 4096, [1000, 3000]))
    bad = img.copy()
    bad[0, 0] = 4096
    with pytest.raises(oracle.OracleError):
        oracle.segment(bad, 4096, [5])


def _seg_mutant(kind):
    def seg(img, M, thresholds):
        ts = [int(t) for t in thresholds if 0 <= int(t) < M]
        if kind != "unsorted":
            ts = sorted(set(ts))
        v = img.astype(np.int64)
        if kind == "unsorted":  # first threshold (in the given order) at or above the value
            cls = np.full(v.shape, len(ts), np.int64)
            for i in range(len(ts) - 1, -1, -1):
                cls[v <= ts[i]] = i
        else:
            cls = np.zeros(v.shape, np.int64)
            for t in ts:
                cls += (v >= t) if kind == "ge" else (v > t)
        out = np.zeros_like(img)
        for c in range(len(ts) + 1):
            m = cls == c
            n = int(m.sum())
            if n:
                s = int(v[m].sum())
                if kind == "floor":
                    out[m] = s // n
                elif kind == "half_even":
                    out[m] = int(np.rint(s / n))
                elif kind == "median":
                    out[m] = int(np.median(v[m]))
                else:
                    out[m] = (2 * s + n) // (2 * n)
        return out
    return seg


@pytest.mark.parametrize("kind", ["ge", "floor", "half_even", "median", "unsorted"])
def test_segment_pins_catch_planted_mistakes(kind):
    assert _seg_pin_suite(_seg_mutant(kind)), f"mutation {kind} was not caught"


def test_segment_pins_pass_on_clean_copy():
    assert _seg_pin_suite(_seg_mutant("none")) == []
