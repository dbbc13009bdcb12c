"""Brute-force statement of Köhler's boundary contrast, used to pin the oracle.

Written independently of ``oracle/`` from Section 2.1 of the paper:
the two classes of Eq. 1 are built as explicit Python sets, the boundary B(t) as
an explicit list of ordered 4-neighbour pairs, and Eq. 2-3 are summed over that
list.  Thresholds use exact fractions.  Only for tiny images.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def n4(x, y, w, h):
    """4-neighbours of (x, y) inside the w x h domain D."""
    for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        xx, yy = x + dx, y + dy
        if 0 <= xx < w and 0 <= yy < h:
            yield (xx, yy)


def n8(x, y, w, h):
    """8-neighbours of (x, y) inside the w x h domain D (the diagonals included)."""
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            xx, yy = x + dx, y + dy
            if (dx or dy) and 0 <= xx < w and 0 <= yy < h:
                yield (xx, yy)


def n6(x, y, w, h):
    """Neighbours of (x, y) on a hexagonal grid stored row by row, odd rows shifted
    half a pixel to the right: the pixel's centre sits at column x + (y mod 2) / 2,
    and its neighbours are the pixels of rows y - 1, y, y + 1 whose centres lie at
    distance exactly 1 (same row) or whose centres are half a column away (rows
    above and below)."""
    cx = Fraction(2 * x + (y % 2), 2)
    for yy in (y - 1, y, y + 1):
        if not 0 <= yy < h:
            continue
        for xx in range(max(0, x - 1), min(w, x + 2)):
            d = Fraction(2 * xx + (yy % 2), 2) - cx
            if (yy == y and abs(d) == 1) or (yy != y and abs(d) == Fraction(1, 2)):
                yield (xx, yy)


def boundary(img, t, nbhd=4):
    """B(t) of Eq. 1 as a list of ordered pairs (x0, x1) of the 4-, hexagonal 6- or
    8-neighbourhood."""
    h, w = img.shape
    f = {(x, y): int(img[y, x]) for y in range(h) for x in range(w)}
    c0 = {p for p, v in f.items() if v <= t}
    c1 = {p for p, v in f.items() if v > t}
    nb = {4: n4, 6: n6, 8: n8}[nbhd]
    return [(x0, x1) for x0 in sorted(c0) for x1 in nb(x0[0], x0[1], w, h) if x1 in c1], f


def curve(img, M, nbhd=4):
    """(card, sumc) lists over t in [0, M[ from the literal sets."""
    card, sumc = [], []
    for t in range(M):
        b, f = boundary(img, t, nbhd)
        card.append(len(b))
        sumc.append(sum(min(f[x1] - t, t - f[x0]) for x0, x1 in b))
    return card, sumc


def contrast_fractions(card, sumc):
    """Exact C(t) (Eq. 3) as Fractions; None where the boundary is empty."""
    return [Fraction(s, c) if c else None for c, s in zip(card, sumc)]


def thresholds(card, sumc, max_k):
    """Ranked local maxima (plateau rule: leftmost point of a plateau whose outside
    neighbours are absent or strictly lower), total count and t0 (Eq. 4)."""
    C = contrast_fractions(card, sumc)
    M = len(C)
    maxima = []
    t = 0
    while t < M:
        if C[t] is None:
            t += 1
            continue
        a = b = t
        while b + 1 < M and C[b + 1] is not None and C[b + 1] == C[a]:
            b += 1
        left = a == 0 or C[a - 1] is None or C[a - 1] < C[a]
        right = b + 1 >= M or C[b + 1] is None or C[b + 1] < C[b]
        if left and right:
            maxima.append(a)
        t = b + 1
    ranked = sorted(maxima, key=lambda u: (-C[u], u))
    valid = [u for u in range(M) if C[u] is not None]
    t0 = min(valid, key=lambda u: (-C[u], u)) if valid else -1
    out = (ranked + [-1] * max_k)[:max_k]
    return out, len(maxima), t0


def curve_batch_numpy(imgs: np.ndarray, M: int):
    """Vectorised Eq. 1-2 over a stack of equal-shape images (n, h, w): for every
    threshold and each of the four neighbour directions, count ordered pairs with
    f(x0) <= t < f(x1) and add min(f(x1) - t, t - f(x0))."""
    imgs = imgs.astype(np.int64)
    n = imgs.shape[0]
    card = np.zeros((n, M), np.int64)
    sumc = np.zeros((n, M), np.int64)
    pairs = []
    if imgs.shape[2] > 1:
        a, b = imgs[:, :, :-1], imgs[:, :, 1:]
        pairs += [(a, b), (b, a)]
    if imgs.shape[1] > 1:
        a, b = imgs[:, :-1, :], imgs[:, 1:, :]
        pairs += [(a, b), (b, a)]
    for t in range(M):
        for f0, f1 in pairs:
            inb = (f0 <= t) & (t < f1)
            card[:, t] += inb.sum(axis=(1, 2))
            sumc[:, t] += np.where(inb, np.minimum(f1 - t, t - f0), 0).sum(axis=(1, 2))
    return card, sumc
