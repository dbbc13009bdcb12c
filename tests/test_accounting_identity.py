"""The per-pixel accounting the strip passes use, checked on CPU against the oracle.

The strip passes do not histogram pair ends directly.  Each pixel p adds, at its
own value, a word holding its number of pair ends and a signed field
  sum over its own lower pairs of m  -  sum over its upper pairs of m
  -  (its lower pairs padded with p itself)  -  (its upper pairs),
with m = -1 when the pair's lower pixel is lower; the right pair adds its
maximum; every own pair (right, down, lower diagonals) adds its sum.  A pair
whose partner is outside the image is replaced by (p, p).  Then
H_hi = Tmax - sum(field), H_lo = E - H_hi, and with H_s the scans of the exact
rewrite give card and sumc.  This restates that bookkeeping pixel by pixel for
the 4-, 8- and hexagonal 6-neighbourhoods and compares the curves with the
oracle's on random tiny images with every border case.
"""
import numpy as np
import pytest

import oracle


def curves_from_histograms(h_lo, h_hi, h_s, M):
    """card and sumc from the three pair histograms (the tent identity)."""
    t = np.arange(M)[:, None]
    v = np.arange(M)[None, :]
    s = np.arange(2 * M - 1)[None, :]
    card = np.cumsum(h_lo) - np.cumsum(h_hi)
    sumc = ((h_lo + h_hi)[None, :] * np.maximum(t - v, 0)).sum(1) - (h_s[None, :] * np.maximum(2 * t - s, 0)).sum(1)
    return card, sumc


def strip_accounting(img, M, nb, mistake=None):
    f = img.astype(np.int64)
    H, W = f.shape
    ends = np.zeros(M, np.int64)
    field = np.zeros(M, np.int64)
    tmax = np.zeros(M, np.int64)
    h_s = np.zeros(2 * M - 1, np.int64)
    for y in range(H):
        odd = (y + (1 if mistake == "row_parity" else 0)) & 1
        own_dr = nb == 8 or (nb == 6 and odd)
        own_dl = nb == 8 or (nb == 6 and not odd)
        up_ul = y > 0 and (nb == 8 or (nb == 6 and not odd))  # lower-right pairs of the row above
        up_ur = y > 0 and (nb == 8 or (nb == 6 and odd))      # lower-left pairs of the row above
        last = y == H - 1
        for x in range(W):
            p = f[y, x]
            left, right = x == 0, x == W - 1
            partner_r = p if right else f[y, x + 1]
            own = [p if last else f[y + 1, x]]
            pads = int(last)
            if own_dr:
                own.append(p if (last or right) else f[y + 1, x + 1])
                pads += int(last or right)
            if own_dl:
                own.append(p if (last or left) else f[y + 1, x - 1])
                pads += int(last or (left and mistake != "left_pad"))
            ups = []
            if y > 0:
                ups.append(f[y - 1, x])
                if up_ul and not left and mistake != "no_upper_diagonals":
                    ups.append(f[y - 1, x - 1])
                if up_ur and not right:
                    ups.append(f[y - 1, x + 1])
            m_own = sum(-1 if q < p else 0 for q in own)
            m_up = sum(-1 if p < u else 0 for u in ups)
            ends[p] += (2 if right else 1) + (0 if left else 1) + len(own) + pads + len(ups)
            field[p] += m_own - m_up - pads - len(ups)
            tmax[max(p, partner_r)] += 1
            h_s[p + partner_r] += 1
            for q in own:
                h_s[p + q] += 1
    h_hi = tmax - field
    h_lo = ends - h_hi
    return curves_from_histograms(h_lo, h_hi, h_s, M)


@pytest.mark.parametrize("nb,route", [(4, oracle.curve), (8, oracle.curve_n8), (6, oracle.curve_n6)])
def test_strip_accounting_reproduces_the_curves(nb, route):
    rng = np.random.default_rng(40 + nb)
    for trial in range(60):
        M = int(rng.integers(2, 12))
        img = rng.integers(0, M, size=(int(rng.integers(1, 7)), int(rng.integers(1, 7)))).astype(np.uint8)
        card, sumc = strip_accounting(img, M, nb)
        want_card, want_sumc = route(img, M)
        assert np.array_equal(card, want_card.astype(np.int64)), (nb, img.tolist())
        assert np.array_equal(sumc, want_sumc.astype(np.int64)), (nb, img.tolist())


@pytest.mark.parametrize("nb,mistake", [(8, "left_pad"), (6, "row_parity"), (8, "no_upper_diagonals")])
def test_planted_mistakes_are_caught(nb, mistake):
    route = oracle.curve_n8 if nb == 8 else oracle.curve_n6
    rng = np.random.default_rng(7)
    caught = False
    for trial in range(60):
        M = int(rng.integers(2, 12))
        img = rng.integers(0, M, size=(int(rng.integers(2, 7)), int(rng.integers(2, 7)))).astype(np.uint8)
        card, sumc = strip_accounting(img, M, nb, mistake)
        want_card, want_sumc = route(img, M)
        if not (np.array_equal(card, want_card.astype(np.int64)) and np.array_equal(sumc, want_sumc.astype(np.int64))):
            caught = True
            break
    assert caught, mistake
