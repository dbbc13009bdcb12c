"""The row-band split on CPU ranks (gloo, world size 2 and 3).

Every pair of the 4-neighbourhood belongs to exactly one band: band [y0, y1)
owns the right pairs of its rows and the lower pairs of its rows.  card(t) and
sumc(t) (Eq. 1-2) are sums over pairs, so the bands' counts add up to the
whole image's.  Each rank computes its band's counts with the oracle, from the
rows the band holds (band_rows: three above, the band, one below), as the
N4* curve of the rows y0 .. y1 (the band and the row below) less the right
pairs of row y1, then the ranks sum them with reduce_histograms; the sum must
equal the oracle's curve of the whole image exactly.  A mistake in the band
bounds (a row counted twice, a lower pair dropped) fails it.
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def band_counts(rows: np.ndarray, first_row: int, H: int, y0: int, y1: int, M: int):
    """(card, sumc) of the pairs band [y0, y1) owns, from the rows it holds."""
    import oracle

    card = np.zeros(M, np.uint64)
    sumc = np.zeros(M, np.uint64)
    if y0 == y1:
        return card, sumc
    lo, hi = y0 - first_row, min(H, y1 + 1) - first_row
    c, s = oracle.curve(np.ascontiguousarray(rows[lo:hi]), M)
    card += c
    sumc += s
    if y1 < H:  # row y1's right pairs belong to the next band
        c, s = oracle.curve(np.ascontiguousarray(rows[hi - 1:hi]), M)
        card -= c
        sumc -= s
    return card, sumc


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    for p in (ROOT, HERE):
        sys.path.insert(0, p)
    try:
        import torch
        import torch.distributed as dist

        import oracle
        import synth
        import paper_1707_05062_gb300 as K

        oracle.build()
        dist.init_process_group("gloo", rank=rank, world_size=world)
        res = []
        for seed, (W, H, M) in enumerate(((97, 61, 256), (40, 7, 120), (33, 2, 256))):
            img = synth.smooth_image(50 + seed, W, H, M)
            if M < 256:
                img = np.minimum(img, M - 1).astype(np.uint8)
            y0, y1 = K.row_bands(H, world)[rank]
            r0, r1 = K.band_rows(H, y0, y1)
            rows = img[r0:r1].copy()  # all this rank holds of the image
            card, sumc = band_counts(rows, r0, H, y0, y1, M)
            t = torch.from_numpy(np.concatenate([card, sumc]).view(np.int64).copy())
            K.reduce_histograms(t)
            got = t.numpy().view(np.uint64)
            wc, ws = oracle.curve(img, M)
            res.append(bool(np.array_equal(got[:M], wc) and np.array_equal(got[M:], ws)))
        dist.destroy_process_group()
        q.put((rank, res, None))
    except Exception as e:  # reported to the parent
        q.put((rank, None, repr(e)))


@pytest.mark.parametrize("world", [2, 3])
def test_band_counts_sum_over_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, world, port, q)) for k in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, res, err in got:
        assert err is None, err
        assert res == [True, True, True], (rank, res)


def test_band_counts_in_one_process():
    """The same decomposition without ranks, over every band count up to H + 2
    (empty bands and bands of one row included), and a planted mistake: bands
    that also keep row y1's right pairs overcount."""
    for p in (ROOT, HERE):
        if p not in sys.path:
            sys.path.insert(0, p)
    import oracle
    import synth
    import paper_1707_05062_gb300 as K

    oracle.build()
    img = synth.smooth_image(60, 29, 11, 256)
    H, M = img.shape[0], 256
    wc, ws = oracle.curve(img, M)
    for n in range(1, H + 3):
        card = np.zeros(M, np.uint64)
        sumc = np.zeros(M, np.uint64)
        bands = K.row_bands(H, n)
        assert bands[0][0] == 0 and bands[-1][1] == H
        assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))
        for y0, y1 in bands:
            r0, r1 = K.band_rows(H, y0, y1)
            assert r0 == max(0, y0 - 3) and r1 == min(H, y1 + 1)
            c, s = band_counts(img[r0:r1], r0, H, y0, y1, M)
            card += c
            sumc += s
        assert np.array_equal(card, wc) and np.array_equal(sumc, ws), n
    # planted: keep the next band's first row's right pairs
    card = np.zeros(M, np.uint64)
    for y0, y1 in K.row_bands(H, 3):
        c, _ = oracle.curve(np.ascontiguousarray(img[y0:min(H, y1 + 1)]), M)
        card += c
    assert not np.array_equal(card, wc)
