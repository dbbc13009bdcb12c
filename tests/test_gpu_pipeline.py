"""Pipelined streams (kohler_stream_overlap mode 2): consecutive one-image calls
run side by side on half the GPU each.  The mode changes where and when kernels
run, never a result: every call's outputs must equal the oracle's exactly, in
eager calls issued back to back without synchronising, in a CUDA graph replayed
several times, across image sizes (grids capped at half the GPU and smaller
ones), around a call whose image has a pixel >= M, and for batched calls.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(600)]
MAX_K = 8


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_05062_gb300 import build

    build.build()
    oracle.build()
    import paper_1707_05062_gb300 as K

    return K


def want_of(img, M=256):
    return oracle.analyze(img, M, MAX_K)


def check(got, want, what):
    card, sumc, c, ts, cnt, t0 = got
    assert np.array_equal(card.cpu().numpy().reshape(-1).view(np.uint64), want[0]), what
    assert np.array_equal(sumc.cpu().numpy().reshape(-1).view(np.uint64), want[1]), what
    assert np.array_equal(c.cpu().numpy().reshape(-1), want[2]), what
    assert np.array_equal(ts.cpu().numpy().reshape(-1), want[3]), what
    assert int(cnt.reshape(-1)[0]) == want[4] and int(t0.reshape(-1)[0]) == want[5], what


@pytest.fixture(scope="module")
def images():
    # 2048x1536 and 3072x1024 take grids capped at half the GPU; 512x200 a
    # small grid; 1000x300 (not a multiple of 16 wide) another pass
    specs = [(2048, 1536, 40), (3072, 1024, 41), (512, 200, 42), (1008, 300, 43), (1000, 300, 44)]
    out = []
    for w, h, seed in specs:
        a = synth.voronoi_image(seed, w, h, max(8, w * h // 40000), 4.0)
        out.append((a, want_of(a)))
    return out


def test_pipelined_eager_back_to_back(K, images):
    s = torch.cuda.Stream()
    K.stream_overlap(s, pipeline=True)
    try:
        dev = [torch.from_numpy(a).cuda() for a, _ in images]
        torch.cuda.synchronize()
        outs = []
        with torch.cuda.stream(s):
            for rep in range(3):
                for j in range(len(dev)):
                    outs.append((j, K.analyze_batch([dev[j]], 256, MAX_K, stream=s)))
        s.synchronize()
        assert K.stream_status(s) == K.OK
        for n, (j, o) in enumerate(outs):
            check(o, images[j][1], f"call {n} (image {j})")
    finally:
        K.stream_overlap(s, False)


def test_pipelined_graph_replays(K, images):
    s = torch.cuda.Stream()
    K.stream_overlap(s, pipeline=True)
    try:
        dev = [torch.from_numpy(a).cuda() for a, _ in images[:2]]
        order = [0, 1, 1, 0, 1, 0, 0]
        with torch.cuda.stream(s):
            for j in range(2):  # the stream's workspace exists before capture
                K.analyze_batch([dev[j]], 256, MAX_K, stream=s)
        s.synchronize()
        outs = []
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for j in order:
                outs.append(K.analyze_batch([dev[j]], 256, MAX_K, stream=s))
        for rep in range(3):
            for o in outs:
                for x in o:
                    x.fill_(-3)
            with torch.cuda.stream(s):
                g.replay()
                g.replay()
            s.synchronize()
            assert K.stream_status(s) == K.OK
            for n, (j, o) in enumerate(zip(order, outs)):
                check(o, images[j][1], f"replay {rep}, call {n}")
    finally:
        K.stream_overlap(s, False)


def test_pipelined_range_error_stays_with_its_call(K, images):
    a0 = images[0][0]
    M = 200
    a0m = np.minimum(a0, M - 1).astype(np.uint8)
    want0 = want_of(a0m, M)
    a1 = a0m.copy()
    a1[700, 1000] = 250  # a pixel >= M in the middle call only
    s = torch.cuda.Stream()
    K.stream_overlap(s, pipeline=True)
    try:
        d0, d1 = torch.from_numpy(a0m).cuda(), torch.from_numpy(a1).cuda()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            o0 = K.analyze_batch([d0], M, MAX_K, stream=s)
            o1 = K.analyze_batch([d1], M, MAX_K, stream=s)
            o2 = K.analyze_batch([d0], M, MAX_K, stream=s)
        s.synchronize()
        assert K.stream_status(s) == K.ERR_RANGE
        assert K.stream_status(s) == K.OK
        check(o0, want0, "call before the bad image")
        check(o2, want0, "call after the bad image")
        assert not o1[0].any() and not o1[1].any()
    finally:
        K.stream_overlap(s, False)


def test_pipelined_batches_and_modes(K, images):
    s = torch.cuda.Stream()
    K.stream_overlap(s, pipeline=True)
    try:
        dev = [torch.from_numpy(a).cuda() for a, _ in images]
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            ob = K.analyze_batch(dev, 256, MAX_K, stream=s)      # several images: the whole GPU
            o1 = K.analyze_batch([dev[0]], 256, MAX_K, stream=s)  # one image: half of it
        s.synchronize()
        assert K.stream_status(s) == K.OK
        for j, (_, want) in enumerate(images):
            check([x[j] for x in ob], want, f"batch image {j}")
        check(o1, images[0][1], "single after batch")
    finally:
        K.stream_overlap(s, False)
    assert K.lib().kohler_stream_overlap(s.cuda_stream, 3) == K.ERR_ARG
    assert K.lib().kohler_stream_overlap(s.cuda_stream, -1) == K.ERR_ARG
