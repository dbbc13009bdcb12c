"""Error paths of the C ABI, forced from the host (no GPU fault is ever made).

  - KOHLER_ERR_TIMEOUT: kohler_poll with a deadline shorter than any frame.
  - KOHLER_ERR_BUSY: a server whose pinned staging cap is filled by queued frames.
  - KOHLER_ERR_NOMEM: injected allocation failures (kohler_test_inject with
    KOHLER_FAULT_ALLOC) on every path that allocates; the call fails cleanly and
    the next call, without injection, succeeds with exact results.  The
    allocation-free entry point allocates nothing, so a pending injection is
    left untouched by it.
  - KOHLER_ERR_CUDA per image: the strip pass's bounded ring wait is made to
    report failure after a wait that completed (KOHLER_FAULT_RING_WAIT), so no
    copy is left in flight: the image's outputs are zero and its status, the
    stream status, the allocation-free call's out_status and a server frame's
    poll all say KOHLER_ERR_CUDA; the next launch is exact again.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(300)]
MAX_K = 8


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_05062_gb300 import build

    build.build()
    oracle.build()
    import paper_1707_05062_gb300 as k

    yield k
    k.test_inject(k.FAULT_ALLOC, 0)
    k.test_inject(k.FAULT_RING_WAIT, 0)


def want_of(img, M=256, nb=4):
    return oracle.analyze(img, M, MAX_K, nbhd=nb)


def same(got, want):
    card, sumc, c, ts, cnt, t0 = got
    return (np.array_equal(card.cpu().numpy().reshape(-1).view(np.uint64), want[0])
            and np.array_equal(sumc.cpu().numpy().reshape(-1).view(np.uint64), want[1])
            and np.array_equal(c.cpu().numpy().reshape(-1), want[2])
            and np.array_equal(ts.cpu().numpy().reshape(-1), want[3])
            and int(cnt.reshape(-1)[0]) == want[4] and int(t0.reshape(-1)[0]) == want[5])


def server(K, M=256, budget=0, inflight=0, staging=0):
    h = ctypes.c_void_p()
    rc = K.lib().kohler_server_create_ex(ctypes.byref(h), M, MAX_K, budget, inflight, staging)
    return rc, h


def submit(K, h, frame, borrowed=False):
    t = ctypes.c_uint64()
    fn = K.lib().kohler_submit_borrowed if borrowed else K.lib().kohler_submit
    rc = fn(h, frame.ctypes.data, 1, frame.shape[1], frame.shape[0], frame.strides[0], ctypes.byref(t))
    return rc, t.value


def poll(K, h, ticket, timeout_us=-1):
    ts = (ctypes.c_int32 * MAX_K)()
    res = K.KohlerResult()
    res.thresholds = ctypes.cast(ts, ctypes.c_void_p)
    rc = K.lib().kohler_poll(h, ctypes.c_uint64(ticket), ctypes.byref(res), timeout_us)
    return rc, (res.t0, res.count, list(ts))


def served_want(frame, M=256):
    w = want_of(frame, M)
    return (int(w[5]), int(w[4]), w[3][:MAX_K].tolist())


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def test_poll_timeout_then_result(K):
    # one output slot: the first frame holds it until it is polled, so the
    # second cannot even be admitted before its deadline
    rc, h = server(K, inflight=1)
    assert rc == 0
    try:
        scene = synth.VideoScene(seed=31)
        f1, f2 = pinned(scene.frame(0, 1920, 1080)), pinned(scene.frame(1, 3840, 2160))
        rc1, t1 = submit(K, h, f1, borrowed=True)
        rc2, t2 = submit(K, h, f2, borrowed=True)
        assert rc1 == 0 and rc2 == 0
        assert poll(K, h, t2, timeout_us=1)[0] == K.ERR_TIMEOUT
        assert poll(K, h, t2, timeout_us=2000)[0] == K.ERR_TIMEOUT  # still waiting for the slot
        rc, res = poll(K, h, t1)
        assert rc == 0 and res == served_want(f1)
        rc, res = poll(K, h, t2)  # the ticket stays valid after its timeouts
        assert rc == 0 and res == served_want(f2)
    finally:
        assert K.lib().kohler_server_destroy(h) == 0


def test_busy_when_staging_full(K):
    # one output slot: the first frame holds it until polled, the next ones wait
    # in a 5 MB staging area (two 1920 x 1080 frames); the fourth does not fit
    rc, h = server(K, inflight=1, staging=5_000_000)
    assert rc == 0
    try:
        scene = synth.VideoScene(seed=32)
        fr = [scene.frame(k, 1920, 1080) for k in range(4)]
        tickets = []
        for f in fr[:3]:
            rc, t = submit(K, h, f)
            assert rc == 0
            tickets.append(t)
        assert submit(K, h, fr[3])[0] == K.ERR_BUSY
        for f, t in zip(fr[:3], tickets):  # polling frees the slot; the queued frames follow
            rc, res = poll(K, h, t)
            assert rc == 0 and res == served_want(f)
        rc, t = submit(K, h, fr[3])  # room again
        assert rc == 0
        rc, res = poll(K, h, t)
        assert rc == 0 and res == served_want(fr[3])
    finally:
        assert K.lib().kohler_server_destroy(h) == 0


def test_injected_allocation_failures(K):
    img_np = synth.smooth_image(41, 320, 200, 256)
    img = torch.from_numpy(img_np).cuda()
    want = want_of(img_np)
    # a stream without a workspace: torch hands out pooled stream handles, which
    # an earlier test may have used, so every workspace is released first and
    # the next call on the stream allocates one
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    assert K.lib().kohler_release() == 0
    K.test_inject(K.FAULT_ALLOC, 1)
    with pytest.raises(K.KohlerError) as e:
        K.analyze_batch([img], 256, MAX_K, stream=s)
    assert e.value.status == K.ERR_NOMEM
    got = K.analyze_batch([img], 256, MAX_K, stream=s)
    torch.cuda.synchronize()
    assert K.stream_status(s) == K.OK and same(got, want)
    # the host-buffer path (its buffers freed first, so that it allocates again)
    assert K.lib().kohler_release() == 0
    K.test_inject(K.FAULT_ALLOC, 1)
    with pytest.raises(K.KohlerError) as e:
        K.analyze_host(img_np, 256, MAX_K)
    assert e.value.status == K.ERR_NOMEM
    card, sumc, c, ts, cnt, t0 = K.analyze_host(img_np, 256, MAX_K)
    assert np.array_equal(card, want[0]) and np.array_equal(sumc, want[1]) and int(t0) == want[5]
    # segmentation scratch of a stream (released first: pooled handles)
    s2 = torch.cuda.Stream()
    out = torch.empty_like(img)
    torch.cuda.synchronize()
    assert K.lib().kohler_release() == 0
    res = K.analyze_batch([img], 256, 6, stream=s2)
    K.test_inject(K.FAULT_ALLOC, 1)
    with pytest.raises(K.KohlerError) as e:
        K.segment(img, 256, res[3][0], res[4][0], out=out, stream=s2)
    assert e.value.status == K.ERR_NOMEM
    K.segment(img, 256, res[3][0], res[4][0], out=out, stream=s2)
    torch.cuda.synchronize()
    ts6 = [int(x) for x in res[3][0].cpu().numpy() if x >= 0]
    assert np.array_equal(out.cpu().numpy(), oracle.segment(img_np, 256, ts6))
    # server creation, then a frame that can never get device memory
    K.test_inject(K.FAULT_ALLOC, 1)
    rc, h = server(K)
    assert rc == K.ERR_NOMEM
    rc, h = server(K)
    assert rc == 0
    try:
        f = synth.VideoScene(seed=33).frame(0, 640, 480)
        K.test_inject(K.FAULT_ALLOC, 2)  # the direct admission and the scheduler's retry both fail
        rc, t = submit(K, h, pinned(f), borrowed=True)
        assert rc == 0
        assert poll(K, h, t)[0] == K.ERR_NOMEM
        K.test_inject(K.FAULT_ALLOC, 0)
        fp = pinned(f)
        rc, t = submit(K, h, fp, borrowed=True)
        rc, res = poll(K, h, t)
        assert rc == 0 and res == served_want(f)
    finally:
        assert K.lib().kohler_server_destroy(h) == 0
    # the allocation-free call allocates nothing: a pending injection stays pending
    outs = [torch.zeros(256, dtype=torch.int64, device="cuda"), torch.zeros(256, dtype=torch.int64, device="cuda"),
            torch.zeros(256, dtype=torch.float64, device="cuda"), torch.zeros(MAX_K, dtype=torch.int32, device="cuda"),
            torch.zeros(1, dtype=torch.int32, device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda"),
            torch.zeros(1, dtype=torch.int32, device="cuda")]
    s3 = torch.cuda.Stream()
    K.test_inject(K.FAULT_ALLOC, 1)
    rc = K.lib().kohler_analyze_noalloc(img.data_ptr(), 1, 320, 200, 320, 256, 4, MAX_K,
                                        *[o.data_ptr() for o in outs], ctypes.c_void_p(s3.cuda_stream))
    s3.synchronize()
    assert rc == 0 and int(outs[6].item()) == 0 and same(outs[:6], want)
    assert K.lib().kohler_release() == 0  # the next call allocates a workspace
    with pytest.raises(K.KohlerError):  # the injection was still pending
        K.analyze_batch([img], 256, MAX_K, stream=torch.cuda.Stream())
    K.test_inject(K.FAULT_ALLOC, 0)


@pytest.mark.parametrize("nb", [8, 6])
def test_ring_wait_failure_other_neighbourhoods(K, nb):
    # the N8 / N6 strip pass takes the same failure path as the N4 one
    img_np = synth.smooth_image(43, 1024, 300, 256)
    img = torch.from_numpy(img_np).cuda()
    want = want_of(img_np, nb=nb)
    s = torch.cuda.Stream()
    got = K.analyze_batch([img], 256, MAX_K, stream=s, nbhd=nb)
    torch.cuda.synchronize()
    assert K.stream_status(s) == K.OK and same(got, want)
    K.test_inject(K.FAULT_RING_WAIT, 1)
    got = K.analyze_batch([img], 256, MAX_K, stream=s, nbhd=nb)
    assert K.stream_status(s) == K.ERR_CUDA
    assert not got[0].any() and not got[1].any() and not got[2].any()
    got = K.analyze_batch([img], 256, MAX_K, stream=s, nbhd=nb)
    assert K.stream_status(s) == K.OK and same(got, want)


def test_ring_wait_failure_reports_cuda_error(K):
    # a 16-byte aligned uint8 image takes the strip pass
    img_np = synth.smooth_image(42, 1024, 300, 256)
    img = torch.from_numpy(img_np).cuda()
    want = want_of(img_np)
    s = torch.cuda.Stream()
    got = K.analyze_batch([img], 256, MAX_K, stream=s)  # workspace made, stream clean
    torch.cuda.synchronize()
    assert K.stream_status(s) == K.OK and same(got, want)
    K.test_inject(K.FAULT_RING_WAIT, 1)
    got = K.analyze_batch([img], 256, MAX_K, stream=s)
    assert K.stream_status(s) == K.ERR_CUDA
    assert not got[0].any() and not got[1].any() and not got[2].any()
    got = K.analyze_batch([img], 256, MAX_K, stream=s)  # the next launch is exact again
    assert K.stream_status(s) == K.OK and same(got, want)
    # the allocation-free call reports it in out_status
    outs = [torch.zeros(256, dtype=torch.int64, device="cuda"), torch.zeros(256, dtype=torch.int64, device="cuda"),
            torch.zeros(256, dtype=torch.float64, device="cuda"), torch.zeros(MAX_K, dtype=torch.int32, device="cuda"),
            torch.zeros(1, dtype=torch.int32, device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda"),
            torch.zeros(1, dtype=torch.int32, device="cuda")]

    def noalloc():
        rc = K.lib().kohler_analyze_noalloc(img.data_ptr(), 1, 1024, 300, 1024, 256, 4, MAX_K,
                                            *[o.data_ptr() for o in outs], ctypes.c_void_p(s.cuda_stream))
        s.synchronize()
        return rc, int(outs[6].item())

    K.test_inject(K.FAULT_RING_WAIT, 1)
    assert noalloc() == (0, K.ERR_CUDA)
    assert not outs[0].any() and not outs[1].any()
    assert noalloc() == (0, K.OK) and same(outs[:6], want)
    # a served frame: its poll returns the error, the next frame is exact
    rc, h = server(K)
    assert rc == 0
    try:
        f = synth.VideoScene(seed=34).frame(0, 1920, 1080)
        K.test_inject(K.FAULT_RING_WAIT, 1)
        rc, t = submit(K, h, f)
        assert rc == 0
        assert poll(K, h, t)[0] == K.ERR_CUDA
        rc, t = submit(K, h, f)
        rc, res = poll(K, h, t)
        assert rc == 0 and res == served_want(f)
    finally:
        assert K.lib().kohler_server_destroy(h) == 0


def test_stream_overlap_results_unchanged(K):
    # the overlap permission changes when kernels may start, never a result
    imgs_np = [synth.smooth_image(50 + k, 512, 96 + 16 * k, 256) for k in range(3)]
    imgs = [torch.from_numpy(a).cuda() for a in imgs_np]
    wants = [want_of(a) for a in imgs_np]
    for enable in (True, False):
        s = torch.cuda.Stream()
        K.stream_overlap(s, enable)
        outs = [K.analyze_batch([im], 256, MAX_K, stream=s) for im in imgs for _ in range(2)]
        torch.cuda.synchronize()
        assert K.stream_status(s) == K.OK
        for j, o in enumerate(outs):
            assert same(o, wants[j // 2])
        K.stream_overlap(s, False)
