"""The continuous-batching frame server (kohler_submit / kohler_poll).

Every frame's thresholds must be the same whether it is served alone or mixed
with other frames that arrive while it is on the GPU (tolerance zero: the
results are exact integers), and equal to the oracle's.
"""
import ctypes
import threading
import time

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

    return k


class Server:
    def __init__(self, K, M=256, budget=0, inflight=0, staging=0):
        self.K = K
        self.L = K.lib()
        self.h = ctypes.c_void_p()
        assert self.L.kohler_server_create_ex(ctypes.byref(self.h), M, MAX_K, budget, inflight, staging) == 0

    def submit_borrowed(self, frame):
        t = ctypes.c_uint64()
        code = 1 if frame.dtype == np.uint8 else 2
        rc = self.L.kohler_submit_borrowed(self.h, frame.ctypes.data, code, frame.shape[1], frame.shape[0],
                                           frame.strides[0], ctypes.byref(t))
        return rc, t.value

    def submit(self, frame):
        t = ctypes.c_uint64()
        code = 1 if frame.dtype == np.uint8 else 2
        rc = self.L.kohler_submit(self.h, frame.ctypes.data, code, frame.shape[1], frame.shape[0], frame.strides[0],
                                  ctypes.byref(t))
        return rc, t.value

    def submit_segment(self, frame, out):
        t = ctypes.c_uint64()
        code = 1 if frame.dtype == np.uint8 else 2
        rc = self.L.kohler_submit_segment(self.h, frame.ctypes.data, code, frame.shape[1], frame.shape[0],
                                          frame.strides[0], out.ctypes.data, out.strides[0], ctypes.byref(t))
        return rc, t.value

    def poll(self, ticket, timeout_us=-1):
        ts = (ctypes.c_int32 * MAX_K)()
        res = self.K.KohlerResult()
        res.thresholds = ctypes.cast(ts, ctypes.c_void_p)
        rc = self.L.kohler_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(res), timeout_us)
        return rc, res.t0, res.count, list(ts), res.latency_s

    def submit_many(self, frs):
        arr = (self.K.KohlerFrame * len(frs))()
        for j, f in enumerate(frs):
            arr[j] = self.K.KohlerFrame(f.ctypes.data, f.shape[1], f.shape[0], f.strides[0])
        tickets = (ctypes.c_uint64 * len(frs))()
        n_done = ctypes.c_int32(-1)
        code = 1 if frs[0].dtype == np.uint8 else 2
        rc = self.L.kohler_submit_borrowed_many(self.h, arr, len(frs), code, tickets, ctypes.byref(n_done))
        return rc, list(tickets), n_done.value

    def poll_many(self, tickets, timeout_us=-1):
        n = len(tickets)
        bufs = [(ctypes.c_int32 * MAX_K)() for _ in range(n)]
        res = (self.K.KohlerResult * n)()
        for j in range(n):
            res[j].thresholds = ctypes.cast(bufs[j], ctypes.c_void_p)
        st = (ctypes.c_int32 * n)()
        tk = (ctypes.c_uint64 * n)(*tickets)
        rc = self.L.kohler_poll_many(self.h, tk, n, res, st, timeout_us)
        return rc, list(st), [(res[j].t0, res[j].count, list(bufs[j])) for j in range(n)]

    def stats(self):
        v = [ctypes.c_uint64() for _ in range(4)]
        assert self.L.kohler_server_stats(self.h, *[ctypes.byref(x) for x in v]) == 0
        return [x.value for x in v]

    def close(self):
        assert self.L.kohler_server_destroy(self.h) == 0


def expected(frame, M=256):
    card, sumc = oracle.curve_alg1(frame, M)
    ts, cnt, t0 = oracle.thresholds(card, sumc, MAX_K)
    return t0, cnt, ts.tolist()


def frames(n, seed=0):
    scene = synth.VideoScene(seed=77 + seed)
    sizes = [(640, 480), (1920, 1080), (320, 240), (1280, 720), (64, 48), (100, 37)]
    return [scene.frame(k, *sizes[k % len(sizes)]) for k in range(n)]


def test_alone_and_mixed(K):
    fr = frames(12)
    want = [expected(f) for f in fr]
    s = Server(K)
    try:
        alone = []
        for f in fr:  # one frame in flight at a time
            rc, t = s.submit(f)
            assert rc == 0
            rc, t0, cnt, ts, lat = s.poll(t)
            assert rc == 0 and lat > 0
            alone.append((t0, cnt, ts))
        # all frames at once from two producer threads: launches batch what is resident
        tickets = [None] * len(fr)

        def produce(idx):
            for i in idx:
                rc, t = s.submit(fr[i])
                assert rc == 0
                tickets[i] = t

        th = [threading.Thread(target=produce, args=(range(j, len(fr), 2),)) for j in range(2)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        mixed = []
        for t in tickets:
            rc, t0, cnt, ts, lat = s.poll(t)
            assert rc == 0
            mixed.append((t0, cnt, ts))
        assert alone == mixed == want
        sub, fin, launches, maxb = s.stats()
        assert sub == fin == 2 * len(fr)
        assert launches <= 2 * len(fr)
    finally:
        s.close()


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def test_borrowed_burst_batches(K):
    # frames submitted without waiting for their copies, from two threads: the
    # copies overlap, and frames whose copies land while launches are on the GPU
    # share one launch; every result equals the frame's own, served alone
    scene = synth.VideoScene(seed=21)
    sizes = [(1920, 1080), (3840, 2160), (640, 480), (1920, 1080)]
    fr = [pinned(scene.frame(k, *sizes[k % len(sizes)])) for k in range(32)]
    want = [expected(f) for f in fr]
    s = Server(K)
    try:
        alone = []
        for f in fr[:4]:
            rc, t = s.submit_borrowed(f)
            assert rc == 0
            rc, t0, cnt, ts, lat = s.poll(t)
            assert rc == 0
            alone.append((t0, cnt, ts))
        assert alone == want[:4]
        tickets = [None] * len(fr)

        def produce(idx):
            for i in idx:
                rc, t = s.submit_borrowed(fr[i])
                assert rc == 0
                tickets[i] = t

        th = [threading.Thread(target=produce, args=(range(j, len(fr), 2),)) for j in range(2)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        mixed = []
        for t in tickets:
            rc, t0, cnt, ts, lat = s.poll(t)
            assert rc == 0
            mixed.append((t0, cnt, ts))
        assert mixed == want
        sub, fin, launches, maxb = s.stats()
        assert sub == fin == 4 + len(fr)
        assert maxb > 1, "no launch took more than one frame"
        assert launches < 4 + len(fr)
    finally:
        s.close()


def test_pending_timeout_unknown_and_curve(K):
    s = Server(K)
    try:
        f = frames(1)[0]
        rc, t = s.submit(f)
        assert rc == 0
        rc0 = s.poll(t, timeout_us=0)[0]
        assert rc0 in (K.OK, K.PENDING)
        if rc0 == K.PENDING:
            # wait for completion, then fetch the device curve before releasing the ticket
            deadline = time.time() + 30
            while time.time() < deadline:
                dc = ctypes.c_void_p()
                r = s.L.kohler_server_curve(s.h, ctypes.c_uint64(t), ctypes.byref(dc))
                if r == K.OK:
                    break
                time.sleep(0.001)
            assert r == K.OK and dc.value
            rc, t0, cnt, ts, lat = s.poll(t, timeout_us=1000000)
            assert rc == 0
            assert (t0, cnt, ts) == expected(f)
        assert s.poll(987654321, timeout_us=0)[0] == K.ERR_ARG  # unknown ticket
    finally:
        s.close()


def test_range_error_frame(K):
    s = Server(K, M=100)
    try:
        bad = synth.smooth_image(3, 64, 32, 100)
        bad[5, 5] = 200
        good = synth.smooth_image(4, 64, 32, 100)
        rb, tb = s.submit(bad)
        rg, tg = s.submit(good)
        assert rb == 0 and rg == 0
        assert s.poll(tb)[0] == K.ERR_RANGE
        rc, t0, cnt, ts, lat = s.poll(tg)
        assert rc == 0
        card, sumc = oracle.curve_alg1(good, 100)
        ots, ocnt, ot0 = oracle.thresholds(card, sumc, MAX_K)
        assert (t0, cnt, ts) == (ot0, ocnt, ots.tolist())
    finally:
        s.close()


def test_memory_budget_admission(K):
    # a budget that holds one 1920x1080 frame at a time: frames wait for memory, none is lost
    s = Server(K, budget=1920 * 1080 + 1024, inflight=4)
    try:
        scene = synth.VideoScene(seed=9)
        fr = [scene.frame(k, 1920, 1080) for k in range(4)]
        tickets = [s.submit(f)[1] for f in fr]
        for f, t in zip(fr, tickets):
            rc, t0, cnt, ts, lat = s.poll(t)
            assert rc == 0 and (t0, cnt, ts) == expected(f)
        # a frame larger than the whole budget can never be admitted
        big = synth.VideoScene(seed=10).frame(0, 3840, 2160)
        rc, t = s.submit(big)
        assert rc == 0
        assert s.poll(t, timeout_us=10_000_000)[0] == K.ERR_NOMEM
    finally:
        s.close()


def test_destroy_with_frames_in_flight(K):
    s = Server(K)
    for f in frames(6, seed=3):
        assert s.submit(f)[0] == 0
    s.close()  # drains admitted frames, drops queued ones, returns


def test_segmented_frames(K):
    # two-class segmentation at each frame's own t0 (Section 4), copied into the
    # caller's buffer; mixed with a plain submission and a constant frame (one
    # class: its mean); uint16 frames on a server with M = 4096
    scene = synth.VideoScene()
    cases = [(256, [scene.frame(k, w, h) for k, (w, h) in enumerate([(640, 480), (1920, 1080), (64, 33), (640, 480)])]
              + [np.full((17, 40), 77, np.uint8)]),
             (4096, [synth.smooth_image(5, 300, 70, 4096, np.uint16), synth.smooth_image(6, 64, 9, 4096, np.uint16)])]
    for M, frames in cases:
        srv = Server(K, M=M)
        outs = []
        for f in frames:
            o = torch.zeros(f.shape, dtype=torch.uint8 if f.dtype == np.uint8 else torch.int16).pin_memory().numpy()
            outs.append(o.view(np.uint16) if f.dtype == np.uint16 else o)
        tickets = []
        for j, (f, o) in enumerate(zip(frames, outs)):
            rc, t = srv.submit(f) if (M == 256 and j == 3) else srv.submit_segment(f, o)
            assert rc == 0
            tickets.append(t)
        for j, (f, o, t) in enumerate(zip(frames, outs, tickets)):
            rc, t0, cnt, ts, _ = srv.poll(t)
            assert rc == 0
            want_t0 = oracle.analyze(f, M, MAX_K)[5]
            assert t0 == want_t0
            if M == 256 and j == 3:
                assert not o.any()  # plain submission: the buffer is untouched
            else:
                assert np.array_equal(o, oracle.segment(f, M, [want_t0])), f"M={M} frame {j}"
        srv.close()


def test_segment_submit_arguments(K):
    srv = Server(K)
    f = np.zeros((8, 16), np.uint8)
    o = np.zeros((8, 8), np.uint8)
    t = ctypes.c_uint64()
    assert srv.L.kohler_submit_segment(srv.h, f.ctypes.data, 1, 16, 8, 16, None, 16, ctypes.byref(t)) == K.ERR_ARG
    assert srv.L.kohler_submit_segment(srv.h, f.ctypes.data, 1, 16, 8, 16, o.ctypes.data, 8, ctypes.byref(t)) == K.ERR_ARG
    srv.close()


def test_submit_and_poll_many(K):
    # batches of frames handed over and collected in one call each: every result
    # equals the oracle's, frames share launches, and the calls' edge cases
    fr = [np.ascontiguousarray(f) for f in frames(40, seed=5)]
    want = [expected(f) for f in fr]
    pinned = [torch.from_numpy(f).pin_memory().numpy() for f in fr]
    s = Server(K)
    try:
        for b0 in range(0, len(fr), 8):
            rc, tickets, n_done = s.submit_many(pinned[b0:b0 + 8])
            assert rc == 0 and n_done == len(tickets)
            rc, st, res = s.poll_many(tickets)
            assert rc == 0 and st == [0] * len(tickets)
            assert res == want[b0:b0 + len(tickets)]
        # several batches in flight before the first poll
        batches = [s.submit_many(pinned[b0:b0 + 10]) for b0 in range(0, 40, 10)]
        for (rc, tickets, _), b0 in zip(batches, range(0, 40, 10)):
            assert rc == 0
            rc, st, res = s.poll_many(tickets)
            assert rc == 0 and res == want[b0:b0 + 10]
        assert s.stats()[3] > 1  # frames shared launches
        # a bad frame stops the batch: the frames before it are submitted
        bad = pinned[:3] + [np.zeros((0, 0), np.uint8)]
        arr = (K.KohlerFrame * 4)()
        for j, f in enumerate(bad[:3]):
            arr[j] = K.KohlerFrame(f.ctypes.data, f.shape[1], f.shape[0], f.strides[0])
        arr[3] = K.KohlerFrame(None, 16, 16, 16)
        tickets = (ctypes.c_uint64 * 4)()
        n_done = ctypes.c_int32(-1)
        assert s.L.kohler_submit_borrowed_many(s.h, arr, 4, 1, tickets, ctypes.byref(n_done)) == K.ERR_ARG
        assert n_done.value == 3
        rc, st, res = s.poll_many(list(tickets)[:3])
        assert rc == 0 and res == want[:3]
        # argument errors
        assert s.L.kohler_poll_many(s.h, None, 1, None, None, -1) == K.ERR_ARG
        assert s.L.kohler_submit_borrowed_many(s.h, arr, 0, 1, tickets, None) == K.ERR_ARG
    finally:
        s.close()


def test_poll_many_deadline_keeps_tickets(K):
    # a deadline that passes before a batch is done leaves its unfinished
    # tickets pending; polling them again returns their results
    big = [np.ascontiguousarray(synth.VideoScene(seed=91).frame(k, 3840, 2160)) for k in range(3)]
    want = [expected(f) for f in big]
    s = Server(K, inflight=1)
    try:
        rcs = [s.submit(f) for f in big]  # one slot: the frames run one after another
        assert all(rc == 0 for rc, _ in rcs)
        tickets = [t for _, t in rcs]
        rc, st, _ = s.poll_many(tickets, timeout_us=0)
        assert rc in (K.PENDING, K.ERR_TIMEOUT) or rc == 0
        if rc != 0:
            k = st.index(rc)
            assert all(x == rc for x in st[k:]) and all(x == 0 for x in st[:k])
            rest = tickets[k:]
            rc2, st2, res2 = s.poll_many(rest)
            assert rc2 == 0 and res2 == want[k:]
    finally:
        s.close()
