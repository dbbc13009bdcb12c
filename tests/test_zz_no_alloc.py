"""The allocation-free entry point against the regular one.

kohler_analyze_noalloc serves callers that cannot allocate device memory while
they run (a real-time loop that must never wait in the allocator, a process
with a fixed memory budget): it keeps its scratch in one fixed array of device
memory instead of a per-stream workspace.  Its results must equal those of
kohler_analyze_batch bit for bit (the tolerance of every parity test here is
zero), on two calls in a row, since the array keeps the previous call's
contents.  Every case is also compared with the CPU oracle directly, so that a
mistake shared by both device paths cannot pass.  This file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
MAX_K = 16


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_05062_gb300 import build

    build.build()
    oracle.build()
    import paper_1707_05062_gb300 as K

    return K


def check_oracle(got, a, M, nb, what):
    card, sumc, c, ts, cnt, t0 = oracle.analyze(a, M, MAX_K, nbhd=nb)
    assert np.array_equal(got[0].view(np.uint64), card), what
    assert np.array_equal(got[1].view(np.uint64), sumc), what
    assert np.array_equal(got[2], c), what
    assert np.array_equal(got[3], ts) and int(got[4][0]) == cnt and int(got[5][0]) == t0, what


def regular(K, img, M, nb=4):
    card, sumc, c, ts, cnt, t0 = K.analyze_batch([img], M, MAX_K, nbhd=nb)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in (card[0], sumc[0], c[0], ts[0], cnt, t0)]


def no_alloc(K, img, M, stream, nb=4):
    dev = img.device
    card = torch.full((M,), -7, dtype=torch.int64, device=dev)
    sumc = torch.full((M,), -7, dtype=torch.int64, device=dev)
    c = torch.full((M,), -7.0, dtype=torch.float64, device=dev)
    ts = torch.full((MAX_K,), -7, dtype=torch.int32, device=dev)
    cnt = torch.full((1,), -7, dtype=torch.int32, device=dev)
    t0 = torch.full((1,), -7, dtype=torch.int32, device=dev)
    st = torch.full((1,), -7, dtype=torch.int32, device=dev)
    code = 1 if img.dtype == torch.uint8 else 2
    rc = K.lib().kohler_analyze_noalloc(img.data_ptr(), code, img.shape[1], img.shape[0],
                                        img.stride(0) * img.element_size(), M, nb, MAX_K, card.data_ptr(),
                                        sumc.data_ptr(), c.data_ptr(), ts.data_ptr(), cnt.data_ptr(), t0.data_ptr(),
                                        st.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, rc
    stream.synchronize()
    return [x.cpu().numpy() for x in (card, sumc, c, ts, cnt, t0)], int(st.item())


CASES = [
    ("blobs 256x256 u8", lambda: synth.blobs_image(), 256),
    ("smooth 300x520 u8, M=200", lambda: synth.smooth_image(5, 520, 300, 200), 200),
    ("smooth 77x93 u8 (generic pass)", lambda: synth.smooth_image(6, 93, 77, 256), 256),
    ("smooth 130x256 u16, M=4096", lambda: synth.smooth_image(7, 256, 130, 4096, np.uint16, noise_sd=30.0), 4096),
]


@pytest.mark.parametrize("name,make,M", CASES, ids=[c[0] for c in CASES])
def test_no_alloc_matches_regular_twice(lib, name, make, M):
    K = lib
    a = make()
    img = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda()
    want = regular(K, img, M)
    s = torch.cuda.Stream()
    for call in range(2):
        got, status = no_alloc(K, img, M, s)
        assert status == 0
        for g, w in zip(got, want):
            assert np.array_equal(g, w), f"{name}: call {call} differs"
        check_oracle(got, a, M, 4, f"{name}: call {call} against the oracle")


@pytest.mark.parametrize("nb", [8, 6])
@pytest.mark.parametrize("name,make,M", CASES, ids=[c[0] for c in CASES])
def test_no_alloc_other_neighbourhoods(lib, name, make, M, nb):
    K = lib
    a = make()
    img = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda()
    want = regular(K, img, M, nb)
    s = torch.cuda.Stream()
    for call in range(2):
        got, status = no_alloc(K, img, M, s, nb)
        assert status == 0
        for g, w in zip(got, want):
            assert np.array_equal(g, w), f"{name} N{nb}: call {call} differs"
        check_oracle(got, a, M, nb, f"{name} N{nb}: call {call} against the oracle")


def test_no_alloc_range_and_limits(lib):
    K = lib
    a = synth.smooth_image(8, 64, 32, 100)
    a[3, 4] = 150  # a pixel >= M
    img = torch.from_numpy(a).cuda()
    s = torch.cuda.Stream()
    got, status = no_alloc(K, img, 100, s)
    assert status == K.ERR_RANGE and not got[0].any() and not got[1].any()
    # the next call on clean data is unaffected by the previous call's contents
    b = synth.smooth_image(9, 64, 32, 100)
    imb = torch.from_numpy(b).cuda()
    got, status = no_alloc(K, imb, 100, s)
    assert status == 0
    want = regular(K, imb, 100)
    assert all(np.array_equal(g, w) for g, w in zip(got, want))
    # sizes beyond the fixed scratch are refused
    big = torch.zeros((4, 8), dtype=torch.int16, device="cuda")
    z = torch.zeros(8192, dtype=torch.int64, device="cuda")
    rc = K.lib().kohler_analyze_noalloc(big.data_ptr(), 2, 8, 4, 16, 8192, 4, 0, z.data_ptr(), z.data_ptr(), None,
                                        None, z.data_ptr(), z.data_ptr(), z.data_ptr(), None)
    assert rc == K.ERR_ARG
