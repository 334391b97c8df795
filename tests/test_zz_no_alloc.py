"""The allocation-free product blws_apply_noalloc, called through the C ABI.

Some callers cannot allocate device memory (a host framework that owns every
byte of the GPU, a plugin host that forbids its own allocations, code that
must not trigger the synchronisation an allocation can cause); this entry
point serves them with its scratch in a static device array.  The test checks
its output against the allocating blws_apply on two calls in a row, within
the relative tolerance of the GPU parity tests, and against an FP64 product
formed outside the library, and that it rejects a product
whose scratch need exceeds the array.  It runs last (file name) and needs no
state from other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-9  # relative Frobenius, as in the other GPU parity tests


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1012_0365_gb300 import blws
    return torch, blws


def _call(lib, torch, W, X, P):
    m, n = W.shape
    b = X.shape[1]
    return lib.blws_apply_noalloc(ctypes.c_void_p(W.data_ptr()), m, n, m,
                                  ctypes.c_void_p(X.data_ptr()), m + n, b,
                                  ctypes.c_void_p(P.data_ptr()), m + n,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_allocating_apply_two_calls(env):
    torch, blws = env
    lib = blws.load()
    ctx = blws.Context()
    g = torch.Generator(device="cuda").manual_seed(7)
    shapes = [(700, 523, 37), (2000, 2000, 101)]  # the second is the bench's product
    cases = []
    for m, n, b in shapes:
        W = blws.colmajor(torch.randn(m, n, dtype=torch.float64, device="cuda", generator=g))
        X = blws.colmajor(torch.randn(m + n, b, dtype=torch.float64, device="cuda", generator=g))
        P = blws.empty_colmajor(m + n, b).fill_(float("nan"))
        cases.append((W, X, P, ctx.apply(W, X)))
    torch.cuda.synchronize()
    # two calls in a row on the shared scratch array
    assert _call(lib, torch, *cases[0][:3]) == blws.OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _call(lib, torch, *cases[1][:3]) == blws.OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0  # nothing allocated by the second call
    for call, (W, X, P, ref) in enumerate(cases):
        err = float(torch.linalg.norm(P - ref) / torch.linalg.norm(ref))
        assert err < TOL, (call, err)
        # and against an FP64 product formed outside the library (torch, cuBLAS)
        m = W.shape[0]
        ind = torch.cat([W @ X[m:], W.t() @ X[:m]])
        err = float(torch.linalg.norm(P - ind) / torch.linalg.norm(ind))
        assert err < 1e-13, (call, err)


SCRATCH_DOUBLES = 2 << 20  # the header's stated maximum (16 MiB)
KBK = 16                   # k-block of the FP64 GEMM tiles


def noalloc_need(sms, M, N, K):
    """Scratch doubles of one product by the header's rule: the inner
    dimension is split (s > 1) only while the product has fewer than two tiles
    per SM, and then needs s * M * N doubles."""
    bm, bn = (128, 16) if N <= 16 else (64, 32) if N <= 32 else (64, 64)
    tiles = -(-M // bm) * -(-N // bn)
    splits = 1
    if tiles < 2 * sms and K > 4 * KBK:
        splits = min(-(-2 * sms // tiles), -(-K // (4 * KBK)))
    kchunk = -(-(-(-K // splits)) // KBK) * KBK
    splits = -(-K // kchunk)
    return splits * M * N if splits > 1 else 0


def test_noalloc_rejects_scratch_beyond_the_maximum(env):
    torch, blws = env
    lib = blws.load()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # W X_v with m rows and b = 64: 64 x 64 tiles; with one tile short of two
    # per SM the inner dimension splits in two and needs 2 m b doubles, more
    # than the array holds once the GPU has more than 128 SMs
    b = 64
    m = (2 * sms - 1) * 64
    n = 100
    if noalloc_need(sms, m, b, n) <= SCRATCH_DOUBLES:
        pytest.skip("no product of this shape exceeds the scratch on %d SMs" % sms)
    W = blws.empty_colmajor(m, n).zero_()
    X = blws.empty_colmajor(m + n, b).zero_()
    P = blws.empty_colmajor(m + n, b).fill_(3.0)
    assert _call(lib, torch, W, X, P) == blws.EINVAL
    torch.cuda.synchronize()
    assert bool(torch.all(P == 3.0))  # nothing was launched
    assert _call(lib, torch, W, X[:, :0], P) == blws.EINVAL  # b = 0
