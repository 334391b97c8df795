"""The allocation-free product blws_apply_noalloc, called through the C ABI.

Some callers cannot allocate device memory (a host framework that owns every
byte of the GPU, a plugin host that forbids its own allocations, code that
must not trigger the synchronisation an allocation can cause); this entry
point serves them with its scratch in a static device array.  The test checks
its output against the allocating blws_apply on two calls in a row, within
the relative tolerance of the GPU parity tests, and that it rejects a product
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


def test_noalloc_rejects_scratch_beyond_the_maximum(env):
    torch, blws = env
    lib = blws.load()
    # m x b = 19000 x 64 fills 297 tiles (< 2 per SM), so the product splits
    # its inner dimension in two: 2 * 19000 * 64 doubles > 2^21
    m, n, b = 19000, 100, 64
    W = blws.empty_colmajor(m, n).zero_()
    X = blws.empty_colmajor(m + n, b).zero_()
    P = blws.empty_colmajor(m + n, b).fill_(3.0)
    assert _call(lib, torch, W, X, P) == blws.EINVAL
    torch.cuda.synchronize()
    assert bool(torch.all(P == 3.0))  # nothing was launched
    assert _call(lib, torch, W, X[:, :0], P) == blws.EINVAL  # b = 0
