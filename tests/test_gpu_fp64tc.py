"""GPU checks of BLWS_PREC_FP64_TC: products with a dense W formed on the tensor
cores from BF16 digit planes (Ozaki-type splitting, exact FP32 sums of 256
terms, double-FP32 / FP64 combination), through the C ABI.

Bars: a product within 1e-13 (relative Frobenius) of an FP64 product formed
independently (torch on the GPU, FP64) — the splitting keeps ~47 bits of
each term, so errors are ~1e-14, within an order of magnitude of the DFMA
GEMM's; the Robust PCA results within the FP64 mode's parity bar (1e-6
against the oracle at tol 1e-10), since the solver cannot tell the two
products apart at this level.
"""
import numpy as np
import pytest

import oracle
from paper_1012_0365_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


@pytest.fixture(scope="module")
def ctxs(torch_mod):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1012_0365_gb300 import blws
    return blws.Context(k=3), blws.Context(k=3, precision=blws.PREC_FP64_TC)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("m,n,b", [(61, 47, 5), (200, 200, 11), (130, 250, 65), (300, 1000, 200),
                                   (2000, 2000, 101), (20000, 200, 15)])
@pytest.mark.parametrize("graded", [False, True])
def test_digit_products_match_fp64(ctxs, torch_mod, m, n, b, graded):
    torch = torch_mod
    _, coz = ctxs
    g = torch.Generator(device="cuda").manual_seed(m * 3 + n + b)
    W = torch.randn(n, m, dtype=torch.float64, device="cuda", generator=g).t()
    if graded:  # rows of W spanning six decades: one scale per row of W, per column of W^T
        W = W * torch.logspace(-3, 3, m, dtype=torch.float64, device="cuda")[:, None]
    X = torch.randn(b, m + n, dtype=torch.float64, device="cuda", generator=g).t()
    P = coz.apply(W, X)
    ref = torch.cat([W @ X[m:], W.t() @ X[:m]])
    torch.cuda.synchronize()
    # row-wise relative error (rows of P_u carry W's row scale)
    err = (torch.linalg.norm(P - ref, dim=1) / torch.linalg.norm(ref, dim=1).clamp_min(1e-300)).max().item()
    # error model: ~2^-47 of the scale of each term (the largest entry of its
    # row / column), summed over K with random signs; against the result this
    # is ~1e-14 for entries of one magnitude, up to ~1e-12 when a column of W
    # spans six decades over K = 20000 terms
    assert err < (2e-12 if graded else 1e-13)


def test_zero_rows_and_columns(ctxs, torch_mod):
    torch = torch_mod
    _, coz = ctxs
    m, n, b = 97, 65, 9
    W = torch.randn(n, m, dtype=torch.float64, device="cuda").t()
    W[5, :] = 0.0
    W[:, 7] = 0.0
    X = torch.randn(b, m + n, dtype=torch.float64, device="cuda").t()
    X[:, 3] = 0.0
    P = coz.apply(W, X)
    ref = torch.cat([W @ X[m:], W.t() @ X[:m]])
    torch.cuda.synchronize()
    assert torch.all(P[5] == 0) and torch.all(P[:, 3] == 0) and torch.all(P[m + 7] == 0)
    assert (torch.linalg.norm(P - ref) / torch.linalg.norm(ref)).item() < 1e-13


@pytest.mark.parametrize("m,n,rank,frac,seed", [(200, 200, 10, 0.05, 0), (61, 47, 3, 0.05, 1),
                                                (400, 40, 2, 0.10, 3)])
def test_rpca_matches_oracle(ctxs, torch_mod, m, n, rank, frac, seed):
    from paper_1012_0365_gb300 import blws
    c64, coz = ctxs
    D, _, _ = syn.rpca_problem(m, n, rank, frac, amp=50.0, seed=seed)
    Dt = blws.colmajor(torch_mod.from_numpy(D))
    A, E, info = coz.rpca_solve(Dt, tol=1e-10)
    ref = oracle.rpca_ialm_full(D, tol=1e-10)
    assert info["status"] == 0 and info["rank"] == ref["rank"]
    assert rel(A.cpu().numpy(), ref["A"]) < 1e-6
    assert rel(E.cpu().numpy(), ref["E"]) < 1e-6
    # and the same trajectory as the DFMA products
    _, _, i64 = c64.rpca_solve(Dt, tol=1e-10)
    assert abs(info["iters"] - i64["iters"]) <= 1


def test_full_size_rpca_2000x2000(ctxs, torch_mod):
    from paper_1012_0365_gb300 import blws
    _, coz = ctxs
    D, L0, S0 = syn.rpca_problem(2000, 2000, 100, 0.10, amp=50.0, seed=0)
    A, E, info = coz.rpca_solve(blws.colmajor(torch_mod.from_numpy(D)), tol=1e-9)
    assert info["status"] == 0 and info["rank"] == 100
    assert rel(A.cpu().numpy(), L0) < 1e-6
    assert rel(E.cpu().numpy(), S0) < 1e-6


def _colmajor_np(torch, x):
    from paper_1012_0365_gb300 import blws
    return blws.colmajor(torch.from_numpy(np.ascontiguousarray(x)))


# shapes of the solver's large products: the Ritz lift Q_k Z (4000 x 101, inner
# 303), a Gram matrix / block coefficient (101 x 101, inner 4000), a refinement
# product of the T_k eigen-solver (303^3), and a ragged case; each has at least
# 8e6 multiply-adds, so it takes the digit-plane route; one small case below
# that threshold stays on the FP64 pipe of the same context
@pytest.mark.parametrize("M,N,K", [(4000, 101, 303), (101, 101, 4000), (303, 303, 303), (517, 230, 1290),
                                   (50, 40, 30)])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_general_digit_products_match_numpy(ctxs, torch_mod, M, N, K, ta, tb):
    # C = alpha op(A) op(B) + beta C through blws_gemm against an FP64 NumPy product
    torch = torch_mod
    _, coz = ctxs
    rng = np.random.default_rng(M * 7 + N * 3 + K + 2 * ta + tb)
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((N, K) if tb else (K, N))
    C0 = rng.standard_normal((M, N))
    alpha, beta = -1.37, 0.61
    C = _colmajor_np(torch, C0)
    coz.gemm(_colmajor_np(torch, A), _colmajor_np(torch, B), C, alpha=alpha, beta=beta, ta=ta, tb=tb)
    opA = A.T if ta else A
    opB = B.T if tb else B
    prod = opA @ opB
    ref = alpha * prod + beta * C0
    # digit truncation: ~2^-49 of each row's / column's largest entry per term,
    # summed over K with random signs: ~1e-14 of the product for Gaussian data
    err = np.linalg.norm(C.cpu().numpy() - ref) / np.linalg.norm(prod)
    assert err < 1e-13, err


@pytest.mark.parametrize("n,K", [(303, 303), (101, 4000)])
def test_symmetric_digit_products_are_exactly_symmetric(ctxs, torch_mod, n, K):
    # X^T (T X) with T symmetric (the eigen-solver's projected matrix) and
    # X^T X (a CholeskyQR Gram matrix): the digit-plane route mirrors one
    # triangle, so the result is symmetric bit for bit, and matches NumPy
    torch = torch_mod
    _, coz = ctxs
    rng = np.random.default_rng(n + K)
    X = rng.standard_normal((K, n))
    G = rng.standard_normal((K, K))
    T = (G + G.T) / 2
    TX = T @ X
    C = _colmajor_np(torch, np.zeros((n, n)))
    coz.gemm(_colmajor_np(torch, X), _colmajor_np(torch, TX), C, ta=True, sym=True)
    Ch = C.cpu().numpy()
    assert np.array_equal(Ch, Ch.T)
    ref = X.T @ TX
    assert np.linalg.norm(Ch - ref) / np.linalg.norm(ref) < 1e-13
    Xg = _colmajor_np(torch, X)
    Gm = _colmajor_np(torch, np.zeros((n, n)))
    coz.gemm(Xg, Xg, Gm, ta=True)  # A^T A is detected and made symmetric by itself
    Gh = Gm.cpu().numpy()
    assert np.array_equal(Gh, Gh.T)
    assert np.linalg.norm(Gh - X.T @ X) / np.linalg.norm(X.T @ X) < 1e-13
