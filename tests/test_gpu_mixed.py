"""GPU checks of the mixed-precision mode (BLWS_PREC_MIXED), through the C ABI.

Products with a dense W, the other block products (Gram matrices, block
coefficients, residual updates, Ritz lift) and the RPCA reconstruction run on
the tensor cores from split TF32 operands (three products, FP32 accumulation
over at most 256 terms, FP64 sums beyond); the Cholesky factorisations, the
eigenproblem of T_k and the count stay FP64.  Bars:

* one product with the augmented matrix: relative Frobenius error <= 1e-5
  against the FP64 product (each of K terms carries ~2^-22 relative error,
  and the FP32 sums of <= 256 terms add ~256 * 2^-24 at worst);
* Robust PCA with the FP64 refinement tail (mixed until the residual is
  below mixed_tol, FP64 after), run to tol 1e-10: the same 1e-6 bar on A and
  E against the FP64 oracle as the FP64 mode, since both converge to the
  unique optimum;
* Robust PCA kept in mixed products throughout (mixed_tol = 0): 1e-4 against
  the FP64 oracle, the mixed-precision target.
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
    return blws.Context(k=3), blws.Context(k=3, precision=blws.PREC_MIXED)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("m,n,b", [(61, 47, 5), (200, 200, 11), (130, 250, 33), (300, 1000, 200),
                                   (2000, 2000, 101), (20000, 200, 15), (333, 129, 256)])
def test_mixed_apply_matches_fp64(ctxs, torch_mod, m, n, b):
    torch = torch_mod
    c64, cmx = ctxs
    g = torch.Generator(device="cuda").manual_seed(m * 7 + n + b)
    W = torch.randn(n, m, dtype=torch.float64, device="cuda", generator=g).t()
    X = torch.randn(b, m + n, dtype=torch.float64, device="cuda", generator=g).t()
    # an FP64 product formed independently of the library (torch, cuBLAS)
    P64 = torch.cat([W @ X[m:], W.t() @ X[:m]])
    Pm = cmx.apply(W, X)
    torch.cuda.synchronize()
    err = (torch.linalg.norm(Pm - P64) / torch.linalg.norm(P64)).item()
    assert err < 1e-5


# the solver's block products in this mode (Gram matrices, block coefficients,
# residual updates, Ritz lift) through blws_gemm: split TF32 operands on the
# tensor cores; one case with more than 256 result columns (the RPCA
# reconstruction A = (U Theta) V^T goes through the accumulator 256 columns
# at a time); against an FP64 NumPy product, at the mode's 1e-5 product bar
@pytest.mark.parametrize("M,N,K", [(4000, 101, 303), (101, 101, 4000), (517, 230, 1290), (700, 600, 64)])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_mixed_general_products_match_numpy(ctxs, torch_mod, M, N, K, ta, tb):
    from paper_1012_0365_gb300 import blws
    torch = torch_mod
    _, cmx = ctxs
    rng = np.random.default_rng(M + 3 * N + 7 * K + 2 * ta + tb)
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((N, K) if tb else (K, N))
    C0 = rng.standard_normal((M, N))
    C = blws.colmajor(torch.from_numpy(C0))
    cmx.gemm(blws.colmajor(torch.from_numpy(A)), blws.colmajor(torch.from_numpy(B)), C, alpha=0.75,
             beta=-0.5, ta=ta, tb=tb)
    prod = (A.T if ta else A) @ (B.T if tb else B)
    ref = 0.75 * prod - 0.5 * C0
    assert np.linalg.norm(C.cpu().numpy() - ref) / np.linalg.norm(prod) < 1e-5


def test_mixed_gram_is_exactly_symmetric(ctxs, torch_mod):
    from paper_1012_0365_gb300 import blws
    torch = torch_mod
    _, cmx = ctxs
    X = np.random.default_rng(5).standard_normal((4000, 101))
    Xg = blws.colmajor(torch.from_numpy(X))
    G = blws.colmajor(torch.zeros(101, 101, dtype=torch.float64))
    cmx.gemm(Xg, Xg, G, ta=True)
    Gh = G.cpu().numpy()
    assert np.array_equal(Gh, Gh.T)
    assert np.linalg.norm(Gh - X.T @ X) / np.linalg.norm(X.T @ X) < 1e-5


def test_mixed_apply_wide_block_keeps_fp64(ctxs, torch_mod):
    # b > 256 exceeds one accumulator: the product stays at the FP64 level
    # (digit planes from 8e6 multiply-adds, as in the FP64-equivalent mode)
    torch = torch_mod
    c64, cmx = ctxs
    W = torch.randn(300, 400, dtype=torch.float64, device="cuda").t()
    X = torch.randn(300, 700, dtype=torch.float64, device="cuda").t()
    err = (torch.linalg.norm(cmx.apply(W, X) - c64.apply(W, X)) / torch.linalg.norm(c64.apply(W, X))).item()
    assert err < 1e-13


@pytest.mark.parametrize("m,n,rank,frac,seed", [(200, 200, 10, 0.05, 0), (61, 47, 3, 0.05, 1),
                                                (400, 40, 2, 0.10, 3)])
def test_mixed_rpca_with_fp64_tail_matches_oracle(ctxs, torch_mod, m, n, rank, frac, seed):
    from paper_1012_0365_gb300 import blws
    _, cmx = ctxs
    D, _, _ = syn.rpca_problem(m, n, rank, frac, amp=50.0, seed=seed)
    A, E, info = cmx.rpca_solve(blws.colmajor(torch_mod.from_numpy(D)), tol=1e-10)
    ref = oracle.rpca_ialm_full(D, tol=1e-10)
    assert info["status"] == 0 and info["mixed_iters"] > 0
    assert rel(A.cpu().numpy(), ref["A"]) < 1e-6
    assert rel(E.cpu().numpy(), ref["E"]) < 1e-6
    assert info["rank"] == ref["rank"]


def test_mixed_only_rpca_within_mixed_target(ctxs, torch_mod):
    from paper_1012_0365_gb300 import blws
    _, cmx = ctxs
    D, _, _ = syn.rpca_problem(200, 200, 10, 0.05, amp=50.0, seed=0)
    A, E, info = cmx.rpca_solve(blws.colmajor(torch_mod.from_numpy(D)), tol=1e-6, mixed_tol=0.0)
    ref = oracle.rpca_ialm_full(D, tol=1e-10)
    assert info["status"] == 0 and info["mixed_iters"] == info["iters"]
    assert rel(A.cpu().numpy(), ref["A"]) < 1e-4
    assert rel(E.cpu().numpy(), ref["E"]) < 1e-4


def test_mixed_svt_matches_fp64_svt(ctxs, torch_mod):
    # the same cold start (same generator draws) in both modes: the factored
    # T_eps(W) may differ only by the precision of the products
    torch = torch_mod
    c64, cmx = ctxs
    rng = np.random.default_rng(3)
    m, n, r = 300, 200, 12
    Uq, _ = np.linalg.qr(rng.standard_normal((m, n)))
    Vq, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.concatenate([np.linspace(50, 10, r), rng.uniform(0, 1, n - r)])
    W = (Uq * s) @ Vq.T
    eps = 5.0
    from paper_1012_0365_gb300 import blws
    Wt = blws.colmajor(torch.from_numpy(W))
    out = []
    for c in (c64, cmx):
        U, V, sig, cnt = c.blws_svt(Wt, eps, r + 4)
        th = np.maximum(sig.cpu().numpy() - eps, 0.0)
        out.append(((U.cpu().numpy() * th) @ V.cpu().numpy().T, cnt))
    (A64, c1), (Am, c2) = out
    assert c1 == c2 == r
    assert rel(Am, A64) < 1e-5


def test_mixed_full_size_rpca_2000x2000(ctxs, torch_mod):
    from paper_1012_0365_gb300 import blws
    _, cmx = ctxs
    D, L0, S0 = syn.rpca_problem(2000, 2000, 100, 0.10, amp=50.0, seed=0)
    A, E, info = cmx.rpca_solve(blws.colmajor(torch_mod.from_numpy(D)))
    assert info["status"] == 0 and info["rank"] == 100 and info["mixed_iters"] >= 10
    assert rel(A.cpu().numpy(), L0) < 1e-6
    assert rel(E.cpu().numpy(), S0) < 1e-6


def test_mixed_mc_svt(ctxs, torch_mod):
    c64, cmx = ctxs
    P = syn.mc_problem(300, 300, 10, 6 * 10 * 590 / 300 ** 2, seed=0)
    args = (300, 300, torch_mod.from_numpy(P["rowptr"]).cuda(), torch_mod.from_numpy(P["cols"]).cuda(),
            torch_mod.from_numpy(P["vals"]).cuda())
    U, th, V, info = cmx.mc_solve(*args, max_rank=60)
    assert info["status"] == 0 and info["rank"] == 10
    X = (U.cpu().numpy() * th.cpu().numpy()) @ V.cpu().numpy().T
    M = P["ML"] @ P["MR"].T
    assert rel(X, M) < 5e-4
