"""GPU parity of one BLWS-SVT evaluation (blws_svt through the C ABI) against
the FP64 oracle's literal Algorithm 2 / 3 on the augmented matrix.

Extra start columns are passed in explicitly (G) so both sides start from the
same block.  Tolerance: the two sides differ only in rounding order (CholeskyQR2
and FP32-Jacobi + FP64 refinement vs Householder QR and LAPACK eigh), so the
thresholded reconstruction A = U diag(max(sigma - eps, 0)) V^T must agree to
1e-9 relative in Frobenius norm and the Ritz values to 1e-10 of sigma_1.
"""
import numpy as np
import pytest

import oracle
from paper_1012_0365_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

A_TOL = 1e-9
SIG_TOL = 1e-10


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


@pytest.fixture(scope="module")
def blws(torch_mod):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1012_0365_gb300 import blws as b
    return b


def gpu(blws, torch, x):
    return blws.colmajor(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)))


def structured(m, n, rank, seed, noise=0.05):
    """Low-rank plus noise, so the top of the spectrum is separated."""
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n))
    return L + noise * np.sqrt(max(m, n)) * rng.standard_normal((m, n))


def recon(U, V, sig, eps):
    th = np.maximum(np.asarray(sig) - eps, 0.0)
    return (np.asarray(U) * th) @ np.asarray(V).T


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


CASES = [
    # m, n, rank of W, w (warm), r (out), k
    (40, 30, 4, 4, 5, 2),
    (67, 41, 6, 5, 7, 3),
    (200, 200, 10, 11, 11, 3),   # config-1 shape, block 11, k = 3
    (300, 17, 3, 3, 4, 2),       # tall, ragged
    (17, 300, 3, 4, 4, 3),       # wide
    (129, 130, 20, 18, 24, 3),   # width not a multiple of any tile, padding columns
    (513, 257, 30, 33, 33, 2),   # T_k of 66
    (600, 400, 40, 60, 60, 3),   # T_k of 180: the block-pair Jacobi path
    (1, 9, 1, 1, 1, 2),          # a single row
]


@pytest.mark.parametrize("m,n,rank,w,r,k", CASES)
def test_blws_svt_matches_oracle(blws, torch_mod, m, n, rank, w, r, k):
    torch = torch_mod
    W = structured(m, n, rank, seed=m * 7 + n)
    s = np.linalg.svd(W, compute_uv=False)
    eps = 0.5 * (s[min(rank, len(s)) - 1] + s[min(rank, len(s) - 1)]) if len(s) > 1 else 0.5 * s[0]
    # warm start: the top-w singular vectors of a perturbed W (the previous iterate)
    Wp = W + 0.01 * syn.gaussian_block(m, n, seed=3)
    Up, _, Vpt = np.linalg.svd(Wp, full_matrices=False)
    U0, V0 = Up[:, :w], Vpt[:w].T
    b = max(r, w)
    G = syn.gaussian_block(m + n, b - w, seed=5) if b > w else None
    ref = oracle.blws_svt_ref(W, eps, U0, V0, k, r, G)
    ctx = blws.Context(k=k)
    U, V, sig, c = ctx.blws_svt(gpu(blws, torch, W), eps, r, gpu(blws, torch, U0),
                                gpu(blws, torch, V0), None if G is None else gpu(blws, torch, G))
    U, V, sig = U.cpu().numpy(), V.cpu().numpy(), sig.cpu().numpy()
    assert c == ref["c"]
    np.testing.assert_allclose(sig, ref["sigma"], rtol=0, atol=SIG_TOL * s[0])
    assert rel(recon(U, V, sig, eps), ref["A"]) < A_TOL


@pytest.mark.parametrize("k", [2, 3])
def test_exact_warm_start_reproduces_full_svt(blws, torch_mod, k):
    # invariant start block: R_1 = 0 is deflated and the result is exact
    torch = torch_mod
    s = np.array([10.0, 8.0, 6.0, 4.0, 2.0, 1.0, 0.5, 0.25])
    U = syn.orthonormal(50, 8, seed=1)
    V = syn.orthonormal(40, 8, seed=2)
    W = (U * s) @ V.T
    ctx = blws.Context(k=k)
    Ug, Vg, sig, c = ctx.blws_svt(gpu(blws, torch, W), 3.0, 4, gpu(blws, torch, U[:, :4]),
                                  gpu(blws, torch, V[:, :4]))
    A, cref = oracle.svt_full(W, 3.0)
    assert c == cref == 4
    assert rel(recon(Ug.cpu().numpy(), Vg.cpu().numpy(), sig.cpu().numpy(), 3.0), A) < 1e-12


def test_cold_start_matches_oracle(blws, torch_mod):
    torch = torch_mod
    W = structured(120, 90, 6, seed=9)
    G = syn.gaussian_block(210, 8, seed=10)
    eps = 0.5 * np.linalg.svd(W, compute_uv=False)[3]
    ref = oracle.cold_svt_ref(W, eps, G, k=4, r=8)
    ctx = blws.Context(k_cold=4)
    # a cold start with the extra columns passed in: w = 0, g = 8
    U, V, sig, c = ctx.blws_svt(gpu(blws, torch, W), eps, 8, None, None, gpu(blws, torch, G))
    assert c == ref["c"]
    assert rel(recon(U.cpu().numpy(), V.cpu().numpy(), sig.cpu().numpy(), eps), ref["A"]) < A_TOL


def test_whole_space_krylov_is_exact(blws, torch_mod):
    torch = torch_mod
    W = syn.gaussian_block(5, 4, seed=30)
    U0, V0 = syn.gaussian_block(5, 3, seed=31), syn.gaussian_block(4, 3, seed=32)
    ctx = blws.Context(k=3)
    # b = 3 warm columns, k = 3 blocks: k b = m + n, the Krylov space is everything
    U, V, sig, c = ctx.blws_svt(gpu(blws, torch, W), 0.7, 3, gpu(blws, torch, U0), gpu(blws, torch, V0))
    s = np.linalg.svd(W, compute_uv=False)
    Ur, sr, Vrt = np.linalg.svd(W)
    np.testing.assert_allclose(sig.cpu().numpy(), s[:3], atol=1e-10)
    A3 = (Ur[:, :3] * np.maximum(s[:3] - 0.7, 0)) @ Vrt[:3]
    assert c == int(np.sum(s[:3] > 0.7))
    assert rel(recon(U.cpu().numpy(), V.cpu().numpy(), sig.cpu().numpy(), 0.7), A3) < 1e-10


@pytest.mark.parametrize("mult,eps", [(12, 7.0), (11, 7.0), (16, 7.0), (12, 11.0), (40, 3.0), (4, 7.0)])
def test_repeated_singular_values(blws, torch_mod, mult, eps):
    # a singular value of multiplicity `mult` gives T_k a cluster of equal
    # eigenvalues: the eigen-solver resolves it as a joint eigenspace (and
    # again on its own when it straddles eps); A = U max(S - eps, 0) V^T is
    # unique even though the singular vectors inside the cluster are not
    torch = torch_mod
    m, n = 160, 130
    s = np.concatenate([[20.0, 15.0], np.full(mult, 10.0), [6.0, 5.0]])  # exact rank mult + 4
    U = syn.orthonormal(m, len(s), seed=40)
    V = syn.orthonormal(n, len(s), seed=41)
    W = (U * s) @ V.T
    r = mult + 8  # a start block wider than the rank: the Krylov space holds range(W) exactly
    A, cref = oracle.svt_full(W, eps)
    ctx = blws.Context(k=3)
    G = syn.gaussian_block(m + n, r, seed=42)
    Ug, Vg, sig, c = ctx.blws_svt(gpu(blws, torch, W), eps, r, None, None, gpu(blws, torch, G))
    assert c == cref
    assert rel(recon(Ug.cpu().numpy(), Vg.cpu().numpy(), sig.cpu().numpy(), eps), A) < 1e-10


def test_rank_deficient_whole_space(blws, torch_mod):
    # W of rank 4 with the Krylov space reaching the whole augmented space:
    # T_k holds a large cluster of zero eigenvalues (too wide for the FP32
    # tridiagonal stage's grouping, which hands the matrix to Jacobi)
    torch = torch_mod
    m = n = 120
    W = syn.gaussian_block(m, 4, seed=50) @ syn.gaussian_block(4, n, seed=51)
    s = np.linalg.svd(W, compute_uv=False)
    eps = 0.5 * s[3]
    A, cref = oracle.svt_full(W, eps)
    ctx = blws.Context(k=2, k_cold=2)
    G = syn.gaussian_block(m + n, 120, seed=52)
    Ug, Vg, sig, c = ctx.blws_svt(gpu(blws, torch, W), eps, 120, None, None, gpu(blws, torch, G))
    assert c == cref
    assert rel(recon(Ug.cpu().numpy(), Vg.cpu().numpy(), sig.cpu().numpy(), eps), A) < 1e-10


@pytest.mark.parametrize("with_lowrank", [False, True])
def test_sparse_operator_matches_dense_oracle(blws, torch_mod, with_lowrank):
    # CSR (+ low-rank term) operator of matrix completion vs the dense oracle
    torch = torch_mod
    m, n = 150, 110
    P = syn.mc_problem(m, n, 4, 0.2, seed=4)
    S = np.zeros((m, n))
    S[P["rows"], P["cols"]] = P["vals"]
    Wd = S.copy()
    extra = ()
    if with_lowrank:
        Ul, Vl = syn.orthonormal(m, 3, seed=6), syn.orthonormal(n, 3, seed=7)
        sl = np.array([30.0, 20.0, 10.0])
        Wd = Wd + (Ul * sl) @ Vl.T
        extra = (gpu(blws, torch, Ul), torch.from_numpy(sl).cuda(), gpu(blws, torch, Vl))
    s = np.linalg.svd(Wd, compute_uv=False)
    eps = 0.5 * (s[5] + s[6])
    U0 = syn.orthonormal(m, 6, seed=8)
    V0 = syn.orthonormal(n, 6, seed=9)
    G = syn.gaussian_block(m + n, 2, seed=11)
    ref = oracle.blws_svt_ref(Wd, eps, U0, V0, 3, 8, G)
    sparse = (m, n, torch.from_numpy(P["rowptr"]).cuda(), torch.from_numpy(P["cols"]).cuda(),
              torch.from_numpy(P["vals"]).cuda()) + extra
    ctx = blws.Context(k=3)
    U, V, sig, c = ctx.blws_svt(None, eps, 8, gpu(blws, torch, U0), gpu(blws, torch, V0),
                                gpu(blws, torch, G), sparse=sparse)
    assert c == ref["c"]
    assert rel(recon(U.cpu().numpy(), V.cpu().numpy(), sig.cpu().numpy(), eps), ref["A"]) < A_TOL


def test_deterministic_and_independent_of_call_history(blws, torch_mod):
    torch = torch_mod
    W = gpu(blws, torch, structured(90, 70, 5, seed=12))
    U0 = gpu(blws, torch, syn.orthonormal(90, 6, seed=13))
    V0 = gpu(blws, torch, syn.orthonormal(70, 6, seed=14))
    ctx = blws.Context(k=3)
    out1 = ctx.blws_svt(W, 1.0, 6, U0, V0)
    ctx.blws_svt(gpu(blws, torch, structured(300, 200, 9, seed=15)), 2.0, 12)  # grows buffers
    out2 = ctx.blws_svt(W, 1.0, 6, U0, V0)
    for a, b in zip(out1[:3], out2[:3]):
        assert torch.equal(a, b)
    assert out1[3] == out2[3]


def test_argument_errors(blws, torch_mod):
    torch = torch_mod
    ctx = blws.Context(k=3)
    W = gpu(blws, torch, structured(20, 10, 2, seed=1))
    with pytest.raises(blws.BlwsError) as e:
        ctx.blws_svt(W, 0.0, 2)
    assert e.value.status == blws.EINVAL
    with pytest.raises(blws.BlwsError):
        ctx.blws_svt(W, 1.0, 11)           # r > min(m, n)
    with pytest.raises(blws.BlwsError):
        ctx.blws_svt(W, 1.0, 10)           # k * b = 30 > m + n
