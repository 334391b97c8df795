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
    (200, 200, 10, 11, 11, 3),   # the 200 x 200 rank-10 shape, block 11, k = 3
    (300, 17, 3, 3, 4, 2),       # tall, ragged
    (17, 300, 3, 4, 4, 3),       # wide
    (129, 130, 20, 18, 24, 3),   # width not a multiple of any tile, padding columns
    (513, 257, 30, 33, 33, 2),   # T_k of 66
    (600, 400, 40, 60, 60, 3),   # T_k of 180: the block-pair Jacobi path
    (1, 9, 1, 1, 1, 2),          # a single row
    (700, 700, 60, 150, 150, 3),  # T_k of 450: tridiagonal reduction on a 4-CTA cluster
    (700, 700, 60, 230, 230, 3),  # T_k of 690: tridiagonal reduction on an 8-CTA cluster
]


@pytest.mark.parametrize("m,n,rank,w,r,k", CASES)
def test_blws_svt_matches_oracle(blws, torch_mod, m, n, rank, w, r, k):
    check_blws_svt(blws, torch_mod, m, n, rank, w, r, k, blws.PREC_FP64)


@pytest.mark.parametrize("m,n,rank,w,r,k", [c for c in CASES if c[0] >= 200])
def test_blws_svt_fp64_tensor_core_matches_oracle(blws, torch_mod, m, n, rank, w, r, k):
    # the FP64-equivalent mode: digit-plane products for W~ X and for every
    # product of at least 8e6 multiply-adds (Gram matrices, projections, Ritz
    # lift, eigen refinement), at the same bars
    check_blws_svt(blws, torch_mod, m, n, rank, w, r, k, blws.PREC_FP64_TC)


def check_blws_svt(blws, torch_mod, m, n, rank, w, r, k, precision):
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
    ctx = blws.Context(k=k, precision=precision)
    U, V, sig, c = ctx.blws_svt(gpu(blws, torch, W), eps, r, gpu(blws, torch, U0),
                                gpu(blws, torch, V0), None if G is None else gpu(blws, torch, G))
    U, V, sig = U.cpu().numpy(), V.cpu().numpy(), sig.cpu().numpy()
    assert c == ref["c"]
    if precision == blws.PREC_FP64:
        np.testing.assert_allclose(sig, ref["sigma"], rtol=0, atol=SIG_TOL * s[0])
    else:
        # the values above eps (the ones the thresholded result uses) at the
        # same bar; below eps a pair closer than the eigen refinement's
        # resolution stays a joint subspace (its values are Rayleigh
        # quotients, accurate to ~1e-9 of sigma_1), which is all the next warm
        # start needs
        np.testing.assert_allclose(sig[:c], ref["sigma"][:c], rtol=0, atol=SIG_TOL * s[0])
        np.testing.assert_allclose(sig, ref["sigma"], rtol=0, atol=1e-8 * s[0])
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


@pytest.mark.parametrize("k", [2, 3])
def test_standard_start_matches_oracle(blws, torch_mod, k):
    # start = 1: the one-sided start block [U0; 0] of Section 4.1; the oracle
    # takes it as the mixed start of (sqrt2 U0, 0)
    torch = torch_mod
    m, n, rank, w, r = 120, 90, 6, 6, 8
    W = structured(m, n, rank, seed=21)
    s = np.linalg.svd(W, compute_uv=False)
    eps = 0.5 * (s[rank - 1] + s[rank])
    Up, _, Vpt = np.linalg.svd(W + 0.01 * syn.gaussian_block(m, n, seed=22), full_matrices=False)
    U0, V0 = Up[:, :w], Vpt[:w].T
    G = syn.gaussian_block(m + n, r - w, seed=23)
    ref = oracle.blws_svt_ref(W, eps, U0 * np.sqrt(2.0), 0.0 * V0, k, r, G)
    ctx = blws.Context(k=k, start=1)
    U, V, sig, c = ctx.blws_svt(gpu(blws, torch, W), eps, r, gpu(blws, torch, U0),
                                gpu(blws, torch, V0), gpu(blws, torch, G))
    assert c == ref["c"]
    np.testing.assert_allclose(sig.cpu().numpy(), ref["sigma"], rtol=0, atol=SIG_TOL * s[0])
    assert rel(recon(U.cpu().numpy(), V.cpu().numpy(), sig.cpu().numpy(), eps), ref["A"]) < A_TOL
    # and the mixed start of the same subspaces is closer to the exact SVT (Section 4.1)
    A_exact, _ = oracle.svt_full(W, eps)
    mixed = oracle.blws_svt_ref(W, eps, U0, V0, k, r, G)
    assert np.linalg.norm(mixed["A"] - A_exact) <= np.linalg.norm(ref["A"] - A_exact)


def sym_structured(m, rank, seed, noise=0.05):
    """Symmetric indefinite: a rank-`rank` part with eigenvalues of both signs
    plus symmetric noise, so the top of the spectrum is separated.  Returns
    (W, eps) with eps between the positive signal eigenvalues and the rest."""
    W, npos = syn.symmetric_problem(m, rank, noise, seed)
    lam_all = np.sort(np.linalg.eigvalsh(W))[::-1]
    return W, 0.5 * (lam_all[npos - 1] + lam_all[npos])


EVD_CASES = [
    # m, rank, w (0: cold), r, k
    (40, 4, 4, 5, 2),
    (200, 10, 11, 12, 3),
    (129, 12, 9, 14, 3),      # r > w: extra columns
    (513, 30, 33, 33, 3),
    (37, 3, 0, 6, 4),         # cold start, full reorthogonalisation
    (5, 2, 0, 5, 1),          # r = m: one block is the whole space
]


@pytest.mark.parametrize("m,rank,w,r,k", EVD_CASES)
def test_blws_evd_matches_oracle(blws, torch_mod, m, rank, w, r, k):
    torch = torch_mod
    W, eps = sym_structured(m, rank, seed=m + 3 * rank)
    lam_all = np.sort(np.linalg.eigvalsh(W))[::-1]
    U0 = None
    if w:
        E = syn.gaussian_block(m, m, seed=7)
        _, Qp = np.linalg.eigh(W + 0.005 * (E + E.T))
        U0 = Qp[:, ::-1][:, :w].copy()
    b = max(r, w)
    G = syn.gaussian_block(m, b - w, seed=8) if b > w else None
    ref = oracle.blws_evd_ref(W, eps, U0, k, r, G)
    ctx = blws.Context(k=k, k_cold=k)
    U, lam, c = ctx.blws_evd(gpu(blws, torch, W), eps, r, None if U0 is None else gpu(blws, torch, U0),
                             None if G is None else gpu(blws, torch, G))
    U, lam = U.cpu().numpy(), lam.cpu().numpy()
    scale = np.max(np.abs(lam_all))
    assert c == ref["c"]
    np.testing.assert_allclose(lam, ref["lam"], rtol=0, atol=SIG_TOL * scale)
    # the thresholded part U diag(max(lam - eps, 0)) U^T (unique where the
    # eigenvector signs and bases of near-equal values are not)
    th = np.maximum(lam - eps, 0.0)
    thr = np.maximum(ref["lam"] - eps, 0.0)
    assert rel((U * th) @ U.T, (ref["U"] * thr) @ ref["U"].T) < A_TOL
    np.testing.assert_allclose(U.T @ U, np.eye(r), atol=1e-10)


def test_blws_evd_full_size(blws, torch_mod):
    # m = 3000, 100 pairs.  (1) One warm call from the exact eigenvectors of a
    # nearby matrix matches the oracle's BL_EVD on the same inputs.  (2)
    # Repeated warm calls on one W converge: the residual of the pairs above
    # eps falls each call to the FP64 level, and those Ritz values match
    # LAPACK's eigenvalues.
    torch = torch_mod
    m, rank, r = 3000, 100, 100
    W, eps = sym_structured(m, rank, seed=11)
    lam_all = np.sort(np.linalg.eigvalsh(W))[::-1]
    scale = np.max(np.abs(lam_all))
    E = syn.gaussian_block(m, m, seed=12)
    _, Qp = np.linalg.eigh(W + 1e-3 * (E + E.T))
    U0 = Qp[:, ::-1][:, :r].copy()
    ref = oracle.blws_evd_ref(W, eps, U0, 3, r)
    Wg = gpu(blws, torch, W)
    ctx = blws.Context(k=3)
    U, lam, c = ctx.blws_evd(Wg, eps, r, gpu(blws, torch, U0))
    assert c == ref["c"] == int(np.count_nonzero(lam_all > eps))
    lh, Uh = lam.cpu().numpy(), U.cpu().numpy()
    np.testing.assert_allclose(lh, ref["lam"], rtol=0, atol=SIG_TOL * scale)
    th, thr = np.maximum(lh - eps, 0.0), np.maximum(ref["lam"] - eps, 0.0)
    assert rel((Uh * th) @ Uh.T, (ref["U"] * thr) @ ref["U"].T) < A_TOL
    res = []
    for _ in range(4):
        U, lam, c = ctx.blws_evd(Wg, eps, r, U)
        Rz = Wg @ U[:, :c] - U[:, :c] * lam[:c]
        res.append(float(torch.linalg.matrix_norm(Rz, ord=2)) / scale)
    assert res[1] < res[0] and res[-1] < 1e-9
    np.testing.assert_allclose(lam[:c].cpu().numpy(), lam_all[:c], rtol=0, atol=1e-12 * scale)


def test_blws_evd_argument_errors(blws, torch_mod):
    torch = torch_mod
    W = gpu(blws, torch, sym_structured(20, 2, seed=1)[0])
    ctx = blws.Context(k=3)
    with pytest.raises(blws.BlwsError):
        ctx.blws_evd(W, 0.0, 21)                 # r > m
    with pytest.raises(blws.BlwsError):
        ctx.blws_evd(W, 0.0, 8)                  # cold k_cold * b = 32 > m
    with pytest.raises(blws.BlwsError):
        ctx.blws_evd(W, float("nan"), 2)
