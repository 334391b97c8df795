"""Pins for the oracle's block Lanczos with warm start: Theorem 1, the
invariants of Algorithm 2, the b = 1 reduction to Algorithm 1, exactness
under an exact warm start (Section 3), and exactness once the Krylov space is
the whole space."""
import numpy as np
import pytest

import oracle
from oracle.blws import augmented, apply_augmented, block_lanczos, assemble_T
from oracle.lanczos import lanczos_alg1, tridiag
from paper_1012_0365_gb300 import synthetic as syn


@pytest.mark.parametrize("m,n", [(3, 5), (5, 3), (4, 4)])
def test_theorem1_spectrum_and_vectors(m, n):
    # Theorem 1: eig(W~) = {+sigma_i} U {-sigma_i} U {0 x |m-n|},
    # eigenvectors (u_i; +-v_i)/sqrt(2).
    W = syn.gaussian_block(m, n, seed=m * 10 + n)
    U, s, Vt = np.linalg.svd(W)
    lam, Z = np.linalg.eigh(augmented(W))
    want = np.sort(np.concatenate([s, -s, np.zeros(abs(m - n))]))
    np.testing.assert_allclose(lam, want, atol=1e-12)
    p = min(m, n)
    for i in range(p):
        top = Z[:, np.argmin(np.abs(lam - s[i]))]
        ref = np.concatenate([U[:, i], Vt[i]]) / np.sqrt(2)
        assert abs(abs(top @ ref) - 1) < 1e-10
        bot = Z[:, np.argmin(np.abs(lam + s[i]))]
        ref = np.concatenate([U[:, i], -Vt[i]]) / np.sqrt(2)
        assert abs(abs(bot @ ref) - 1) < 1e-10


def test_apply_augmented_skips_zero_blocks_exactly():
    W = syn.gaussian_block(7, 4, seed=5)
    X = syn.gaussian_block(11, 3, seed=6)
    np.testing.assert_allclose(apply_augmented(W, X), augmented(W) @ X, atol=1e-13)


@pytest.mark.parametrize("k,b", [(2, 3), (3, 4), (4, 2)])
def test_alg2_invariants(k, b):
    # Q_k orthonormal, T_k symmetric and W~ Q_k = Q_k T_k + R_k E_k^T (Eq. 12).
    W = syn.gaussian_block(20, 16, seed=k * 7 + b)
    op = lambda X: apply_augmented(W, X)
    X1, _ = np.linalg.qr(syn.gaussian_block(36, b, seed=b))
    Xs, Ms, Bs, Rk = block_lanczos(op, X1, k)
    Q = np.hstack(Xs)
    T = assemble_T(Ms, Bs)
    np.testing.assert_allclose(Q.T @ Q, np.eye(k * b), atol=1e-12)
    np.testing.assert_allclose(T, T.T, atol=0)
    lhs = op(Q)
    rhs = Q @ T
    rhs[:, (k - 1) * b:] += Rk
    np.testing.assert_allclose(lhs, rhs, atol=1e-11 * np.abs(lhs).max())
    # B_l is upper triangular (the R factor of the QR of R_l)
    for B in Bs:
        np.testing.assert_allclose(np.tril(B, -1), 0, atol=0)


def test_alg1_full_krylov_reproduces_spectrum():
    # Algorithm 1 with k = size: T_k is similar to W, so eig(T_k) = eig(W).
    A = syn.gaussian_block(6, 6, seed=11)
    W = A + A.T
    q1 = syn.gaussian_block(6, 1, seed=12)[:, 0]
    q1 /= np.linalg.norm(q1)
    Q, alpha, beta = lanczos_alg1(W, q1, 6)
    np.testing.assert_allclose(np.linalg.eigvalsh(tridiag(alpha, beta)),
                               np.linalg.eigvalsh(W), atol=1e-9)
    np.testing.assert_allclose(Q.T @ W @ Q, tridiag(alpha, beta), atol=1e-9)


def test_block_b1_reduces_to_alg1():
    # Algorithm 2 with one column per block is Algorithm 1 (Section 4).
    W = syn.gaussian_block(9, 8, seed=13)
    Wt = augmented(W)
    q1 = syn.gaussian_block(17, 1, seed=14)
    q1 /= np.linalg.norm(q1)
    k = 5
    Q1, alpha, beta = lanczos_alg1(Wt, q1[:, 0], k)
    Xs, Ms, Bs, _ = block_lanczos(lambda X: apply_augmented(W, X), q1, k)
    np.testing.assert_allclose([M[0, 0] for M in Ms], alpha, atol=1e-10)
    np.testing.assert_allclose([abs(B[0, 0]) for B in Bs], beta, atol=1e-10)
    for l in range(k):
        assert abs(abs(Xs[l][:, 0] @ Q1[:, l]) - 1) < 1e-9


def _known_svd(m, n, s, seed):
    p = len(s)
    U = syn.orthonormal(m, p, seed=seed)
    V = syn.orthonormal(n, p, seed=seed + 1)
    return U, V, (U * s) @ V.T


@pytest.mark.parametrize("k", [2, 3])
def test_exact_warm_start_is_exact(k):
    # Section 3/4: a start block spanning a paired top singular subspace is
    # invariant under W~, R_1 = 0 (deflated), and BLWS returns T_eps(W) exactly.
    s = np.array([10.0, 8.0, 6.0, 4.0, 2.0, 1.0, 0.5])
    U, V, W = _known_svd(12, 9, s, seed=20)
    r = 4
    out = oracle.blws_svt_ref(W, 3.0, U[:, :r], V[:, :r], k, r)
    A, c = oracle.svt_full(W, 3.0)
    np.testing.assert_allclose(out["A"], A, atol=1e-12 * np.abs(A).max())
    np.testing.assert_allclose(out["sigma"], s[:r], atol=1e-12)
    assert out["c"] == c == 4


def test_whole_space_krylov_is_exact():
    # k*b >= m + n: the Krylov space is everything, Ritz pairs are exact.
    W = syn.gaussian_block(5, 4, seed=30)
    U0 = syn.gaussian_block(5, 3, seed=31)
    V0 = syn.gaussian_block(4, 3, seed=32)
    eps = 0.7
    out = oracle.blws_svt_ref(W, eps, U0, V0, k=3, r=4)
    A, c = oracle.svt_full(W, eps)
    np.testing.assert_allclose(out["sigma"], np.linalg.svd(W, compute_uv=False), atol=1e-10)
    np.testing.assert_allclose(out["A"], A, atol=1e-10)
    assert out["c"] == c


def test_cold_start_whole_space_is_exact():
    W = syn.gaussian_block(6, 5, seed=40)
    G = syn.gaussian_block(11, 4, seed=41)
    out = oracle.cold_svt_ref(W, 0.5, G, k=3, r=5)
    A, c = oracle.svt_full(W, 0.5)
    np.testing.assert_allclose(out["A"], A, atol=1e-10)


def test_warm_start_error_shrinks_with_perturbation():
    # Section 4.1: W_i close to W_{i-1} makes a few steps accurate.  BLWS
    # started from W's top subspace and applied to W + d G has an error that
    # falls in proportion to d, and each extra block step divides it by about
    # the gap ratio sigma_7 / sigma_6 = 0.2 (Discussion, Section 6).
    s = np.concatenate([np.linspace(20, 10, 6), np.linspace(2, 0.1, 14)])
    U, V, W = _known_svd(40, 30, s, seed=50)
    G = syn.gaussian_block(40, 30, seed=51)
    errs = {2: [], 3: []}
    for d in (1e-2, 1e-3, 1e-4, 1e-5):
        Wd = W + d * G
        A, _ = oracle.svt_full(Wd, 5.0)
        for k in (2, 3):
            out = oracle.blws_svt_ref(Wd, 5.0, U[:, :6], V[:, :6], k=k, r=6)
            errs[k].append(np.linalg.norm(out["A"] - A) / np.linalg.norm(A))
    for k in (2, 3):
        ratios = np.array(errs[k][:-1]) / np.array(errs[k][1:])
        assert np.all((ratios > 8) & (ratios < 12)), ratios
    assert all(e3 < 0.3 * e2 for e2, e3 in zip(errs[2], errs[3]))
    assert errs[3][-1] < 1e-6


def test_mixed_start_beats_one_sided_start():
    # Section 4.1: the mixed start (U;V)/sqrt2 gives higher precision than the
    # standard (U;0) start for the same number of steps.
    s = np.concatenate([np.linspace(20, 10, 5), np.linspace(3, 0.1, 25)])
    U, V, W = _known_svd(50, 40, s, seed=60)
    G = syn.gaussian_block(50, 40, seed=61)
    Wd = W + 0.3 * G
    A, _ = oracle.svt_full(Wd, 5.0)
    mixed = oracle.blws_svt_ref(Wd, 5.0, U[:, :5], V[:, :5], k=2, r=5)
    one_sided = oracle.blws_svt_ref(Wd, 5.0, U[:, :5] * np.sqrt(2), 0 * V[:, :5], k=2, r=5)
    e_mixed = np.linalg.norm(mixed["A"] - A)
    e_one = np.linalg.norm(one_sided["A"] - A)
    assert e_mixed < e_one


def test_qr_deflation_of_a_dependent_middle_column():
    # Alg. 2 "qr" with deflation: a column in the span of earlier ones dies,
    # keeps its coefficients in B, and leaks no direction into later columns.
    rng = np.random.default_rng(70)
    R = rng.standard_normal((30, 4))
    R[:, 1] = 2.0 * R[:, 0]  # exactly dependent on column 0
    X, B = oracle.qr_deflate(R, scale=np.linalg.norm(R, axis=0).max())
    assert np.all(X[:, 1] == 0) and np.all(B[1, :] == 0)
    live = [0, 2, 3]
    np.testing.assert_allclose(X[:, live].T @ X[:, live], np.eye(3), atol=1e-14)
    np.testing.assert_allclose(X @ B, R, atol=1e-12)
    # later columns stay in span(R): no component outside it
    P = R @ np.linalg.pinv(R)
    np.testing.assert_allclose(P @ X, X, atol=1e-12)


def test_blws_adm_stable_far_past_convergence():
    # BLWS inside inexact ALM run to tol 1e-15 on a case where a deflated
    # column occurs late: the count of values above eps stays at the rank.
    from paper_1012_0365_gb300 import synthetic as s2
    D, L0, _ = s2.rpca_problem(47, 61, 3, 0.05, seed=2)
    rng = np.random.default_rng(3)
    out = oracle.rpca_ialm_blws(D, lambda r, c: rng.standard_normal((r, c)), tol=1e-15, max_iter=45)
    assert max(h[1] for h in out["history"][10:]) == 3
    assert min(h[0] for h in out["history"]) < 1e-12


def _sym_with_spectrum(lam, seed):
    Q = syn.orthonormal(len(lam), len(lam), seed=seed)
    return (Q * np.asarray(lam, float)) @ Q.T, Q


def test_evd_whole_space_is_exact_and_algebraic():
    # BL_EVD on a symmetric indefinite W: once k*b = m the Krylov space is the
    # whole space, so the Ritz pairs are W's eigenpairs, ordered algebraically
    # (-12 has the largest magnitude but is not among the top four).
    lam = [9.0, 7.0, 4.0, 1.0, -0.5, -3.0, -12.0, 0.25, 2.5, -6.0, 5.5, -1.5]
    W, Q = _sym_with_spectrum(lam, seed=40)
    G = syn.gaussian_block(12, 4, seed=41)
    out = oracle.blws_evd_ref(W, 2.0, None, 3, 4, G)
    np.testing.assert_allclose(out["lam"], [9.0, 7.0, 5.5, 4.0], atol=1e-12)
    assert out["c"] == 4
    want = Q[:, [0, 1, 10, 2]]
    np.testing.assert_allclose(np.abs(np.sum(out["U"] * want, axis=0)), 1.0, atol=1e-10)
    np.testing.assert_allclose(W @ out["U"], out["U"] * out["lam"], atol=1e-11)


@pytest.mark.parametrize("k", [1, 2])
def test_evd_exact_warm_start_is_exact(k):
    # an invariant start block (the exact leading eigenvectors) gives R_1 = 0:
    # the leading eigenpairs come out exactly for any k
    lam = np.array([10.0, 6.0, 3.0, -1.0, -2.0, 0.5, 1.5, -8.0, 2.0, 0.0])
    W, Q = _sym_with_spectrum(lam, seed=42)
    out = oracle.blws_evd_ref(W, 0.0, Q[:, :3], k, 3)
    np.testing.assert_allclose(out["lam"], [10.0, 6.0, 3.0], atol=1e-12)
    np.testing.assert_allclose(np.abs(np.sum(out["U"] * Q[:, :3], axis=0)), 1.0, atol=1e-12)


def test_evd_warm_start_error_shrinks_with_perturbation():
    # Section 4.1's argument for BL_EVD: warm-started from the eigenvectors of
    # a nearby W_{i-1}, a small k recovers W_i's leading pairs with an error
    # that falls with the distance between the two
    lam = np.concatenate([[20.0, 15.0, 12.0, 10.0], np.linspace(-1.0, 1.0, 56)])
    W0, Q = _sym_with_spectrum(lam, seed=43)
    E = syn.gaussian_block(60, 60, seed=44)
    E = (E + E.T) / 2
    errs = {1: [], 2: [], 3: []}
    for delta in (1e-1, 1e-2, 1e-3):
        W = W0 + delta * E
        ref = np.sort(np.linalg.eigvalsh(W))[::-1][:4]
        for k in errs:
            out = oracle.blws_evd_ref(W, 5.0, Q[:, :4], k, 4)
            errs[k].append(np.max(np.abs(out["lam"] - ref)))
    for k, e in errs.items():
        assert e[0] > e[1] > e[2]          # falls with the distance
    for i in range(3):
        assert errs[1][i] > errs[2][i] > errs[3][i]   # and with more blocks
    assert errs[2][2] < 1e-7 and errs[3][2] < 1e-9


def test_evd_of_augmented_matrix_gives_singular_values():
    # Theorem 1 link: BL_EVD on the explicit W~ from the mixed start is the
    # SVD-side procedure, so its Ritz values are the singular-value estimates
    W = syn.gaussian_block(9, 7, seed=45)
    U, s, Vt = np.linalg.svd(W)
    X0 = np.vstack([U[:, :3], Vt[:3].T]) / np.sqrt(2.0)
    out = oracle.blws_evd_ref(augmented(W), 0.5, X0, 2, 3)
    np.testing.assert_allclose(out["lam"], s[:3], atol=1e-12)


def test_warm_start_block_is_the_mixed_start_orthonormalised():
    # Section 4.1: X~_1 = [U; V] / sqrt(2); with orthonormal U, V its columns are
    # already orthonormal, so the QR keeps them (up to sign) and appends the
    # extra columns' orthogonal complement
    U = syn.orthonormal(20, 3, seed=50)
    V = syn.orthonormal(15, 3, seed=51)
    G = syn.gaussian_block(35, 2, seed=52)
    X = oracle.warm_start_block(U, V, G)
    np.testing.assert_allclose(X.T @ X, np.eye(5), atol=1e-13)
    mixed = np.vstack([U, V]) / np.sqrt(2.0)
    np.testing.assert_allclose(np.abs(np.sum(X[:, :3] * mixed, axis=0)), 1.0, atol=1e-13)
    # the extra columns lie in span(mixed, G)
    B = np.hstack([mixed, G])
    P = B @ np.linalg.lstsq(B, X[:, 3:], rcond=None)[0]
    np.testing.assert_allclose(P, X[:, 3:], atol=1e-12)
