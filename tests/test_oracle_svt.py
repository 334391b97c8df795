"""Pins for the oracle's SVT (Eq. 3-4) against closed forms, an independent C
Jacobi SVD, and the optimality condition of Eq. (3)."""
import numpy as np
import pytest

import oracle
from oracle.cjacobi import jacobi_svd
from paper_1012_0365_gb300 import synthetic as syn


def test_theta_closed_form():
    # Eq. (4): Theta_eps(x) = sgn(x) max(|x| - eps, 0), with sgn(0) = 0.
    x = np.array([3.0, -3.0, 0.5, -0.5, 1.0, -1.0, 0.0, 1.0 + 1e-12])
    got = oracle.theta(x, 1.0)
    want = np.array([2.0, -2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1e-12])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)
    assert np.all(np.sign(got[got != 0]) == np.sign(x[got != 0]))


@pytest.mark.parametrize("m,n", [(7, 5), (5, 7), (6, 6), (30, 12)])
def test_svt_constructed_svd(m, n):
    # W = U* diag(s*) V*^T with known factors: T_eps(W) = U* diag(max(s*-eps,0)) V*^T.
    p = min(m, n)
    U = syn.orthonormal(m, p, seed=1)
    V = syn.orthonormal(n, p, seed=2)
    s = np.linspace(10.0, 0.5, p)
    W = (U * s) @ V.T
    eps = 3.3
    A, c = oracle.svt_full(W, eps)
    want = (U * np.maximum(s - eps, 0)) @ V.T
    np.testing.assert_allclose(A, want, atol=1e-12 * np.abs(want).max())
    assert c == int(np.sum(s > eps))


def test_svt_value_at_threshold_is_dropped():
    # sigma == eps maps to 0 and is not counted (strict inequality, Eq. 4).
    U = syn.orthonormal(6, 3, seed=3)
    V = syn.orthonormal(5, 3, seed=4)
    s = np.array([4.0, 2.0, 1.0])
    W = (U * s) @ V.T
    # pick eps exactly at the computed second singular value
    eps = np.linalg.svd(W, compute_uv=False)[1]
    A, c = oracle.svt_full(W, eps)
    assert c == 1
    np.testing.assert_allclose(A, np.outer(U[:, 0], V[:, 0]) * (4.0 - eps), atol=1e-12)


@pytest.mark.parametrize("m,n,seed", [(6, 4, 0), (4, 9, 1), (12, 12, 2), (11, 3, 3)])
def test_svt_matches_c_jacobi(m, n, seed):
    # Brute force: the same SVT evaluated with an independent C Jacobi SVD.
    W = syn.gaussian_block(m, n, seed=seed)
    Uj, sj, Vj = jacobi_svd(W)
    np.testing.assert_allclose(Uj @ np.diag(sj) @ Vj.T, W, atol=1e-12)
    np.testing.assert_allclose(sj, np.linalg.svd(W, compute_uv=False), rtol=1e-12)
    eps = 0.5 * float(sj[len(sj) // 2 - 1] + sj[len(sj) // 2])
    A, c = oracle.svt_full(W, eps)
    Aj = (Uj * np.maximum(sj - eps, 0)) @ Vj.T
    np.testing.assert_allclose(A, Aj, atol=1e-11)
    assert c == int(np.sum(sj > eps))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_svt_optimality_condition(seed):
    # Eq. (3): A = T_eps(W) iff W - A lies in eps * subdifferential of ||A||_*,
    # i.e. W - A = eps (U V^T + R) with U^T R = 0, R V = 0, ||R||_2 <= 1.
    W = syn.gaussian_block(15, 11, seed=seed) * 3
    eps = 4.0
    U, th, V, c = oracle.svt_factored(W, eps)
    A = (U * th) @ V.T
    G = (W - A) / eps
    assert np.linalg.norm(G, 2) <= 1 + 1e-12
    np.testing.assert_allclose(U.T @ G @ V, np.eye(c), atol=1e-12)
    # and A beats random perturbations on the objective of Eq. (3)
    f = lambda X: eps * np.linalg.svd(X, compute_uv=False).sum() + 0.5 * np.linalg.norm(X - W) ** 2
    rng = np.random.default_rng(seed)
    f0 = f(A)
    for _ in range(20):
        assert f(A + 1e-3 * rng.standard_normal(A.shape)) >= f0 - 1e-12
