"""Algorithm 1, the single-vector Lanczos procedure (oracle; test infrastructure only).

Paper Section 2, Algorithm 1 and Eq. (5)-(6).  For a symmetric W and a unit
start vector q_1 it builds an orthonormal basis Q_k = (q_1, ..., q_k) of the
Krylov space K(W, q_1, k) and the tridiagonal T_k with diagonal alpha_l and
off-diagonal beta_l, such that W Q_k ~= Q_k T_k.

Reading of the loop bounds: the printed loop is garbled (it increments the
loop counter inside the body).  The procedure here produces k Lanczos vectors
and a k x k matrix T_k, which is what Eq. (6) shows and what the block
procedure of Algorithm 2 produces with k blocks.
"""
import numpy as np


def lanczos_alg1(W, q1, k):
    """Return (Q, alpha, beta): Q is m x k, alpha has k entries, beta k-1.

    Step by step: r_0 = q_1, beta_0 = 1, q_0 = 0; then for l = 1..k:
    q_l = r_{l-1} / beta_{l-1};  alpha_l = q_l^T W q_l;
    r_l = W q_l - alpha_l q_l - beta_{l-1} q_{l-1};  beta_l = ||r_l||_2.
    No reorthogonalisation (Section 2 notes orthogonality is lost as k grows).
    """
    W = np.asarray(W, dtype=np.float64)
    m = W.shape[0]
    q_prev = np.zeros(m)
    r = np.asarray(q1, dtype=np.float64).copy()
    beta_prev = 1.0
    Q = np.zeros((m, k))
    alpha = np.zeros(k)
    beta = np.zeros(k)
    for l in range(k):
        q = r / beta_prev
        Q[:, l] = q
        Wq = W @ q
        alpha[l] = q @ Wq
        # beta_{l-1} q_{l-1}; at l = 0 q_prev is zero so the term vanishes
        r = Wq - alpha[l] * q - (beta[l - 1] if l > 0 else 0.0) * q_prev
        beta[l] = np.linalg.norm(r)
        q_prev = q
        beta_prev = beta[l]
    return Q, alpha, beta[: k - 1]


def tridiag(alpha, beta):
    """T_k of Eq. (6) from its diagonal and off-diagonal."""
    return np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
