"""Singular value thresholding by full SVD (oracle; test infrastructure only).

Paper, Section 1, Eq. (3)-(4): the minimiser of  eps*||A||_* + 0.5*||A - W||_F^2
is  T_eps(W) = U Theta_eps(S) V^T  where  U S V^T  is the SVD of W and
Theta_eps(x) = sgn(x) * max(|x| - eps, 0)  acts entrywise.  The full SVD is
the O(p^3) baseline the paper measures against (Section 1, after Eq. (4)).
"""
import numpy as np


def theta(x, eps):
    """Shrinkage operator of Eq. (4), entrywise: sgn(x) * max(|x| - eps, 0).

    sgn(0) = 0, so an entry with |x| <= eps maps to exactly 0.
    """
    x = np.asarray(x, dtype=np.float64)
    return np.sign(x) * np.maximum(np.abs(x) - eps, 0.0)


def svt_factored(W, eps):
    """Factored T_eps(W) by full LAPACK SVD (Eq. 4).

    Returns (U, th, V, c): U is m x c, th the c thresholded singular values
    (descending), V is n x c, and c = #{sigma_i > eps} (strict inequality: a
    singular value equal to eps maps to 0 and is not counted).
    """
    W = np.asarray(W, dtype=np.float64)
    U, s, Vt = np.linalg.svd(W, full_matrices=False)
    c = int(np.count_nonzero(s > eps))
    th = theta(s[:c], eps)
    return U[:, :c], th, Vt[:c].T, c


def svt_full(W, eps):
    """Dense T_eps(W) = U diag(max(s - eps, 0)) V^T and the count c (Eq. 4)."""
    U, th, V, c = svt_factored(W, eps)
    A = (U * th) @ V.T if c else np.zeros_like(np.asarray(W, dtype=np.float64))
    return A, c
