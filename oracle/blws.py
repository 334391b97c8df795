"""Block Lanczos with warm start on the augmented matrix (oracle; test infrastructure only).

Paper references (all by section / equation / algorithm):
  * Eq. (7) and Theorem 1 (Section 2): W~ = [[0, W], [W^T, 0]] has eigenvalues
    +-sigma_i plus |m - n| zeros, with eigenvectors (u_i; +-v_i)/sqrt(2).
  * Eq. (10)-(13), Algorithm 2 (Section 4): the block Lanczos procedure.
      M_1 = X_1^T W X_1;  for l = 1..k-1:
          R_l = W X_l - X_l M_l - X_{l-1} B_{l-1}^T,  (X_{l+1}, B_l) = qr(R_l),
          M_{l+1} = X_{l+1}^T W X_{l+1}.
  * Eq. (11): T_k is block tridiagonal, M_l on the diagonal, B_l below and
    B_l^T above it.
  * Algorithm 3: EVD of T_k with eigenvalues in decreasing order; the leading r
    Ritz pairs are Lambda(1:r) and Q_k V_k(:, 1:r).
  * Section 4, end: the procedure runs on W~ by skipping its zero blocks, i.e.
    W~ [X_u; X_v] = [W X_v; W^T X_u].
  * Section 4.1: small k (typically 2) and no reorthogonalisation; the mixed
    start X~_1 = (1/sqrt 2) (U_{i-1}; V_{i-1}).
  * Section 4.2: the number r of Ritz pairs output follows the predicted rank
    while the start block is the previous output.

Readings where the paper is silent (each listed in the design notes):
  * U and V are the sqrt(2)-scaled halves of the Ritz vectors of W~
    (Theorem 1 read backwards).
  * "Decreasing order" is algebraic, so the +sigma side comes first.
  * The start block is orthonormalised by a QR of the stacked block, warm
    columns first, extra columns (passed in, e.g. seeded Gaussian) after.
  * R_l is projected once more against X_l and X_{l-1} (the blocks the
    three-term recurrence already uses) before its QR.  With a warm start
    R_l is small, so its computed direction carries rounding error of
    relative size u ||W X_l|| / ||R_l|| along X_l; without this second pass
    Q_k loses orthogonality as the outer solver converges, spurious Ritz
    values appear and the host diverges (observed at k = 3).  It costs
    O((m + n) b^2), not a pass over W, and touches no older block.
  * ``full_reorth=True`` (cold start only, when there is no previous
    subspace) projects R_l against every previous block instead.
  * qr(R_l) deflates: Gram-Schmidt (twice per column) in column order; a
    column whose remainder is below ``DEFL_TOL * scale`` is set to zero in
    X_{l+1} and its row in B_l to zero.  ``scale`` is the largest column norm
    of W~ X_1.  (Householder QR followed by zeroing dead columns is not the
    same: it gives a dead column an arbitrary direction that leaks into the
    later columns.)
  * Theta is applied to the Ritz values as max(lambda - eps, 0): singular
    values are nonnegative, so a Ritz value <= eps contributes nothing.
"""
import numpy as np

DEFL_TOL = 1e-12


def augmented(W):
    """Explicit W~ of Eq. (7); for tiny test cases only."""
    W = np.asarray(W, dtype=np.float64)
    m, n = W.shape
    Wt = np.zeros((m + n, m + n))
    Wt[:m, m:] = W
    Wt[m:, :m] = W.T
    return Wt


def apply_augmented(W, X):
    """W~ X computed without forming W~ (zero blocks skipped, Section 4).

    X has m + n rows: the first m are the u-part, the last n the v-part.
    """
    W = np.asarray(W, dtype=np.float64)
    m = W.shape[0]
    return np.vstack([W @ X[m:], W.T @ X[:m]])


def qr_deflate(R, scale):
    """(X, B) = qr(R) with deflation, by Gram-Schmidt run twice per column.

    Column j is orthogonalised (twice) against the earlier live columns; if
    what remains has norm <= DEFL_TOL * scale the column is dead: its column
    of X and its row of B are zero, and its coefficients on the earlier
    columns stay in B, so R = X B up to the dropped remainders.
    """
    N, b = R.shape
    X = np.zeros((N, b))
    B = np.zeros((b, b))
    live = []
    for j in range(b):
        v = np.array(R[:, j], dtype=np.float64)
        for _ in range(2):
            if live:
                c = X[:, live].T @ v
                v = v - X[:, live] @ c
                B[live, j] += c
        nrm = float(np.linalg.norm(v))
        if nrm > DEFL_TOL * scale:
            X[:, j] = v / nrm
            B[j, j] = nrm
            live.append(j)
    return X, B


def _sym(M):
    # M_l = X_l^T W~ X_l is symmetric in exact arithmetic; keep it symmetric.
    return 0.5 * (M + M.T)


def block_lanczos(apply, X1, k, full_reorth=False):
    """Algorithm 2 for a symmetric operator ``apply`` (X -> W X).

    Returns (Xs, Ms, Bs, R_k): the k blocks X_1..X_k, the k diagonal blocks
    M_l, the k-1 off-diagonal blocks B_l, and the final residual
    R_k = W X_k - X_k M_k - X_{k-1} B_{k-1}^T (used only to check the
    three-term recurrence W Q_k = Q_k T_k + R_k E_k^T).
    """
    Xs, Ms, Bs = [X1], [], []
    P = apply(X1)
    scale = max(float(np.max(np.linalg.norm(P, axis=0))), np.finfo(float).tiny)
    Ms.append(_sym(X1.T @ P))
    for l in range(k - 1):
        R = P - Xs[l] @ Ms[l]
        if l > 0:
            R = R - Xs[l - 1] @ Bs[l - 1].T
        for Xj in (Xs if full_reorth else Xs[max(l - 1, 0):l + 1]):
            R = R - Xj @ (Xj.T @ R)
        Xn, Bn = qr_deflate(R, scale)
        Xs.append(Xn)
        Bs.append(Bn)
        P = apply(Xn)
        Ms.append(_sym(Xn.T @ P))
    Rk = P - Xs[-1] @ Ms[-1]
    if k > 1:
        Rk = Rk - Xs[-2] @ Bs[-1].T
    return Xs, Ms, Bs, Rk


def assemble_T(Ms, Bs):
    """Block tridiagonal T_k of Eq. (11)."""
    b = Ms[0].shape[0]
    k = len(Ms)
    T = np.zeros((k * b, k * b))
    for l in range(k):
        T[l * b:(l + 1) * b, l * b:(l + 1) * b] = Ms[l]
    for l in range(k - 1):
        T[(l + 1) * b:(l + 2) * b, l * b:(l + 1) * b] = Bs[l]
        T[l * b:(l + 1) * b, (l + 1) * b:(l + 2) * b] = Bs[l].T
    return T


def bl_evd(apply, X1, k, r, full_reorth=False):
    """Algorithm 3: (U, lam) = (Q_k V_k(:, 1:r), Lambda_k(1:r)), decreasing order."""
    Xs, Ms, Bs, _ = block_lanczos(apply, X1, k, full_reorth)
    T = assemble_T(Ms, Bs)
    lam, Z = np.linalg.eigh(T)          # ascending
    order = np.argsort(-lam, kind="stable")
    lam = lam[order][:r]
    Z = Z[:, order][:, :r]
    Q = np.hstack(Xs)
    return Q @ Z, lam


def warm_start_block(U0, V0, G=None):
    """Mixed start of Section 4.1, orthonormalised: qr([U0; V0]/sqrt(2) | G).

    U0 is m x w, V0 is n x w (the previous principal subspaces); G is an
    optional (m + n) x e block of extra start columns, placed after the warm
    ones, used when the predicted rank exceeds w (Section 4.2).
    """
    X = np.vstack([np.asarray(U0, float), np.asarray(V0, float)]) / np.sqrt(2.0)
    if G is not None and G.shape[1] > 0:
        X = np.hstack([X, np.asarray(G, float)])
    Q, _ = np.linalg.qr(X, mode="reduced")
    return Q


def cold_svt_ref(W, eps, G, k, r):
    """T_eps(W) from a cold start (no previous subspace): block Lanczos on W~
    from the orthonormalised start block G ((m + n) x b, e.g. seeded
    Gaussian) with full reorthogonalisation; same outputs as blws_svt_ref."""
    W = np.asarray(W, dtype=np.float64)
    m, n = W.shape
    X1, _ = np.linalg.qr(np.asarray(G, float), mode="reduced")
    Y, lam = bl_evd(lambda X: apply_augmented(W, X), X1, k, r, full_reorth=True)
    return _svt_from_ritz(Y, lam, eps, m)


def _svt_from_ritz(Y, lam, eps, m):
    U = np.sqrt(2.0) * Y[:m]
    V = np.sqrt(2.0) * Y[m:]
    th = np.maximum(lam - eps, 0.0)
    c = int(np.count_nonzero(lam > eps))
    A = (U * th) @ V.T
    return {"sigma": lam, "U": U, "V": V, "th": th, "c": c, "A": A}


def blws_svt_ref(W, eps, U0, V0, k, r, G=None):
    """One BLWS evaluation of T_eps(W) (Sections 4, 4.1, 4.2; Eq. 4).

    Returns a dict with the Ritz values ``sigma`` (r, decreasing), the factors
    ``U`` (m x r) and ``V`` (n x r), the thresholded values ``th``, the count
    ``c = #{sigma > eps}`` and the dense ``A = U diag(th) V^T``.
    """
    W = np.asarray(W, dtype=np.float64)
    m, n = W.shape
    X1 = warm_start_block(U0, V0, G)
    Y, lam = bl_evd(lambda X: apply_augmented(W, X), X1, k, r)
    return _svt_from_ritz(Y, lam, eps, m)


def blws_evd_ref(W, eps, U0, k, r, G=None):
    """BL_EVD of a symmetric W warm-started from its previous principal
    eigen-subspace: the BLWS definition of Section 4,
    (U_i, Lambda_i) = BL_EVD(W_i, U_{i-1}, k_i), with Algorithms 2 and 3 run on
    W itself.

    U0 is m x w (w may be 0: a cold start, which then needs G); G is an
    optional m x e block of extra start columns after the warm ones.  The
    start block is qr([U0 | G]).  A cold start (w = 0) reorthogonalises fully,
    as for the SVD.  Returns ``lam`` (r, decreasing algebraically), ``U``
    (m x r) and ``c = #{lam > eps}``.
    """
    W = np.asarray(W, dtype=np.float64)
    m = W.shape[0]
    blocks = [np.asarray(U0, float).reshape(m, -1)] if U0 is not None else []
    if G is not None and G.shape[1] > 0:
        blocks.append(np.asarray(G, float))
    X1, _ = np.linalg.qr(np.hstack(blocks), mode="reduced")
    cold = U0 is None or np.asarray(U0).size == 0
    U, lam = bl_evd(lambda X: W @ X, X1, k, r, full_reorth=cold)
    return {"lam": lam, "U": U, "c": int(np.count_nonzero(lam > eps))}
