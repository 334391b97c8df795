"""Robust PCA by inexact ALM with full-SVD SVT (oracle; test infrastructure only).

Paper Section 5 runs the ADM / inexact augmented Lagrange multiplier method
of its references [Yuan09, Lin09] on the convex RPCA program
    min ||A||_* + lambda ||E||_1   s.t.  D = A + E         (Eq. 1 relaxed, Section 1)
with lambda = 1/sqrt(m) for square m x m data.  The paper does not restate the
host's step rules; the ones below are the published inexact-ALM algorithm of
[Lin09], written out as mathematics:

  Y_0 = D / J(D),  J(D) = max(||D||_2, ||D||_inf / lambda);   E_0 = A_0 = 0
  mu_0 = 1.25 / ||D||_2,  mu_bar = 1e7 * mu_0,  rho = 1.5
  repeat:
      E  <- Theta_{lambda/mu}(D - A + Y/mu)            entrywise shrinkage
      A  <- T_{1/mu}(D - E + Y/mu)                     SVT, Eq. (3)-(4)
      Z  <- D - A - E;  Y <- Y + mu Z;  mu <- min(rho mu, mu_bar)
  until ||Z||_F / ||D||_F < tol

The SVT here is the full SVD (Eq. 4), the baseline of Section 1.  The rank
prediction rule of [Lin09] (``rank_predict``) is tracked so that tests can
compare the predicted-rank trajectory; it does not change a full-SVD result.
"""
import math

import numpy as np

from .svt import theta, svt_factored


def rank_predict(sv, svp, n):
    """[Lin09] rank prediction: grow by one past the count, or by 5% of n."""
    if svp < sv:
        return min(svp + 1, n)
    return min(svp + int(round(0.05 * n)), n)


def rpca_ialm_full(D, lam=None, tol=1e-7, max_iter=1000, rho=1.5, sv0=10,
                   mu0_factor=1.25, mu_bar_ratio=1e7, progress=None):
    """Inexact-ALM RPCA with full-SVD SVT.  Returns a dict of results.

    ``progress`` (optional, for timing only) is called with no arguments once
    the set-up (||D||_2, Y_0, mu_0) is done and again at the end of every
    iteration; it sees none of the arithmetic."""
    D = np.asarray(D, dtype=np.float64)
    m, n = D.shape
    if lam is None:
        lam = 1.0 / math.sqrt(max(m, n))
    norm_two = float(np.linalg.svd(D, compute_uv=False)[0])
    norm_inf = float(np.max(np.abs(D))) / lam
    J = max(norm_two, norm_inf)
    Y = D / J
    A = np.zeros_like(D)
    E = np.zeros_like(D)
    mu = mu0_factor / norm_two
    mu_bar = mu * mu_bar_ratio
    d_norm = float(np.linalg.norm(D, "fro"))
    sv = sv0
    hist = []
    svp = 0
    it = 0
    if progress:
        progress()
    for it in range(1, max_iter + 1):
        E = theta(D - A + Y / mu, lam / mu)
        U, th, V, svp = svt_factored(D - E + Y / mu, 1.0 / mu)
        A = (U * th) @ V.T
        sv = rank_predict(sv, svp, n)
        Z = D - A - E
        Y = Y + mu * Z
        mu = min(mu * rho, mu_bar)
        res = float(np.linalg.norm(Z, "fro")) / d_norm
        hist.append((res, svp, sv))
        if progress:
            progress()
        if res < tol:
            break
    return {"A": A, "E": E, "Y": Y, "iters": it, "rank": svp,
            "nnzE": int(np.count_nonzero(E)), "residual": hist[-1][0],
            "history": hist, "lam": lam, "norm_two": norm_two}


def rpca_ialm_blws(D, extra_cols, lam=None, tol=1e-7, max_iter=1000, rho=1.5,
                   sv0=10, k=3, k_cold=4, mu0_factor=1.25, mu_bar_ratio=1e7):
    """BLWS-ADM of Section 5 / Table 1: the same inexact ALM with each SVT
    evaluated by BLWS (Sections 4, 4.1, 4.2) instead of a full SVD.

    ``extra_cols(rows, cols)`` supplies start columns (seeded Gaussian): the
    whole cold-start block at the first iteration, and the columns that pad
    the warm block when the predicted rank sv exceeds the w columns output
    last time (block width b = max(sv, w)).  The first SVT runs block Lanczos
    from that cold block for ``k_cold`` blocks with full reorthogonalisation;
    every later one restarts from the previous (U, V) for ``k`` blocks.
    """
    from .blws import blws_svt_ref, cold_svt_ref
    D = np.asarray(D, dtype=np.float64)
    m, n = D.shape
    if lam is None:
        lam = 1.0 / math.sqrt(max(m, n))
    norm_two = float(np.linalg.svd(D, compute_uv=False)[0])
    J = max(norm_two, float(np.max(np.abs(D))) / lam)
    Y = D / J
    A = np.zeros_like(D)
    E = np.zeros_like(D)
    mu = mu0_factor / norm_two
    mu_bar = mu * mu_bar_ratio
    d_norm = float(np.linalg.norm(D, "fro"))
    sv = sv0
    U = V = None
    hist = []
    svp = 0
    it = 0
    for it in range(1, max_iter + 1):
        E = theta(D - A + Y / mu, lam / mu)
        W = D - E + Y / mu
        if U is None:
            res = cold_svt_ref(W, 1.0 / mu, extra_cols(m + n, sv), k_cold, sv)
        else:
            w = U.shape[1]
            b = max(sv, w)
            G = extra_cols(m + n, b - w) if b > w else None
            res = blws_svt_ref(W, 1.0 / mu, U, V, k, sv, G)
        U, V, svp = res["U"], res["V"], res["c"]
        A = res["A"]
        sv = rank_predict(sv, svp, n)
        Z = D - A - E
        Y = Y + mu * Z
        mu = min(mu * rho, mu_bar)
        r = float(np.linalg.norm(Z, "fro")) / d_norm
        hist.append((r, svp, sv))
        if r < tol:
            break
    return {"A": A, "E": E, "Y": Y, "iters": it, "rank": svp,
            "nnzE": int(np.count_nonzero(E)), "residual": hist[-1][0],
            "history": hist, "lam": lam, "norm_two": norm_two}
