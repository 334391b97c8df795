"""Matrix completion hosts with full-SVD SVT (oracle; test infrastructure only).

Paper Section 5 solves the MC problem (Eq. 2, relaxed in Section 1) with the
SVT algorithm of its reference [Cai08] and swaps the SVD for BLWS; it does not
restate the host.  The steps below are the published algorithms, written out
as mathematics.  The observed set Omega is given as COO index arrays.

``mc_svt_full`` -- SVT of [Cai08]:
    min tau ||X||_* + 0.5 ||X||_F^2  s.t.  P_Omega(X) = P_Omega(M)
    k0 = ceil(tau / (delta ||P_Omega M||_2));  Y^0 = k0 delta P_Omega(M)
    repeat k = 1, 2, ...:
        X^k = T_tau(Y^{k-1})                                 (Eq. 3-4)
        stop if ||P_Omega(X^k - M)||_F / ||P_Omega M||_F <= tol
        Y^k = Y^{k-1} + delta P_Omega(M - X^k)
    defaults of [Cai08]: tau = 5 sqrt(m n), delta = 1.2 m n / |Omega|.
    W = Y is supported on Omega, so its SVT input is purely sparse.

``mc_prox_full`` -- the proximal-gradient (fixed-point) form of the same
nuclear-norm program, FPC of [Ma09] (cited in Section 1 and Section 4.2):
    W_k = X_k + delta P_Omega(M - X_k)        (low-rank X_k + sparse residual)
    X_{k+1} = T_tau(W_k)
    with delta = 1 and continuation on the threshold: tau starts at
    eta ||P_Omega M||_2 (eta = 1/4) and drops to max(eta tau, tau_min) each
    time the iterate settles (relative change below xtol), as in FPC; same
    stopping rule on the observed residual.
"""
import math

import numpy as np

from .svt import svt_factored


def _observed(m, n, rows, cols, vals):
    Mo = np.zeros((m, n))
    Mo[np.asarray(rows), np.asarray(cols)] = np.asarray(vals, dtype=np.float64)
    mask = np.zeros((m, n), dtype=bool)
    mask[np.asarray(rows), np.asarray(cols)] = True
    return Mo, mask


def mc_svt_full(m, n, rows, cols, vals, tau=None, delta=None, tol=1e-4,
                max_iter=500):
    """SVT matrix completion [Cai08] with full-SVD SVT.  Returns a dict."""
    Mo, mask = _observed(m, n, rows, cols, vals)
    s = int(mask.sum())
    if tau is None:
        tau = 5.0 * math.sqrt(m * n)
    if delta is None:
        delta = 1.2 * m * n / s
    norm_pm = float(np.linalg.norm(Mo, "fro"))
    norm2 = float(np.linalg.svd(Mo, compute_uv=False)[0])
    k0 = math.ceil(tau / (delta * norm2))
    Y = k0 * delta * Mo
    hist = []
    U = th = V = None
    r = 0
    it = 0
    for it in range(1, max_iter + 1):
        U, th, V, r = svt_factored(Y, tau)
        X = (U * th) @ V.T
        resid = np.where(mask, X - Mo, 0.0)
        res = float(np.linalg.norm(resid, "fro")) / norm_pm
        hist.append((res, r))
        if res <= tol:
            break
        Y = Y - delta * resid
    return {"U": U, "th": th, "V": V, "rank": r, "iters": it, "residual": res,
            "history": hist, "tau": tau, "delta": delta, "k0": k0}


def mc_prox_full(m, n, rows, cols, vals, eta=0.25, tau_min_rel=1e-4, xtol=1e-3,
                 delta=1.0, tol=1e-4, max_iter=1000):
    """Proximal (FPC-type) matrix completion with threshold continuation.

    Each step forms W_k = X_k + delta P_Omega(M - X_k) and X_{k+1} =
    T_tau(W_k).  tau starts at eta ||P_Omega M||_2 and is lowered to
    max(eta tau, tau_min) once the iterate settles, i.e. once
    ||X_{k+1} - X_k||_F / max(1, ||X_k||_F) < xtol.
    """
    Mo, mask = _observed(m, n, rows, cols, vals)
    norm_pm = float(np.linalg.norm(Mo, "fro"))
    norm2 = float(np.linalg.svd(Mo, compute_uv=False)[0])
    tau_min = tau_min_rel * norm2
    tau = eta * norm2
    X = np.zeros((m, n))
    hist = []
    U = th = V = None
    r = 0
    it = 0
    res = 1.0
    for it in range(1, max_iter + 1):
        W = X + delta * np.where(mask, Mo - X, 0.0)
        U, th, V, r = svt_factored(W, tau)
        Xn = (U * th) @ V.T
        dx = float(np.linalg.norm(Xn - X, "fro")) / max(1.0, float(np.linalg.norm(X, "fro")))
        X = Xn
        res = float(np.linalg.norm(np.where(mask, X - Mo, 0.0), "fro")) / norm_pm
        hist.append((res, r, tau))
        if res <= tol:
            break
        if dx < xtol and tau > tau_min:
            tau = max(eta * tau, tau_min)
    return {"U": U, "th": th, "V": V, "rank": r, "iters": it, "residual": res,
            "history": hist, "tau_min": tau_min, "tau": tau}
