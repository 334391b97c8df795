"""Seeded synthetic workloads shaped like the paper's experiments (Section 5).

Input code only: this module draws data and holds none of the method's
arithmetic.  Both the CUDA path's tests/bench and the oracle's tests take their
inputs from here; nothing here calls either of them.

Recipes (NumPy PCG64, one seed per instance):
  * RPCA (Section 5, Table 1 pattern): L0 = X Y^T with X (m x r), Y (n x r)
    i.i.d. N(0, 1) -- an instance of the independent random orthogonal model,
    since Gaussian factors have Haar-distributed singular vectors; S0 has
    round(frac * m * n) entries at positions drawn without replacement, values
    uniform in [-amp, amp]; D = L0 + S0.
  * BL_EVD of a symmetric matrix (Section 4): see symmetric_problem.
  * MC (Section 5, Table 2 pattern): M = M_L M_R^T with i.i.d. N(0, 1) factors;
    Omega = round(frac * m * n) positions drawn uniformly without replacement,
    returned sorted by (row, col) with CSR row pointers (int32).
"""
import math

import numpy as np


def rpca_problem(m, n, rank, frac, amp=50.0, seed=0):
    """Return (D, L0, S0) as float64 arrays of shape (m, n)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, rank))
    Y = rng.standard_normal((n, rank))
    L0 = X @ Y.T
    nnz = int(round(frac * m * n))
    pos = rng.choice(m * n, size=nnz, replace=False)
    S0 = np.zeros(m * n)
    S0[pos] = rng.uniform(-amp, amp, size=nnz)
    S0 = S0.reshape(m, n)
    return L0 + S0, L0, S0


def mc_problem(m, n, rank, frac, seed=0):
    """Return a dict: rows, cols (int32, sorted by row then col), vals (float64),
    rowptr (int32, m + 1), the factors ML, MR, and nnz."""
    rng = np.random.default_rng(seed)
    ML = rng.standard_normal((m, rank))
    MR = rng.standard_normal((n, rank))
    nnz = int(round(frac * m * n))
    pos = np.sort(rng.choice(m * n, size=nnz, replace=False))
    rows = (pos // n).astype(np.int32)
    cols = (pos % n).astype(np.int32)
    vals = np.einsum("ij,ij->i", ML[rows], MR[cols])
    rowptr = np.zeros(m + 1, dtype=np.int32)
    np.cumsum(np.bincount(rows, minlength=m), out=rowptr[1:])
    return {"rows": rows, "cols": cols, "vals": vals, "rowptr": rowptr,
            "ML": ML, "MR": MR, "nnz": nnz, "m": m, "n": n}


def symmetric_problem(m, rank, noise=0.05, seed=0):
    """A symmetric indefinite m x m matrix for BL_EVD: W = X diag(d) X^T / m
    plus noise * sqrt(m) * (E + E^T) / 2, with X (m x rank) and E i.i.d.
    N(0, 1) and |d_i| ~ U[m, 2m], every third d_i negative.  Returns (W, npos)
    with npos the number of positive d_i (the eigenvalues that stand above
    the noise edge)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, rank))
    d = np.where(np.arange(rank) % 3 == 2, -1.0, 1.0) * rng.uniform(1.0, 2.0, rank) * m
    E = rng.standard_normal((m, m))
    W = (X * d) @ X.T / m + noise * math.sqrt(m) * (E + E.T) / 2
    W = (W + W.T) / 2  # exactly symmetric (the product above is only to rounding)
    return W, int(np.count_nonzero(d > 0))


def gaussian_block(rows, cols, seed=0):
    """i.i.d. N(0, 1) block (e.g. extra start columns for a block Lanczos)."""
    return np.random.default_rng(seed).standard_normal((rows, cols))


def orthonormal(rows, cols, seed=0):
    """Haar-random orthonormal columns, via the sign-fixed QR of a Gaussian."""
    G = gaussian_block(rows, cols, seed)
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))


def batched_rpca_specs(count, lo=100, hi=1000, seed=0):
    """Sizes for a batch of uneven RPCA instances: m, n ~ U{lo..hi},
    rank = round(5% of min(m, n)), corruption fraction ~ U[0.05, 0.10]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.integers(lo, hi + 1))
        n = int(rng.integers(lo, hi + 1))
        rank = max(1, int(round(0.05 * min(m, n))))
        frac = float(rng.uniform(0.05, 0.10))
        out.append({"m": m, "n": n, "rank": rank, "frac": frac, "seed": seed * 100003 + i})
    return out


def lam_default(m, n):
    """lambda = 1/sqrt(max(m, n)) (Section 5 uses 1/sqrt(m) for m x m data)."""
    return 1.0 / math.sqrt(max(m, n))


def serving_specs(count, seed=0):
    """A stream of mixed requests: 70% Robust PCA with m, n ~ U{200..4000},
    30% matrix completion with m, n ~ U{1000..8000} and 5-20% of the entries
    observed; ranks ~ U{5..100}, an MC rank clamped so that the samples per
    degree of freedom s / (r (m + n - r)) stay >= 4 (below that the SVT
    iteration of [Cai08] did not reach tol 1e-4 within 500 iterations)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        r = int(rng.integers(5, 101))
        if rng.uniform() < 0.7:
            m, n = int(rng.integers(200, 4001)), int(rng.integers(200, 4001))
            r = min(r, max(1, min(m, n) // 20))
            out.append({"kind": "rpca", "m": m, "n": n, "rank": r, "frac": 0.1, "seed": seed * 7919 + i})
        else:
            m, n = int(rng.integers(1000, 8001)), int(rng.integers(1000, 8001))
            frac = float(rng.uniform(0.05, 0.20))
            while r > 1 and frac * m * n < 4 * r * (m + n - r):
                r -= 1
            out.append({"kind": "mc", "m": m, "n": n, "rank": r, "frac": frac, "seed": seed * 7919 + i})
    return out
