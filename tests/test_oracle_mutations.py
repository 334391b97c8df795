"""Planted mistakes: each test breaks one step of the oracle in a plausible way
(on the CPU, through monkeypatching) and checks that a pin catches it."""
import numpy as np

import oracle
import oracle.blws as ob
from paper_1012_0365_gb300 import synthetic as syn


def _whole_space_error():
    W = syn.gaussian_block(5, 4, seed=30)
    out = oracle.blws_svt_ref(W, 0.7, syn.gaussian_block(5, 3, seed=31),
                              syn.gaussian_block(4, 3, seed=32), k=3, r=4)
    A, _ = oracle.svt_full(W, 0.7)
    return np.abs(out["A"] - A).max()


def test_pins_catch_transposed_offdiagonal_block(monkeypatch):
    orig = ob.assemble_T
    monkeypatch.setattr(ob, "assemble_T", lambda Ms, Bs: orig(Ms, [B.T for B in Bs]))
    assert _whole_space_error() > 1e-6


def test_pins_catch_dropped_three_term(monkeypatch):
    # drop X_{l-1} B_{l-1}^T and its re-projection: R_l keeps a component
    # along X_{l-1}
    def bad_block_lanczos(apply, X1, k, full_reorth=False):
        Xs, Ms, Bs = [X1], [], []
        P = apply(X1)
        scale = float(np.max(np.linalg.norm(P, axis=0)))
        Ms.append(ob._sym(X1.T @ P))
        for l in range(k - 1):
            R = P - Xs[l] @ Ms[l]
            Xn, Bn = ob.qr_deflate(R, scale)
            Xs.append(Xn)
            Bs.append(Bn)
            P = apply(Xn)
            Ms.append(ob._sym(Xn.T @ P))
        return Xs, Ms, Bs, P
    monkeypatch.setattr(ob, "block_lanczos", bad_block_lanczos)
    assert _whole_space_error() > 1e-6


def test_pins_catch_missing_sqrt2(monkeypatch):
    orig = ob._svt_from_ritz
    monkeypatch.setattr(ob, "_svt_from_ritz", lambda Y, lam, eps, m: orig(Y / np.sqrt(2), lam, eps, m))
    assert _whole_space_error() > 1e-6


def test_pins_catch_wrong_shrink_sign(monkeypatch):
    # E-shrink with the wrong sign convention breaks planted recovery
    import oracle.rpca as orp
    monkeypatch.setattr(orp, "theta", lambda x, e: np.sign(x) * np.maximum(np.abs(x) + e, 0))
    D, L0, S0 = syn.rpca_problem(60, 60, 3, 0.05, seed=1)
    out = orp.rpca_ialm_full(D, tol=1e-8, max_iter=200)
    assert np.linalg.norm(out["A"] - L0) / np.linalg.norm(L0) > 1e-3


def _evd_whole_space_error():
    lam = [9.0, 7.0, 4.0, 1.0, -0.5, -3.0, -12.0, 0.25]
    Q = syn.orthonormal(8, 8, seed=33)
    W = (Q * np.asarray(lam)) @ Q.T
    out = oracle.blws_evd_ref(W, 2.0, None, 2, 3, syn.gaussian_block(8, 4, seed=34))
    return np.abs(out["lam"] - np.array([9.0, 7.0, 4.0])).max()


def test_pins_catch_magnitude_ordering_in_bl_evd(monkeypatch):
    # Algorithm 3 orders the eigenvalues of T_k algebraically; ordering by
    # magnitude would put -12 first on an indefinite W
    def bad_bl_evd(apply, X1, k, r, full_reorth=False):
        Xs, Ms, Bs, _ = ob.block_lanczos(apply, X1, k, full_reorth)
        lam, Z = np.linalg.eigh(ob.assemble_T(Ms, Bs))
        order = np.argsort(-np.abs(lam), kind="stable")
        return np.hstack(Xs) @ Z[:, order][:, :r], lam[order][:r]
    assert _evd_whole_space_error() < 1e-12
    monkeypatch.setattr(ob, "bl_evd", bad_bl_evd)
    assert _evd_whole_space_error() > 1e-6


def test_pins_catch_a_start_block_without_the_warm_columns(monkeypatch):
    # BLWS's start block is the previous subspace: dropping it (random start
    # only) loses the exactness of an invariant warm start at k = 1
    lam = np.array([10.0, 6.0, 3.0, -1.0, -2.0, 0.5, 1.5, -8.0, 2.0, 0.0])
    Q = syn.orthonormal(10, 10, seed=35)
    W = (Q * lam) @ Q.T
    ok = oracle.blws_evd_ref(W, 0.0, Q[:, :3], 1, 3)
    assert np.abs(ok["lam"] - lam[:3]).max() < 1e-12
    orig = ob.blws_evd_ref

    def no_warm(W, eps, U0, k, r, G=None):
        return orig(W, eps, None, k, r, syn.gaussian_block(W.shape[0], r, seed=36))
    monkeypatch.setattr(oracle, "blws_evd_ref", no_warm)
    bad = oracle.blws_evd_ref(W, 0.0, Q[:, :3], 1, 3)
    assert np.abs(bad["lam"] - lam[:3]).max() > 1e-3
