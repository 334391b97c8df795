"""Pins for the oracle's matrix-completion hosts: Table 2's pattern for SVT,
transpose equivariance, full observation (closed form), and one proximal step
with full observation equal to a plain SVT (Eq. 4)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1012_0365_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense(P):
    return P["ML"] @ P["MR"].T


@pytest.fixture(scope="module")
def small_mc():
    m, r, sdr = 300, 10, 6
    s = sdr * r * (2 * m - r)
    P = syn.mc_problem(m, m, r, s / (m * m), seed=0)
    return P, oracle.mc_svt_full(m, m, P["rows"], P["cols"], P["vals"])


def test_svt_table2_pattern(small_mc):
    # Table 2 (s/d_r = 6 rows): relative error 1.68e-4 .. 1.75e-4, 123-124
    # iterations, at tol 1e-4.  A smaller m keeps the same pattern.
    P, out = small_mc
    rows = [r for r in json.load(open(os.path.join(GOLDEN, "table2_mc.json")))["rows"]
            if r["s_over_dr"] == 6]
    M = _dense(P)
    X = (out["U"] * out["th"]) @ out["V"].T
    rel = np.linalg.norm(X - M) / np.linalg.norm(M)
    assert out["rank"] == 10
    assert rel < 3 * max(r["relerr"] for r in rows)
    assert out["residual"] <= 1e-4
    assert 60 <= out["iters"] <= 1.3 * max(r["iters"] for r in rows)


def test_svt_is_transpose_equivariant():
    # SVT on the transposed problem (rows and columns of Omega swapped, m and
    # n swapped) is the transposed iteration: the same singular values and
    # X' = X^T.  A non-square problem, so an m/n mix-up or a transposed
    # operand in the oracle shows.
    m, n, r = 240, 300, 6
    P = syn.mc_problem(m, n, r, 6 * r * (m + n - r) / (m * n), seed=4)
    a = oracle.mc_svt_full(m, n, P["rows"], P["cols"], P["vals"], max_iter=8)
    t = oracle.mc_svt_full(n, m, P["cols"], P["rows"], P["vals"], max_iter=8)
    assert a["iters"] == t["iters"] and a["rank"] == t["rank"]
    np.testing.assert_allclose(t["th"], a["th"], rtol=1e-10)
    Xa = (a["U"] * a["th"]) @ a["V"].T
    Xt = (t["U"] * t["th"]) @ t["V"].T
    assert Xa.shape == (m, n) and Xt.shape == (n, m)
    assert np.linalg.norm(Xt.T - Xa) <= 1e-10 * np.linalg.norm(Xa)


def test_svt_full_observation_recovers_m():
    # Omega = everything: the constraint fixes X = M.
    m = 40
    P = syn.mc_problem(m, m, 3, 1.0, seed=1)
    out = oracle.mc_svt_full(m, m, P["rows"], P["cols"], P["vals"], tol=1e-6, max_iter=2000)
    M = _dense(P)
    X = (out["U"] * out["th"]) @ out["V"].T
    assert np.linalg.norm(X - M) / np.linalg.norm(M) < 1e-5


def test_prox_full_observation_first_step_is_svt():
    # delta = 1 and Omega = everything: W_0 = M, so X_1 = T_tau0(M) (Eq. 4).
    m = 30
    P = syn.mc_problem(m, 25, 4, 1.0, seed=2)
    out = oracle.mc_prox_full(m, 25, P["rows"], P["cols"], P["vals"], max_iter=1)
    M = _dense(P)
    tau0 = 0.25 * np.linalg.svd(M, compute_uv=False)[0]
    A, c = oracle.svt_full(M, tau0)
    np.testing.assert_allclose((out["U"] * out["th"]) @ out["V"].T, A, atol=1e-10)
    assert out["rank"] == c


def test_prox_fixed_point_kkt():
    # At a fixed point of X = T_tau(X + P_Omega(M - X)) the iterate solves
    # min tau ||X||_* + 0.5 ||P_Omega(X - M)||_F^2: G = P_Omega(M - X) / tau
    # is a subgradient of ||X||_* (U^T G V = I, ||G||_2 <= 1).
    m, r = 80, 3
    s = 6 * r * (2 * m - r)
    P = syn.mc_problem(m, m, r, s / (m * m), seed=3)
    out = oracle.mc_prox_full(m, m, P["rows"], P["cols"], P["vals"], tau_min_rel=1e-2,
                              xtol=1e-6, tol=0.0, max_iter=3000)
    assert out["tau"] == out["tau_min"]
    X = (out["U"] * out["th"]) @ out["V"].T
    Mo = np.zeros((m, m))
    Mo[P["rows"], P["cols"]] = P["vals"]
    mask = Mo != 0
    G = np.where(mask, Mo - X, 0.0) / out["tau"]
    assert np.linalg.norm(out["U"].T @ G @ out["V"] - np.eye(out["rank"])) < 1e-4
    assert np.linalg.norm(G, 2) <= 1 + 1e-4
