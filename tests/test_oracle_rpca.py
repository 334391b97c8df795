"""Pins for the oracle's inexact-ALM RPCA: exact recovery of planted data
(Section 1), the KKT certificate of the convex program, D = A + E at
convergence, BLWS-ADM agreeing with full-SVD ADM, and Table 1's pattern."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1012_0365_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def kkt_residuals(D, A, E, Y, lam):
    """Optimality of min ||A||_* + lam ||E||_1 s.t. D = A + E, certified by Y:
    Y in d||A||_*  (U^T Y V = I, ||(I-UU^T) Y (I-VV^T)||_2 <= 1) and
    Y in lam d||E||_1 (Y = lam sgn(E) on supp E, |Y| <= lam elsewhere)."""
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    r = int(np.sum(s > 1e-8 * s[0]))
    U, V = U[:, :r], Vt[:r].T
    on = np.linalg.norm(U.T @ Y @ V - np.eye(r))
    Pu = np.eye(A.shape[0]) - U @ U.T
    Pv = np.eye(A.shape[1]) - V @ V.T
    perp = np.linalg.norm(Pu @ Y @ Pv, 2)
    supp = E != 0
    sgn = np.max(np.abs(Y[supp] - lam * np.sign(E[supp]))) / lam
    box = np.max(np.abs(Y[~supp])) / lam
    feas = np.linalg.norm(D - A - E) / np.linalg.norm(D)
    return {"rank": r, "on": on, "perp": perp, "sgn": sgn, "box": box, "feas": feas}


@pytest.fixture(scope="module")
def c1():
    D, L0, S0 = syn.rpca_problem(200, 200, 10, 0.05, amp=50.0, seed=0)
    return D, L0, S0, oracle.rpca_ialm_full(D, tol=1e-10)


def test_planted_recovery_c1(c1):
    D, L0, S0, out = c1
    assert np.linalg.norm(out["A"] - L0) / np.linalg.norm(L0) < 1e-6
    assert np.linalg.norm(out["E"] - S0) / np.linalg.norm(S0) < 1e-6
    assert out["rank"] == 10
    assert abs(out["nnzE"] - 2000) <= 20


def test_kkt_certificate_c1(c1):
    D, L0, S0, out = c1
    k = kkt_residuals(D, out["A"], out["E"], out["Y"], out["lam"])
    assert k["rank"] == 10
    assert k["on"] < 1e-6
    assert k["perp"] <= 1 + 1e-6
    # the dual iterate carries the last mu*Z update, so it is ~mu_bar*tol off
    assert k["sgn"] < 1e-3
    assert k["box"] <= 1 + 1e-6
    assert k["feas"] < 1e-10


def test_blws_adm_reaches_the_same_optimum(c1):
    D, L0, S0, ref = c1
    rng = np.random.default_rng(123)
    out = oracle.rpca_ialm_blws(D, lambda r, c: rng.standard_normal((r, c)), tol=1e-10)
    assert np.linalg.norm(out["A"] - ref["A"]) / np.linalg.norm(ref["A"]) < 1e-8
    assert np.linalg.norm(out["E"] - ref["E"]) / np.linalg.norm(ref["E"]) < 1e-8
    assert abs(out["iters"] - ref["iters"]) <= 3


def test_rank_prediction_rule():
    # [Lin09]: grow by one past the count, or by 5% of n when all were kept.
    assert oracle.rank_predict(10, 6, 200) == 7
    assert oracle.rank_predict(10, 10, 200) == 20
    assert oracle.rank_predict(10, 10, 2000) == 110
    assert oracle.rank_predict(199, 199, 200) == 200


def test_table1_pattern_m500():
    # Table 1, m = 500 rows: rank(A^) = 50, ||E^||_0 ~ 25000, ~30 iterations,
    # relative error vs truth a few 1e-6, at the host's default tol 1e-7.
    rows = json.load(open(os.path.join(GOLDEN, "table1_rpca.json")))["rows"]
    ref = [r for r in rows if r["m"] == 500]
    D, L0, S0 = syn.rpca_problem(500, 500, 50, 0.10, amp=500.0, seed=7)
    out = oracle.rpca_ialm_full(D, lam=1 / math.sqrt(500), tol=1e-7)
    rel = np.linalg.norm(out["A"] - L0) / np.linalg.norm(L0)
    assert out["rank"] == ref[0]["rank"]
    assert abs(out["nnzE"] - 25000) < 0.01 * 25000
    assert min(r["iters"] for r in ref) - 6 <= out["iters"] <= max(r["iters"] for r in ref) + 10
    assert rel < 5 * max(r["relerr"] for r in ref)
