"""The seeded input generators: exact sizes, structure and determinism (they
feed both the oracle and the CUDA path, so a slip here would hide in both)."""
import numpy as np

from paper_1012_0365_gb300 import synthetic as syn


def test_rpca_problem_structure():
    D, L0, S0 = syn.rpca_problem(60, 45, 4, 0.1, amp=50.0, seed=3)
    assert D.shape == L0.shape == S0.shape == (60, 45)
    np.testing.assert_array_equal(D, L0 + S0)
    assert np.linalg.matrix_rank(L0) == 4
    assert np.count_nonzero(S0) == round(0.1 * 60 * 45)
    assert np.abs(S0).max() <= 50.0
    D2, _, _ = syn.rpca_problem(60, 45, 4, 0.1, amp=50.0, seed=3)
    np.testing.assert_array_equal(D, D2)


def test_mc_problem_is_a_sorted_csr_of_the_planted_matrix():
    P = syn.mc_problem(30, 40, 3, 0.2, seed=5)
    rows, cols, vals, rowptr = P["rows"], P["cols"], P["vals"], P["rowptr"]
    assert rows.dtype == cols.dtype == rowptr.dtype == np.int32
    assert P["nnz"] == len(vals) == round(0.2 * 30 * 40)
    key = rows.astype(np.int64) * 40 + cols
    assert np.all(np.diff(key) > 0)                   # sorted by (row, col), no repeats
    assert rowptr[0] == 0 and rowptr[-1] == P["nnz"]
    for i in range(30):
        assert np.all(rows[rowptr[i]:rowptr[i + 1]] == i)
    M = P["ML"] @ P["MR"].T
    np.testing.assert_allclose(vals, M[rows, cols], rtol=0, atol=1e-13 * np.abs(M).max())


def test_symmetric_problem():
    W, npos = syn.symmetric_problem(50, 6, seed=2)
    np.testing.assert_array_equal(W, W.T)
    assert npos == 4                                  # every third of 6 is negative
    lam = np.sort(np.linalg.eigvalsh(W))[::-1]
    assert lam[npos - 1] > 5 * abs(lam[npos])         # the positive signal stands above the rest


def test_batch_and_serving_specs():
    specs = syn.batched_rpca_specs(20, seed=1)
    assert len(specs) == 20
    for sp in specs:
        assert 100 <= sp["m"] <= 1000 and 100 <= sp["n"] <= 1000
        assert sp["rank"] == max(1, int(round(0.05 * min(sp["m"], sp["n"]))))
        assert 0.05 <= sp["frac"] <= 0.10
    for sp in syn.serving_specs(40, seed=2):
        if sp["kind"] == "mc":
            r, m, n = sp["rank"], sp["m"], sp["n"]
            assert r == 1 or sp["frac"] * m * n >= 4 * r * (m + n - r)
        else:
            assert sp["rank"] <= max(1, min(sp["m"], sp["n"]) // 20)


def test_orthonormal_is_orthonormal():
    Q = syn.orthonormal(30, 7, seed=4)
    np.testing.assert_allclose(Q.T @ Q, np.eye(7), atol=1e-13)
