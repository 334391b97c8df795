"""The product autotuner (blws_config.tune): tile shapes and K splits timed per
size bucket, kept process-wide and in the file BLWS_TUNE_FILE names.

A tuned product differs from the fixed rule's only in how its split-K sums
are grouped, so a tuned solve agrees with the FP64 oracle at the same bar,
and with graphs on and off it stays bit-identical (both read the same
process-wide choices)."""
import numpy as np
import pytest

import oracle
from paper_1012_0365_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def run(ctx, torch, D, **kw):
    from paper_1012_0365_gb300 import blws
    A, E, info = ctx.rpca_solve(blws.colmajor(torch.from_numpy(D)), **kw)
    torch.cuda.synchronize()
    return A.cpu().numpy(), E.cpu().numpy(), info


def test_tuned_solve_matches_oracle_and_is_recorded(torch_mod, tmp_path, monkeypatch):
    from paper_1012_0365_gb300 import blws
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("BLWS_TUNE_FILE", str(path))
    before = blws.Context.tune_count()
    ctx = blws.Context(tune=1)
    D = syn.rpca_problem(260, 230, 12, 0.05, amp=50.0, seed=11)[0]
    A, E, info = run(ctx, torch_mod, D, tol=1e-10)
    ref = oracle.rpca_ialm_full(D, tol=1e-10)
    assert info["status"] == 0
    assert np.linalg.norm(A - ref["A"]) / np.linalg.norm(ref["A"]) < 1e-6
    assert np.linalg.norm(E - ref["E"]) / np.linalg.norm(ref["E"]) < 1e-6
    after = blws.Context.tune_count()
    assert after > before
    if before == 0:  # this process read the file first: every choice went to it
        lines = [l for l in path.read_text().splitlines() if l.startswith("tune ")]
        assert len(lines) == after
        for l in lines:
            f = [int(x) for x in l.split()[1:]]
            assert len(f) == 10
            if f[1] == 100:  # digit-plane product: its K split count
                assert f[8] >= 1 and f[9] == 0
            else:  # CUDA-core product: tile shape and split target
                assert 0 <= f[8] < 5 and 0 <= f[9] <= 3


def test_tuned_graphs_bit_identical(torch_mod):
    from paper_1012_0365_gb300 import blws
    D = syn.rpca_problem(310, 280, 14, 0.06, amp=50.0, seed=12)[0]
    g = blws.Context(tune=1, graphs=1)
    d = blws.Context(tune=1, graphs=0)
    Ad, Ed, idd = run(d, torch_mod, D, tol=1e-9)  # tunes the buckets it meets
    Ag, Eg, ig = run(g, torch_mod, D, tol=1e-9)
    Ag2, Eg2, _ = run(g, torch_mod, D, tol=1e-9)  # replays
    assert idd["status"] == 0 and ig["status"] == 0
    assert np.array_equal(Ag, Ad) and np.array_equal(Eg, Ed)
    assert np.array_equal(Ag2, Ad) and np.array_equal(Eg2, Ed)
    assert g.graph_stats()[1] > 0
