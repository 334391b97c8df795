"""CUDA graphs of the RPCA solver's outer-iteration phases (blws_config.graphs).

A replayed graph launches the kernels it captured, with the arguments it
captured; the per-iteration scalars (mu, eps) come from device memory.  So a
solve with graphs must give bit-identical A and E to the same solve launched
kernel by kernel, in every precision mode, and over repeated solves that
replay graphs captured by an earlier one.  Agreement with the FP64 oracle is
checked too, on the graph path itself.
"""
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


def ctx_pair(precision):
    from paper_1012_0365_gb300 import blws
    return blws.Context(precision=precision, graphs=1), blws.Context(precision=precision, graphs=0)


def run(ctx, torch, D, **kw):
    from paper_1012_0365_gb300 import blws
    A, E, info = ctx.rpca_solve(blws.colmajor(torch.from_numpy(D)), **kw)
    torch.cuda.synchronize()
    return A.cpu().numpy(), E.cpu().numpy(), info


@pytest.mark.parametrize("precision,m,n,rank,frac,seed", [
    (0, 300, 300, 15, 0.05, 0),    # FP64
    (0, 173, 251, 9, 0.08, 1),     # ragged
    (2, 900, 900, 66, 0.05, 2),    # FP64-equivalent, A as a digit-plane product (rank >= 64)
    (2, 257, 129, 8, 0.06, 3),
    (1, 300, 260, 12, 0.05, 4),    # mixed, with its digit-plane refinement tail
])
def test_graphs_bit_identical_to_direct_launches(torch_mod, precision, m, n, rank, frac, seed):
    g, d = ctx_pair(precision)
    D = syn.rpca_problem(m, n, rank, frac, amp=50.0, seed=seed)[0]
    Ag, Eg, ig = run(g, torch_mod, D, tol=1e-9)
    Ad, Ed, idd = run(d, torch_mod, D, tol=1e-9)
    assert ig["status"] == 0 and idd["status"] == 0
    assert (ig["iters"], ig["rank"], ig["nnzE"]) == (idd["iters"], idd["rank"], idd["nnzE"])
    assert np.array_equal(Ag, Ad)
    assert np.array_equal(Eg, Ed)
    caps, reps = g.graph_stats()
    assert caps > 0 and reps > 0, (caps, reps)
    assert d.graph_stats() == (0, 0)
    # a second solve on the same buffers replays graphs captured by the first
    Ag2, Eg2, ig2 = run(g, torch_mod, D, tol=1e-9)
    caps2, reps2 = g.graph_stats()
    assert reps2 - reps > ig2["iters"], (reps, reps2, ig2["iters"])
    assert np.array_equal(Ag2, Ag) and np.array_equal(Eg2, Eg)


def test_graph_path_matches_oracle(torch_mod):
    from paper_1012_0365_gb300 import blws
    ctx = blws.Context(graphs=1)
    D = syn.rpca_problem(220, 180, 9, 0.05, amp=50.0, seed=7)[0]
    run(ctx, torch_mod, D, tol=1e-10)  # captures
    A, E, info = run(ctx, torch_mod, D, tol=1e-10)  # replays from the first iteration on
    ref = oracle.rpca_ialm_full(D, tol=1e-10)
    assert info["status"] == 0
    assert np.linalg.norm(A - ref["A"]) / np.linalg.norm(ref["A"]) < 1e-6
    assert np.linalg.norm(E - ref["E"]) / np.linalg.norm(ref["E"]) < 1e-6


def test_graph_timing_records_match_direct(torch_mod):
    """Products timed inside replayed graphs are read back after each replay:
    the same number of timed products, with the same work, as direct launches."""
    g, d = ctx_pair(2)
    D = syn.rpca_problem(300, 300, 15, 0.05, amp=50.0, seed=5)[0]
    out = []
    for c in (g, d):
        run(c, torch_mod, D, tol=1e-9)  # warm (captures on the graph context)
        c.timing_start()
        run(c, torch_mod, D, tol=1e-9)
        ms, n, work = c.timing_stop()
        recs = c.timing_records()
        assert n == len(recs) and n > 0 and ms > 0.0
        out.append(sorted((w, kd) for _, w, kd in recs))
    assert out[0] == out[1]
    assert g.graph_stats()[1] > 0


def test_graphs_off_by_environment(torch_mod, monkeypatch):
    from paper_1012_0365_gb300 import blws
    monkeypatch.setenv("BLWS_GRAPH", "0")
    ctx = blws.Context(graphs=1)
    D = syn.rpca_problem(120, 100, 5, 0.05, amp=50.0, seed=8)[0]
    run(ctx, torch_mod, D, tol=1e-8)
    run(ctx, torch_mod, D, tol=1e-8)
    assert ctx.graph_stats() == (0, 0)


@pytest.mark.parametrize("variant,m,n,r,sdr,seed,kw", [
    (0, 300, 300, 10, 6, 0, {"tol": 1e-6}),
    (0, 257, 190, 5, 5, 1, {"tol": 1e-6}),
    (1, 120, 120, 4, 6, 3, {"tol": 1e-3, "max_rank": 120}),  # continuation: tau moves
])
def test_mc_graphs_bit_identical_to_direct_launches(torch_mod, variant, m, n, r, sdr, seed, kw):
    """The matrix-completion solver's three phases (block steps; Ritz lift and
    count; thresholds and SDDMM) replayed as graphs: the same factors as with
    direct launches, for the SVT host and the proximal form (whose tau moves)."""
    from paper_1012_0365_gb300 import blws
    P = syn.mc_problem(m, n, r, sdr * r * (m + n - r) / (m * n), seed=seed)
    out = []
    for graphs in (1, 0):
        ctx = blws.Context(graphs=graphs)
        U, th, V, info = ctx.mc_solve(m, n, torch_mod.from_numpy(P["rowptr"]).cuda(),
                                      torch_mod.from_numpy(P["cols"]).cuda(),
                                      torch_mod.from_numpy(P["vals"]).cuda(),
                                      max_rank=kw.get("max_rank", 60), variant=variant, tol=kw["tol"],
                                      max_iter=3000, allow_noconv=True)
        torch_mod.cuda.synchronize()
        out.append((U.cpu().numpy(), th.cpu().numpy(), V.cpu().numpy(), info, ctx.graph_stats()))
    (Ug, tg, Vg, ig, sg), (Ud, td, Vd, idd, sd) = out
    assert (ig["status"], ig["iters"], ig["rank"]) == (idd["status"], idd["iters"], idd["rank"])
    assert ig["iters"] > 10
    assert np.array_equal(Ug, Ud) and np.array_equal(tg, td) and np.array_equal(Vg, Vd)
    assert sg[1] > 0 and sd == (0, 0)


def test_guard_off_threshold_is_bit_identical_and_forced_restarts_match_oracle(torch_mod):
    """The Ritz-residual guard only adds work on dead buffers until it fires:
    with a threshold no pair reaches, a solve is bit-identical to one without
    it; with a threshold every pair exceeds, each call runs again with up to
    two more blocks, and the solve still reaches the oracle's optimum."""
    from paper_1012_0365_gb300 import blws
    D = syn.rpca_problem(220, 180, 9, 0.05, amp=50.0, seed=7)[0]
    A0, E0, i0 = run(blws.Context(), torch_mod, D, tol=1e-10)
    A1, E1, i1 = run(blws.Context(guard=1e6), torch_mod, D, tol=1e-10)
    assert i1["restarts"] == 0 and i0["restarts"] == 0
    assert np.array_equal(A0, A1) and np.array_equal(E0, E1)
    A2, E2, i2 = run(blws.Context(guard=1e-300), torch_mod, D, tol=1e-10)
    assert i2["restarts"] >= i2["iters"]
    ref = oracle.rpca_ialm_full(D, tol=1e-10)
    assert np.linalg.norm(A2 - ref["A"]) / np.linalg.norm(ref["A"]) < 1e-6
    assert np.linalg.norm(E2 - ref["E"]) / np.linalg.norm(ref["E"]) < 1e-6
