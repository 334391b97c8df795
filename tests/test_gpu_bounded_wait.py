"""The bounded device waits of the tensor-core kernels, end to end.

Every wait of a producer/consumer tensor-core kernel is capped; a wait that
runs out raises the context's error word, the kernel returns, and the calls
that synchronise report BLWS_ETIMEOUT.  blws_wait_probe runs a small kernel
that waits, through the same bounded wait, on a barrier nothing arrives at,
with a cap of a few hundred polls: no copy, MMA or tensor memory is in flight,
so the context stays usable, which the test checks by solving afterwards.
"""
import numpy as np
import pytest

from paper_1012_0365_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def blws_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1012_0365_gb300 import blws
    return torch, blws


def test_wait_that_runs_out_returns_etimeout(blws_mod):
    torch, blws = blws_mod
    ctx = blws.Context(precision=blws.PREC_FP64_TC)
    assert ctx.wait_probe(polls=256) == blws.ETIMEOUT
    assert "gave up" in blws.load().blws_last_error(ctx._h).decode()
    assert ctx.wait_probe(polls=0) == blws.EINVAL
    # the flag does not leak into the next call: a solve on the same context
    # (tensor-core products, whose entry point clears the flag) succeeds
    D, L0, _ = syn.rpca_problem(120, 100, 4, 0.05, seed=3)
    A, E, info = ctx.rpca_solve(blws.colmajor(torch.from_numpy(D)), tol=1e-9)
    assert info["status"] == blws.OK
    assert np.linalg.norm(A.cpu().numpy() - L0) / np.linalg.norm(L0) < 1e-6
