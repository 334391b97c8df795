"""bench.py's multi-rank arithmetic on CPU: two gloo ranks, each timing its own
replica, report the slowest rank's time and the whole job's throughput (the
units all ranks processed over that time)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [1000.0, 1500.0][rank]          # rank 1 is the slower replica
        worst = bench.max_over_ranks(dist, local_ms, "cpu")
        rate = bench.job_rate(world, 3, worst)      # 3 steps per rank
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            f.write("%r %r" % (worst, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        worst, rate = map(float, (tmp_path / ("rank%d.txt" % rank)).read_text().split())
        assert worst == 1500.0                       # every rank sees the slowest time
        assert rate == pytest.approx(2 * 3 / 1.5)    # 6 solves over 1.5 s


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 12.5, "cpu") == 12.5
    assert bench.job_rate(1, 5, 2000.0) == pytest.approx(2.5)
