"""The multi-GPU form is replicas only (no collective on the data path):
the host logic that joins them -- the slowest replica's step time and the
whole-job rate -- on two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    # rank r took (1 + r) ms, (2 + 3r) ms and 5 ms for its three timings
    t = bench.max_over_ranks([1.0 + rank, 2.0 + 3.0 * rank, 5.0])
    out.put((rank, t, bench.job_rate(1000, world, t[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == [2.0, 5.0, 5.0]          # the slowest replica, per timing
        assert rate == pytest.approx(1000 * 2 / 2e-3)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.job_rate(10, 1, 2.0) == pytest.approx(5000.0)
