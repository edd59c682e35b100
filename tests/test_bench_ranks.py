"""The benchmark's multi-rank aggregation on two CPU ranks (gloo): every rank
times its own independent problem; the reported time is the slowest rank's
and the rate counts the work of all ranks (weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [3.0, 5.0][rank]                     # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, world, "cpu")
    rate = bench.whole_job_rate(world, 1000.0, ms * 1e-3)
    out.put((rank, ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_slowest_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in res:
        assert ms == pytest.approx(5.0)
        assert rate == pytest.approx(2 * 1000.0 / 5e-3)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(4.0, 1, "cpu") == 4.0
    assert bench.whole_job_rate(1, 10.0, 2.0) == 5.0
