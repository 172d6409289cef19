"""The multi-rank host path of bench.py on CPU ranks (gloo, world size 2): every rank times the
same steps, the job's time is the slowest rank's, and the reported throughput is the rays all
ranks processed over that time.  Replicas only: the render path has no collective."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms_by_rank, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(ms_by_rank[rank], world)
        out[rank] = (ms, bench.job_mrays_s(1_000_000, ms, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ms_by_rank", [(12.5, 10.0), (7.0, 9.25)])
def test_slowest_rank_sets_the_job_time(ms_by_rank):
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, ms_by_rank, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        slow = max(ms_by_rank)
        for r in range(world):
            ms, value = out[r]
            assert ms == slow
            assert value == pytest.approx(2 * 1_000_000 / slow / 1e3)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_mrays_s(2_000_000, 4.0, 1) == pytest.approx(500.0)  # 2M rays in 4 ms
