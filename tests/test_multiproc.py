"""The N > 1 host logic of bench.py on CPU: two ranks over gloo.

Each GPU runs an independent replica of the step (the transform needs no data
exchange), so the only cross-rank logic is the timing: the job rate divides
the units all ranks processed by the slowest rank's time (a MAX all-reduce).
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, local_ms, out_q):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = bench.dist_env()
        rate, ms = bench.whole_job_rate(local_ms[rank], 1000, 10, w, "cpu")
        out_q.put((rank, r, w, loc, rate, ms))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_take_the_slowest_time():
    world = 2
    local_ms = [40.0, 25.0]      # rank 0 is the slow one
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, local_ms, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=90) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, r, w, loc, rate, ms in got:
        assert (r, w, loc) == (rank, world, rank)
        assert ms == max(local_ms)
        # 2 ranks x 1000 units x 10 steps in 40 ms
        assert rate == pytest.approx(world * 1000 * 10 / 0.040)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    rate, ms = bench.whole_job_rate(12.5, 100, 4, 1)
    assert ms == 12.5 and rate == pytest.approx(100 * 4 / 0.0125)
