"""CPU tests of bench.py's host logic: the multi-rank path (world_size 2,
gloo, 127.0.0.1) and the clock-sample summary. No GPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, world)   # rank 1 is the slow one
    bench.barrier(world)
    value = bench.aggregate(1.0e12, world, ms)
    q.put((rank, ms, value, bench.dist_env()))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, env in out:
        assert ms == 150.0                      # max over ranks
        assert value == pytest.approx(2 * 1.0e12 / 0.150)   # both ranks' work / slowest time
        assert env == (2, rank, rank)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate(10.0, 1, 1000.0) == 10.0


def test_clock_summary():
    sys.path.insert(0, ROOT)
    import bench
    lines = [
        "0, 345, 2070, 120.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1010.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = bench.summarize_clocks(lines)
    assert c["sm_max_mhz"] == 2070
    assert c["sm_mhz"] == 2070          # the idle 345 MHz sample is not "under load"
    assert c["reasons"] == ["sw_power_cap"]
    assert bench.summarize_clocks([])["samples"] == 0
