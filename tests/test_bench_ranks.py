"""bench.py's multi-rank aggregation on CPU with two gloo ranks.

Several GPUs run independent replicas of the sweep (weak scaling). The
whole-job rate counts every rank's units and divides by the slowest rank's
time, the max over ranks.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, local_ms: list, q) -> None:
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        value, total_ms = bench.whole_job_rate(local_ms[rank], 1000, 5, dist, torch.device("cpu"))
        q.put((rank, value, total_ms))
    finally:
        dist.destroy_process_group()


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench

    value, total_ms = bench.whole_job_rate(125.0, 1000, 5)
    assert total_ms == 125.0
    assert value == pytest.approx(1000 * 5 / 0.125)


def test_two_rank_rate_takes_the_slowest_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    local_ms = [120.0, 200.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, local_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        results = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [r for r, _, _ in results] == [0, 1]
    for _, value, total_ms in results:
        assert total_ms == 200.0  # max over ranks
        assert value == pytest.approx(2 * 1000 * 5 / 0.2)  # both ranks' units over the slowest time
    assert all(p.exitcode == 0 for p in procs)
