"""The replicas-only multi-GPU path of bench.py on CPU: two gloo ranks, each
with its own time, agree on the slowest one, and the job value counts the
updates of both ranks (no data-path collective exists)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 20.0][rank]
        job = bench.aggregate_ms(ms, dist)
        out[rank] = (job, bench.job_value(1e9, 10, world, job))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    # 2 ranks x 1e9 points x 10 steps in 20 ms
    assert abs(res[0][1] - 2 * 1e9 * 10 / 0.020 / 1e9) < 1e-9


def test_single_rank_is_unchanged():
    assert bench.aggregate_ms(7.0, None) == 7.0
    assert bench.job_value(2e9, 3, 1, 1000.0) == pytest.approx(6.0)
