"""The multi-GPU bookkeeping of bench.py on CPU: two gloo ranks, each with its
own (different) timed total, agree on the slowest rank's time, and the
whole-job throughput counts every rank's queries (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 + 5.0 * rank          # ms: rank 1 is the slower one
        slowest = bench.max_over_ranks(dist, mine, torch.device("cpu"))
        out[rank] = (slowest, bench.job_throughput(ws, 16, 20, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        slowest, qps = res[r]
        assert slowest == 15.0
        assert qps == pytest.approx(2 * 16 * 20 / 0.015)


def test_single_rank_passes_through():
    assert bench.max_over_ranks(None, 7.5, torch.device("cpu")) == 7.5
    assert bench.job_throughput(1, 16, 10, 5.0) == pytest.approx(32000.0)
