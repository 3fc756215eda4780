"""Row-sharded search, host side, on CPU: the row partition covers every row
once, and the exchange over two gloo ranks delivers every shard's top-k
list and the global selected-row count, so that the k best of the gathered
lists (global ids = local ids + the shard's row offset) are the exact
filtered top-k of the whole table.  The shard lists come from the float64
oracle on each rank's rows; the GPU merge kernel itself is tested in
test_gpu_shards.py."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402
from _parity import check_topk  # noqa: E402
from paper_2403_15807_gb300 import shards  # noqa: E402


@pytest.mark.parametrize("n,world", [(1, 1), (7, 3), (1000, 2), (1001, 4), (5, 8)])
def test_shard_rows_partition(n, world):
    seen = np.zeros(n, dtype=int)
    prev = 0
    for r in range(world):
        lo, hi = shards.shard_rows(n, world, r)
        assert lo == prev and hi >= lo and hi - lo in (n // world, n // world + 1)
        seen[lo:hi] += 1
        prev = hi
    assert prev == n and np.all(seen == 1)
    assert list(shards.row_offsets(n, world)) == [shards.shard_rows(n, world, r)[0]
                                                  for r in range(world)]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


N, D, B, K = 3001, 16, 6, 8


def _inputs():
    mix = gen.Mixture(D, seed=5)
    return gen.vectors(N, mix), gen.queries(B, mix), gen.attributes(N, 1, 100, seed=5)


def _rank(rank, world, port, metric, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, q, attrs = _inputs()
        lo, hi = shards.shard_rows(N, world, rank)
        # attr < 3 keeps ~3 % of the rows: some shards hold fewer than K
        pred = gen.pred_less_than(3)
        ids, dd, cnt = oracle.query(x[lo:hi], attrs[:, lo:hi], q, [pred], K, metric)
        ids_all, d_all = shards.gather_topk(dist, torch.from_numpy(ids),
                                            torch.from_numpy(dd.astype(np.float32)))
        total = shards.global_count(dist, int(cnt[0]), torch.device("cpu"))
        out[rank] = (ids_all.numpy(), d_all.numpy(), total)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _reference_merge(ids_all, d_all, offsets, metric):
    """k best of the gathered lists by (key, global id): the test's own merge."""
    w, b, k = ids_all.shape
    out_i = np.full((b, k), -1, dtype=np.int64)
    out_d = np.full((b, k), np.inf, dtype=np.float64)
    for i in range(b):
        c = [((v if metric == "l2" else -v), int(g) + int(offsets[s]))
             for s in range(w) for g, v in zip(ids_all[s, i], d_all[s, i]) if g >= 0]
        c.sort()
        for j, (key, gid) in enumerate(c[:k]):
            out_i[i, j] = gid
            out_d[i, j] = key if metric == "l2" else -key
    return out_i, out_d


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_two_gloo_ranks_exchange_and_merge(metric):
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), metric, out), nprocs=world, join=True)
        res = dict(out)
    x, q, attrs = _inputs()
    pred = gen.pred_less_than(3)
    rid, rdist, rcnt = oracle.query(x, attrs, q, [pred], K + 1, metric)
    offsets = shards.row_offsets(N, world)
    for r in range(world):
        ids_all, d_all, total = res[r]
        assert ids_all.shape == (world, B, K)
        assert total == int(rcnt[0])          # the global count is the sum
        gi, gd = _reference_merge(ids_all, d_all, offsets, metric)
        check_topk(x, q, attrs, [pred], np.int32([K]), metric, gi, gd, rid, rdist, rcnt)
