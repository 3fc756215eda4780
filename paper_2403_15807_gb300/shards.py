"""Row-sharded filtered top-k over several GPUs: one process, one GPU and one
engine per shard.

The table's rows are split into contiguous ranges, one per rank (rows are
independent under the relational selection and the distance, Sec. 3: the
selection filters rows one by one).  Every rank answers the same query batch
over its own rows with vrs_query, the ranks exchange their [batch x k] lists
with one all-gather, and vrs_merge_shards keeps each query's k best of the
union after turning local row ids into global ones.  The selected-row count
of a shared predicate is the sum of the shards' counts.

Only the exchange is host code (torch.distributed: NCCL between GPUs, gloo
on CPU); the search and the merge run in the library's kernels.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def shard_rows(n: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous row range [lo, hi) of `rank` among `world` shards (sizes
    differ by at most one row)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} out of 0..{world - 1}")
    return n * rank // world, n * (rank + 1) // world


def row_offsets(n: int, world: int) -> np.ndarray:
    """Global id of each shard's row 0."""
    return np.array([shard_rows(n, world, r)[0] for r in range(world)], dtype=np.int64)


def gather_topk(dist, ids, dists):
    """All-gather every rank's [batch x k] top-k lists (torch tensors on this
    rank's device: CUDA with NCCL, CPU with gloo).  Returns shard-major
    [world x batch x k] tensors."""
    import torch
    world = dist.get_world_size()
    out_i = [torch.empty_like(ids) for _ in range(world)]
    out_d = [torch.empty_like(dists) for _ in range(world)]
    dist.all_gather(out_i, ids.contiguous())
    dist.all_gather(out_d, dists.contiguous())
    return torch.stack(out_i), torch.stack(out_d)


def global_count(dist, count: int, device) -> int:
    """Selected rows over all shards (sum of the local counts)."""
    import torch
    t = torch.tensor([int(count)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


def merge(vrs, ids_all, dists_all, offsets, metric: int, stream=None):
    """Global top-k from the gathered lists (vrs_merge_shards, on the GPU
    holding the tensors)."""
    return vrs.vrs_merge_shards(ids_all.contiguous(), dists_all.contiguous(), offsets, metric,
                                stream=stream)
