"""Id-range shards across GPUs and the one exchange step of a sharded query.

Each rank holds the series of one contiguous id range and answers every query
on its shard; a query's global top-k is then the k smallest (distance, id)
pairs among the ranks' local top-k lists, gathered with one all-gather of
[nq, k] ids and distances. Ids are global: a rank adds its range start to the
ids of its index. Empty slots (id -1, distance +inf) sort last.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) ids of rank's shard: contiguous ranges, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def merge_topk(ids: np.ndarray, dists: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Global top-k from per-rank lists: ids/dists [ranks, nq, k] (global ids, -1 empty)
    -> ([nq, k] ids, [nq, k] distances) ordered by (distance, id)."""
    ids = np.asarray(ids)
    dists = np.asarray(dists, dtype=np.float32)
    r, nq, kk = ids.shape
    flat_i = ids.transpose(1, 0, 2).reshape(nq, r * kk)
    flat_d = dists.transpose(1, 0, 2).reshape(nq, r * kk).astype(np.float64)
    flat_d = np.where(flat_i < 0, np.inf, flat_d)
    id_key = np.where(flat_i < 0, np.iinfo(np.int64).max, flat_i)
    # every row at once: order by (distance, id), empty slots last, keep the first k
    order = np.lexsort((id_key, flat_d), axis=-1)[:, :k]
    top_i = np.take_along_axis(flat_i, order, axis=1).astype(np.int64)
    top_d = np.take_along_axis(flat_d, order, axis=1)
    out_i = np.full((nq, k), -1, np.int64)
    out_d = np.full((nq, k), np.inf, np.float32)
    w = top_i.shape[1]
    out_i[:, :w] = np.where(top_i >= 0, top_i, -1)
    out_d[:, :w] = np.where(top_i >= 0, top_d, np.inf).astype(np.float32)
    return out_i, out_d


def allgather_topk(ids, dists, k: int, group=None):
    """The exchange step: all-gather every rank's [nq, k] global ids and distances
    (torch tensors on the process group's device) and merge them on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    gi = [torch.empty_like(ids) for _ in range(world)]
    gd = [torch.empty_like(dists) for _ in range(world)]
    dist.all_gather(gi, ids.contiguous(), group=group)
    dist.all_gather(gd, dists.contiguous(), group=group)
    all_i = np.stack([t.cpu().numpy() for t in gi])
    all_d = np.stack([t.cpu().numpy() for t in gd])
    return merge_topk(all_i, all_d, k)
