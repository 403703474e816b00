"""The sharded query's host logic on CPU: id ranges, and the all-gather merge of
per-rank top-k lists run by two gloo processes, against the top-k of the whole
collection computed in one place (the oracle's banded DTW over tiny series)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1610_07328_gb300 import shard, synth

torch = pytest.importorskip("torch")


def test_shard_bounds_cover_the_ids_once():
    for n in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            ranges = [shard.shard_bounds(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_bounds(10, 2, 2)


def test_merge_topk_orders_by_distance_then_id_and_drops_empty_slots():
    ids = np.array([[[5, 9, -1]], [[2, 7, 8]]])
    d = np.array([[[1.0, 3.0, np.inf]], [[1.0, 2.0, 3.0]]], np.float32)
    mi, md = shard.merge_topk(ids, d, 4)
    assert mi.tolist() == [[2, 5, 7, 8]]
    assert md.tolist() == [[1.0, 1.0, 2.0, 3.0]]
    mi, md = shard.merge_topk(np.full((2, 1, 2), -1), np.full((2, 1, 2), np.inf, np.float32), 3)
    assert mi.tolist() == [[-1, -1, -1]] and np.isinf(md).all()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, db, qs, k, rb, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard.shard_bounds(len(db), rank, world)
    ids = np.full((len(qs), k), -1, np.int64)
    dd = np.full((len(qs), k), np.inf, np.float32)
    for i, q in enumerate(qs):
        li, ld = oracle.topk_dtw(q, db[lo:hi], np.arange(lo, hi), rb, k)
        ids[i], dd[i] = li, ld
    mi, md = shard.allgather_topk(torch.from_numpy(ids), torch.from_numpy(dd), k)
    out[rank] = (mi, md)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_to_the_global_topk():
    import torch.multiprocessing as mp
    db = synth.random_walk(60, 32, seed=2)
    qs, _ = synth.perturbed_queries(db, 5, seed=3)
    k, rb = 4, oracle.band_radius(0.1, 32)
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, db, qs, k, rb, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for i, q in enumerate(qs):
        gi, gd = oracle.topk_dtw(q, db, np.arange(len(db)), rb, k)
        for r in range(2):
            mi, md = out[r]
            assert mi[i].tolist() == list(gi)
            np.testing.assert_allclose(md[i], gd, rtol=1e-6)
