"""The serving loop (continuous batching over batch-plan slots, streamed inserts).

A request must get the same rows alone and in a mix: batching changes neither
its candidate set nor its DTW arithmetic, so ids and distances are compared
for equality, and every served row is also compared with the per-length group
path and the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1610_07328_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

LENS = (128, 256, 512)


def _indexes(binding, n=300):
    dbs = {m: synth.random_walk(n, m, seed=m + 11) for m in LENS}
    idxs = []
    for m in LENS:
        ix = binding.SSHIndex(m // 8, 3, 15, 4, 25, 0.05, 0)
        ix.add(dbs[m])
        idxs.append(ix)
    return dbs, idxs


def _group_rows(binding, idxs, q, m, k):
    d_q = torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda()
    ids = torch.empty((1, k), dtype=torch.int64, device="cuda")
    dd = torch.empty((1, k), dtype=torch.float32, device="cuda")
    binding.ssh_group_query_device([ix.handle for ix in idxs], d_q, np.array([m], np.int32), k, ids, dd)
    torch.cuda.synchronize()
    return ids.cpu().numpy()[0], dd.cpu().numpy()[0]


def test_server_rows_are_the_same_alone_and_in_a_mix():
    from paper_1610_07328_gb300 import binding
    dbs, idxs = _indexes(binding)
    k = 5
    rng = np.random.default_rng(3)
    try:
        with binding.SSHServer(idxs, k=k, max_batch=16, max_slots=3, reserve_bytes=0) as srv:
            q0, _ = synth.perturbed_queries(dbs[256], 1, seed=99)
            t0 = srv.submit(q0, np.array([256], np.int32))
            ids0, d0, which0, lat0 = srv.wait(t0[0])
            assert which0 == LENS.index(256) and lat0 > 0
            # warm-up: every slot runs its first batch directly and captures its graph
            wq, _ = synth.perturbed_queries(dbs[512], 48, seed=98)
            for t in srv.submit(wq, np.full(48, 512, np.int32)):
                srv.wait(t)
            # a mix of 150 queries of all lengths in three waves, q0 at a random place of the second
            qs, ls = [], []
            for t in range(150):
                m = LENS[int(rng.integers(0, 3))]
                q, _ = synth.perturbed_queries(dbs[m], 1, seed=500 + t)
                qs.append(q[0])
                ls.append(m)
            pos = 50 + int(rng.integers(0, 50))
            qs.insert(pos, q0[0])
            ls.insert(pos, 256)
            tickets = []
            for a, b in ((0, 50), (50, 101), (101, 151)):
                tickets.extend(srv.submit(np.concatenate(qs[a:b]), np.array(ls[a:b], np.int32)).tolist())
            rows = [srv.wait(t) for t in tickets]
            ids_mix, d_mix, which_mix, _ = rows[pos]
            assert np.array_equal(ids_mix, ids0) and np.array_equal(d_mix, d0)
            for i in range(0, 151, 10):  # every tenth row against the group path and the oracle
                m = ls[i]
                gi, gd = _group_rows(binding, idxs, qs[i], m, k)
                assert np.array_equal(rows[i][0], gi) and np.array_equal(rows[i][1], gd)
                assert rows[i][2] == LENS.index(m)
            ref = oracle.OracleIndex(W=32, delta=3, n=15, K=4, L=25, band=0.05, seed=0)
            ref.add(dbs[256])
            oi, od = ref.query(q0[0], k)
            real = oi >= 0
            assert np.array_equal(ids0 >= 0, real)
            np.testing.assert_allclose(d0[real], od[real], rtol=1e-5)
            st = srv.stats()
            assert st["queries_done"] == 152 + 48 and st["errors"] == 0
            assert st["batches"] >= 10 and 1.0 <= st["mean_batch"] <= 16.0
            assert st["slots"] == 3 and st["max_inflight"] >= 2
            # continuous batching: a batch was launched while another slot's batch was still
            # executing on the GPU, and every row above equals its row alone
            assert st["max_inflight_device"] >= 2, st
            assert st["deferred"] == 0 and st["refused"] == 0
    finally:
        for ix in idxs:
            ix.close()


def test_server_inserts_become_visible_and_unknown_lengths_are_refused():
    from paper_1610_07328_gb300 import binding
    dbs, idxs = _indexes(binding, n=200)
    k = 3
    try:
        with binding.SSHServer(idxs, k=k, max_batch=8, max_slots=2, reserve_bytes=0) as srv:
            # queries keep flowing while the inserts arrive
            qs, _ = synth.perturbed_queries(dbs[128], 20, seed=5)
            srv.submit(qs, np.full(20, 128, np.int32))
            new = synth.random_walk(10, 128, seed=321)
            srv.insert(new, np.full(10, 128, np.int32))
            srv.flush(60.0)
            st = srv.stats()
            assert st["inserts_applied"] == 10 and st["insert_errors"] == 0
            t = srv.submit(new[4:5], np.array([128], np.int32))
            ids, dists, which, _ = srv.wait(t[0])
            assert ids[0] == 200 + 4 and dists[0] == 0.0 and which == 0
            with pytest.raises(binding.SSHError) as e:
                srv.submit(np.zeros(100, np.float32), np.array([100], np.int32))
            assert e.value.status == binding.SSH_ELENGTH
    finally:
        for ix in idxs:
            ix.close()


def test_server_admits_candidate_buffers_by_free_memory():
    """Pair buffers grow only while the reserve of free device memory holds. With a reserve of
    the whole device no growth is admitted: a batch whose candidates overflow its slot's 64
    pairs is requeued and split, a single query that still does not fit is answered SSH_EBUSY
    (never SSH_ENOMEM), and queries whose candidates fit are served in smaller batches with the
    same rows as the group path. Without a reserve the same queries are served by growing."""
    from paper_1610_07328_gb300 import binding
    many = synth.random_walk(256, 128, seed=61)   # n = 8, one hash per table: most rows are candidates
    few = synth.random_walk(20, 256, seed=62)     # at most 20 candidates per query
    ix_many = binding.SSHIndex(16, 3, 8, 1, 8, 0.05, 0)
    ix_few = binding.SSHIndex(32, 3, 15, 4, 25, 0.05, 0)
    k = 4
    try:
        ix_many.add(many)
        ix_few.add(few)
        idxs = [ix_many, ix_few]
        q_many, _ = synth.perturbed_queries(many, 8, seed=63)
        q_few, _ = synth.perturbed_queries(few, 4, seed=64)
        # each query's candidate count: alone in a batch, more than 64 pairs cannot be admitted
        n_cand = []
        for q in q_many:
            ix_many.reset_stats()
            ix_many.query(q[None, :], k)
            n_cand.append(ix_many.stats()["candidates"])
        too_big = [c > 64 for c in n_cand]
        assert sum(too_big) >= 4, n_cand
        total = torch.cuda.mem_get_info()[1]
        with binding.SSHServer(idxs, k=k, max_batch=8, max_slots=2, reserve_bytes=total, max_pairs=64) as srv:
            assert srv.stats()["slots"] == 1  # the reserve admits no second slot either
            tickets = srv.submit(q_many, np.full(8, 128, np.int32))
            srv.flush(60.0)
            got = {}
            while len(got) < 8:
                tk, _, _, _, status = srv.collect(64, 1.0)
                got.update(zip(tk.tolist(), status.tolist()))
            assert sorted(got) == sorted(tickets.tolist())
            for t, big in zip(tickets.tolist(), too_big):
                assert got[t] == (binding.SSH_EBUSY if big else binding.SSH_OK), (t, got, n_cand)
            st = srv.stats()
            assert st["refused"] == sum(too_big) and st["errors"] == 0 and st["deferred"] >= 8
            # queries whose candidates fit the admitted buffers are served (in smaller batches)
            t_few = srv.submit(q_few, np.full(4, 256, np.int32))
            rows = [srv.wait(t, 30.0) for t in t_few]
            for i, q in enumerate(q_few):
                gi, gd = _group_rows(binding, idxs, q, 256, k)
                assert np.array_equal(rows[i][0], gi) and np.array_equal(rows[i][1], gd)
                assert rows[i][2] == 1
        with binding.SSHServer(idxs, k=k, max_batch=8, max_slots=2, reserve_bytes=0, max_pairs=64) as srv:
            t_many = srv.submit(q_many, np.full(8, 128, np.int32))
            rows = [srv.wait(t, 30.0) for t in t_many]
            for i, q in enumerate(q_many):
                gi, gd = _group_rows(binding, idxs, q, 128, k)
                assert np.array_equal(rows[i][0], gi) and np.array_equal(rows[i][1], gd)
            st = srv.stats()
            assert st["deferred"] == 0 and st["refused"] == 0 and st["errors"] == 0
    finally:
        ix_many.close()
        ix_few.close()
