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
            assert st["queries_done"] == 152 and st["errors"] == 0
            assert st["batches"] >= 10 and 1.0 <= st["mean_batch"] <= 16.0
            assert st["slots"] >= 1 and st["max_inflight"] >= 1
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
