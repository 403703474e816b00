"""Parity at the full benchmark size, in the launch configuration the benchmark
times: 1,000,000 random walks of length 512 (W=80, delta=3, n=15, K=4, L=25,
band 5%), added as one borrowed device batch and queried with 100 perturbed
database series (top-10), as one benchmark step does.

The oracle cannot hash a million series in a test, so it checks sampled outputs
one by one:
- bucket keys of 64 rows (the first, the last, and rows spread over the whole
  batch) from the same million-row hash launch, bit-exact;
- for 4 of the queries, the exact top-10 by the oracle's banded DTW over the
  query's whole candidate set (every row that shares a bucket key with the
  oracle's keys of the query), against the returned ids and distances;
- for all 100 queries, properties that hold at any size: ids in (distance, id)
  order, no repeats, and every returned distance the oracle's DTW of that pair
  (on the sampled queries).
"""
import numpy as np
import pytest

import oracle
from paper_1610_07328_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

RTOL = 1e-5
N, M, NQ, K = 1_000_000, 512, 100, 10
CFG = dict(W=80, delta=3, n=15, K=4, L=25, band=0.05, seed=0)


@pytest.fixture(scope="module")
def scale_run():
    from paper_1610_07328_gb300 import binding
    db = synth.random_walk(N, M, seed=CFG["seed"])
    qs, _ = synth.perturbed_queries(db[:10_000], NQ, seed=1)
    d_db = torch.from_numpy(db).cuda()
    d_q = torch.from_numpy(qs).cuda()
    ids = torch.empty((NQ, K), dtype=torch.int64, device="cuda")
    dd = torch.empty((NQ, K), dtype=torch.float32, device="cuda")
    keys = torch.empty((CFG["L"], N), dtype=torch.int64, device="cuda")
    with binding.SSHIndex(CFG["W"], CFG["delta"], CFG["n"], CFG["K"], CFG["L"], CFG["band"], CFG["seed"]) as idx:
        idx.add_device(d_db, borrow=True)
        idx.query_device(d_q, K, ids, dd)
        binding.ssh_hash_device(idx.handle, d_db, M, N, d_keys=keys)
        torch.cuda.synchronize()
        out = dict(db=db, qs=qs, ids=ids.cpu().numpy(), dists=dd.cpu().numpy(), keys=keys,
                   stats=idx.stats())
    del d_db, d_q
    return out


def test_sampled_bucket_keys_of_the_million_row_launch(scale_run):
    db, keys = scale_run["db"], scale_run["keys"]
    r = oracle.filter_r(CFG["seed"], CFG["W"])
    rows = np.unique(np.concatenate([[0, N - 1], np.random.default_rng(5).integers(0, N, 62)]))
    got = keys[:, torch.from_numpy(rows).cuda()].cpu().numpy().view(np.uint64)
    for c, i in enumerate(rows):
        ks, ts = oracle.hash_series(db[i], r, CFG["delta"], CFG["n"], CFG["seed"], CFG["K"], CFG["L"])
        for l in range(CFG["L"]):
            assert int(got[l, c]) == oracle.bucket_key(CFG["seed"], l, CFG["K"], ks, ts), (i, l)


def test_every_query_row_is_ordered_and_distinct(scale_run):
    ids, d = scale_run["ids"], scale_run["dists"]
    for i in range(NQ):
        real = ids[i] >= 0
        n = int(real.sum())
        assert real[:n].all() and not real[n:].any()
        assert np.isinf(d[i, n:]).all() and np.isfinite(d[i, :n]).all()
        assert len(set(ids[i, :n].tolist())) == n
        pairs = list(zip(d[i, :n].tolist(), ids[i, :n].tolist()))
        assert pairs == sorted(pairs)


@pytest.mark.parametrize("qi", [0, 31, 62, 99])
def test_sampled_queries_equal_the_oracle_topk_over_their_candidates(scale_run, qi):
    db, qs, keys = scale_run["db"], scale_run["qs"], scale_run["keys"]
    q = qs[qi]
    r = oracle.filter_r(CFG["seed"], CFG["W"])
    ks, ts = oracle.hash_series(q, r, CFG["delta"], CFG["n"], CFG["seed"], CFG["K"], CFG["L"])
    qkeys = np.array([oracle.bucket_key(CFG["seed"], l, CFG["K"], ks, ts) for l in range(CFG["L"])], np.uint64)
    qk = torch.from_numpy(qkeys.view(np.int64)).cuda().view(-1, 1)
    cand = torch.nonzero((keys == qk).any(dim=0)).flatten().cpu().numpy().astype(np.int64)
    rb = oracle.band_radius(CFG["band"], M)
    oi, od = oracle.topk_dtw(q, db[cand], cand, rb, K)
    gi, gd = scale_run["ids"][qi], scale_run["dists"][qi]
    real = oi >= 0
    assert np.array_equal(gi >= 0, real)
    np.testing.assert_allclose(gd[real], od[real], rtol=RTOL, atol=0)
    cset = set(cand.tolist())
    for t in np.nonzero(real)[0]:
        assert int(gi[t]) in cset
        if gi[t] != oi[t]:  # a near tie: the returned id's exact distance is the oracle's t-th
            dd = oracle.dtw(q, db[int(gi[t])], rb)
            assert abs(dd - od[t]) <= RTOL * od[t], (t, gi[t], oi[t], dd, od[t])
