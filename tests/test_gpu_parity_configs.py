"""GPU parity at the long-series configurations: the ECG-like configuration
(m = 1024, W = 120, delta = 5, n = 15, K = 4, L = 50, band 10%, so the
Sakoe-Chiba radius is 102), and batch plans whose length classes are 1024 and
2048 (W = m/8, radii 51 and 102, several lanes per DTW pair).

Each query goes end to end through the C ABI (hash, probe + union, LB_Keogh,
the seed DTWs that bound the k-th distance, early-abandoning DTW of the
survivors, top-k) and is compared with the oracle's Algorithm 2 (or its exact
brute-force top-k for the exact scan): ids exactly, up to near ties, and
distances within 1e-5 relative.
"""
import numpy as np
import pytest

import oracle
from paper_1610_07328_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

RTOL = 1e-5
CFG3 = dict(W=120, delta=5, n=15, K=4, L=50, band=0.10, seed=0)


def _binding():
    from paper_1610_07328_gb300 import binding
    return binding


def _index(cfg):
    return _binding().SSHIndex(cfg["W"], cfg["delta"], cfg["n"], cfg["K"], cfg["L"], cfg["band"], cfg["seed"])


def assert_topk_match(q, ids_g, d_g, ids_o, d_o, db_by_id, rb):
    real = ids_o >= 0
    assert np.array_equal(ids_g >= 0, real)
    np.testing.assert_allclose(d_g[real], d_o[real], rtol=RTOL, atol=0)
    for t in np.nonzero(real)[0]:
        if ids_g[t] != ids_o[t]:
            # a near tie: the returned id's exact distance must equal the oracle's t-th distance
            dd = oracle.dtw(q, db_by_id(int(ids_g[t])), rb)
            assert abs(dd - d_o[t]) <= RTOL * d_o[t], (t, ids_g[t], ids_o[t], dd, d_o[t])
    assert len(set(ids_g[real].tolist())) == int(real.sum())


@pytest.fixture(scope="module")
def ecg():
    """1,200 ECG-like series of length 1024 and 10 queries made from them (noise and a shift),
    with the oracle's index over the same rows."""
    db = synth.ecg_like(1200, 1024, seed=31)
    qs, _ = synth.perturbed_queries(db, 10, seed=32)
    ref = oracle.OracleIndex(**CFG3)
    ref.add(db)
    return db, qs, ref


@pytest.mark.parametrize("prune", [True, False])
def test_ecg_config_query_matches_oracle(ecg, prune):
    db, qs, ref = ecg
    rb = oracle.band_radius(CFG3["band"], 1024)
    assert rb == 102
    with _index(CFG3) as idx:
        idx.set_lb_prune(prune)
        idx.add(db)
        ids, d = idx.query(qs, 10)
        st = idx.stats()
    for i, q in enumerate(qs):
        oi, od = ref.query(q, 10)
        assert_topk_match(q, ids[i], d[i], oi, od, lambda j: db[j], rb)
    assert st["candidates"] == sum(len(ref.candidates(q)) for q in qs)


@pytest.mark.parametrize("prune", [True, False])
def test_ecg_config_exact_scan_with_seed_bound_and_abandoning(ecg, prune):
    """Every one of the 1,200 rows is a candidate: the 160 rows of smallest LB_Keogh are the
    seeds whose DTWs give the bound U, the rest are pruned by LB_Keogh against U or run with
    early abandoning (band checked every few anti-diagonals) at radius 102."""
    db, qs, ref = ecg
    rb = oracle.band_radius(CFG3["band"], 1024)
    qs = qs[:6]
    with _index(CFG3) as idx:
        idx.add(db)
        idx.set_exact_scan(True)
        idx.set_lb_prune(prune)
        ids, d = idx.query(qs, 10)
        st = idx.stats()
    assert st["candidates"] == len(qs) * len(db)
    if prune:
        assert st["dtw_computed"] + st["lb_pruned"] == st["candidates"]
    else:
        assert st["dtw_computed"] == st["candidates"]
    for i, q in enumerate(qs):
        oi, od = ref.exact_topk(q, 10)
        assert_topk_match(q, ids[i], d[i], oi, od, lambda j: db[j], rb)


def test_ecg_config_abandoning_cuts_dtw_work(ecg):
    """The abandon test fires at radius 102: with pruning on, the survivors' DTW pass computes
    fewer cells than complete DTWs of the same pairs would (the library's per-group cell count
    is the work actually done), while the results equal the oracle's."""
    db, qs, ref = ecg
    with _index(CFG3) as idx:
        idx.add(db)
        idx.set_exact_scan(True)
        idx.set_kernel_timing(True)
        ids, d = idx.query(qs[:4], 10)
        st = idx.stats()
        kt = idx.kernel_times()
    rb = oracle.band_radius(CFG3["band"], 1024)
    full_cells = 1024 * (2 * rb + 1) - rb * (rb + 1)
    done = kt["query.dtw"]["units"]
    assert 0 < done < st["dtw_computed"] * full_cells
    for i, q in enumerate(qs[:4]):
        oi, od = ref.exact_topk(q, 10)
        assert_topk_match(q, ids[i], d[i], oi, od, lambda j: db[j], rb)


# ------------------------------------------------ batch plans: the long length classes

def _mixed(dbs, lens, nq, seed):
    rng = np.random.default_rng(seed)
    qs, qlens = [], []
    for t in range(nq):
        m = lens[int(rng.integers(0, len(lens)))]
        q, _ = synth.perturbed_queries(dbs[m], 1, seed=seed * 1000 + t)
        qs.append(q[0])
        qlens.append(m)
    return qs, np.array(qlens, np.int32)


def _run_batch(bt, qs, qlens, k):
    d_q = torch.from_numpy(np.concatenate(qs)).cuda()
    ids = torch.full((len(qs), k), -7, dtype=torch.int64, device="cuda")
    dd = torch.zeros((len(qs), k), dtype=torch.float32, device="cuda")
    which = torch.full((len(qs),), -1, dtype=torch.int32, device="cuda")
    bt.query(d_q, qlens, ids, dd, which)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dd.cpu().numpy(), which.cpu().numpy()


def _run_group(idxs, qs, qlens, k):
    d_q = torch.from_numpy(np.concatenate(qs)).cuda()
    ids = torch.empty((len(qs), k), dtype=torch.int64, device="cuda")
    dd = torch.empty((len(qs), k), dtype=torch.float32, device="cuda")
    which = torch.full((len(qs),), -1, dtype=torch.int32, device="cuda")
    _binding().ssh_group_query_device([ix.handle for ix in idxs], d_q, qlens, k, ids, dd, which)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dd.cpu().numpy(), which.cpu().numpy()


@pytest.mark.parametrize("n,K,rows", [(15, 4, 150), (8, 1, 400)], ids=["config4-params", "many-candidates"])
def test_batch_plan_long_classes_match_oracle(n, K, rows):
    """Classes 1024 and 2048 (W = m/8, radii 51 and 102) through one plan, direct and replayed.
    With n = 8 and one hash per table most rows are candidates, so the seed bound and early
    abandoning run in the plan's per-class DTW passes."""
    b = _binding()
    lens = (1024, 2048, 128)
    nrows = {1024: rows, 2048: rows * 3 // 4, 128: rows}
    dbs = {m: synth.random_walk(nrows[m], m, seed=m + 11) for m in lens}
    cfgs = {m: dict(W=m // 8, delta=3, n=n, K=K, L=25, band=0.05, seed=0) for m in lens}
    idxs, refs = [], {}
    try:
        for m in lens:
            ix = _index(cfgs[m])
            ix.add(dbs[m])
            idxs.append(ix)
            refs[m] = oracle.OracleIndex(**cfgs[m])
            refs[m].add(dbs[m])
        k = 10
        with b.SSHBatch(idxs, max_queries=32, k=k) as bt:
            for rep in range(2):  # rep 0 runs directly, rep 1 replays the graph
                qs, qlens = _mixed(dbs, lens, 12 + 4 * rep, seed=40 + rep)
                ids, dd, which = _run_batch(bt, qs, qlens, k)
                for i, (q, m) in enumerate(zip(qs, qlens)):
                    assert which[i] == lens.index(m)
                    oi, od = refs[m].query(q, k)
                    assert_topk_match(q, ids[i], dd[i], oi, od, lambda j: dbs[m][j], oracle.band_radius(0.05, m))
                gi, gd, gw = _run_group(idxs, qs, qlens, k)
                assert np.array_equal(ids, gi) and np.array_equal(dd, gd) and np.array_equal(which, gw)
            st = bt.stats()
            assert st["pairs"] > 0 and 0 < st["dtw"] <= st["pairs"]
            if K == 1:
                assert st["pairs"] > 16 * k * 12  # more candidates than seeds: survivors were filtered
    finally:
        for ix in idxs:
            ix.close()


def test_reversed_lb_skip_is_counted():
    """A length whose candidate envelopes do not fit in shared memory (m = 12,000): the
    requested reversed LB_Keogh pass is skipped, counted per query in lb2_skipped, and the
    results equal those of the cascade without it."""
    m = 12_000
    cfg = dict(W=1500, delta=50, n=8, K=2, L=4, band=0.01, seed=0)  # radius 120
    db = synth.random_walk(40, m, seed=51)
    qs, _ = synth.perturbed_queries(db, 3, seed=52)
    with _index(cfg) as idx:
        idx.add(db)
        idx.set_exact_scan(True)
        idx.set_lb_cascade(1)
        ids1, d1 = idx.query(qs, 5)
        idx.reset_stats()
        idx.set_lb_cascade(2)
        ids2, d2 = idx.query(qs, 5)
        st = idx.stats()
    assert st["lb2_skipped"] == len(qs) and st["lb2_pruned"] == 0
    assert np.array_equal(ids1, ids2) and np.array_equal(d1, d2)
    # At this length the FP32 path sum (about 2m terms) is outside the 1e-5 bound the configured
    # lengths (128 .. 2048) meet; its own bound is the worst case of a 2m-term sum of
    # non-negative FP32 terms, 2m 2^-24 relative.
    rb = oracle.band_radius(cfg["band"], m)
    tol = 2 * m * 2.0 ** -24
    for i, q in enumerate(qs):
        oi, od = oracle.topk_dtw(q, db, np.arange(len(db)), rb, 5)
        np.testing.assert_allclose(d2[i], od, rtol=tol, atol=0)
        for t in range(5):
            if ids2[i, t] != oi[t]:  # a near tie at this tolerance
                assert abs(oracle.dtw(q, db[ids2[i, t]], rb) - od[t]) <= 2 * tol * od[t]


# --------------------------------------------- shingles longer than the draw tables

def _unpack_bits(words, nb):
    return np.array([(int(words[i // 32]) >> (31 - i % 32)) & 1 for i in range(nb)], np.uint8)


@pytest.mark.parametrize("n", [17, 20, 32])
def test_long_shingles_hash_and_query_match_the_oracle(n):
    """n > 16: no draw tables; every minhash is the FP64 argmin with its Philox draws computed
    in the kernel. Sketch bits, shingle sets, (k*, t*) and keys are bit-exact with the oracle,
    and queries equal the oracle's Algorithm 2."""
    b = _binding()
    cfg = dict(W=16, delta=2, n=n, K=2, L=8, band=0.05, seed=3)
    m, N = 128, 300
    x = synth.random_walk(N, m, seed=70 + n)
    nb = (m - cfg["W"]) // cfg["delta"] + 1
    S = nb - n + 1
    KL = cfg["K"] * cfg["L"]
    r = oracle.filter_r(cfg["seed"], cfg["W"])
    with _index(cfg) as idx:
        d_x = torch.from_numpy(x).cuda()
        bits = torch.zeros((N, (nb + 31) // 32), dtype=torch.int32, device="cuda")
        ids = torch.zeros((N, S), dtype=torch.int32, device="cuda")
        cnt = torch.zeros((N, S), dtype=torch.int32, device="cuda")
        nnz = torch.zeros(N, dtype=torch.int32, device="cuda")
        ks = torch.zeros((N, KL), dtype=torch.int32, device="cuda")
        ts = torch.zeros((N, KL), dtype=torch.int32, device="cuda")
        keys = torch.zeros((cfg["L"], N), dtype=torch.int64, device="cuda")
        b.ssh_hash_device(idx.handle, d_x, m, N, bits, ids, cnt, nnz, ks, ts, keys)
        torch.cuda.synchronize()
        u32 = lambda t: t.cpu().numpy().view(np.uint32)
        g_bits, g_ids, g_cnt, g_ks, g_ts = u32(bits), u32(ids), u32(cnt), u32(ks), u32(ts)
        g_nnz, g_keys = nnz.cpu().numpy(), keys.cpu().numpy().view(np.uint64)
        for i in range(0, N, 7):
            ob = oracle.sketch(x[i], r, cfg["delta"])
            assert np.array_equal(_unpack_bits(g_bits[i], nb), ob), i
            sid, scnt = oracle.shingle(ob, n)
            k = int(g_nnz[i])
            assert k == len(sid) and np.array_equal(g_ids[i, :k], sid) and np.array_equal(g_cnt[i, :k], scnt), i
            oks, ots = oracle.cws(cfg["seed"], KL, sid, scnt)
            assert np.array_equal(g_ks[i], oks) and np.array_equal(g_ts[i], ots), i
            for l in range(cfg["L"]):
                assert int(g_keys[l, i]) == oracle.bucket_key(cfg["seed"], l, cfg["K"], oks, ots), (l, i)
        # Algorithm 2 end to end
        idx.add(x)
        qs, _ = synth.perturbed_queries(x, 6, seed=80 + n)
        q_ids, q_d = idx.query(qs, 5)
        st = idx.stats()
    ref = oracle.OracleIndex(**cfg)
    ref.add(x)
    rb = oracle.band_radius(cfg["band"], m)
    for i, q in enumerate(qs):
        oi, od = ref.query(q, 5)
        assert_topk_match(q, q_ids[i], q_d[i], oi, od, lambda j: x[j], rb)
    assert st["candidates"] == sum(len(ref.candidates(q)) for q in qs)


@pytest.mark.parametrize("n,K", [(15, 4), (8, 1)], ids=["config4-params", "many-candidates"])
def test_persistent_rerank_equals_per_class_kernels_at_all_lengths(n, K):
    """The batch's rerank as one persistent launch and as per-class kernels give the same rows
    bit for bit at every length class (128 .. 2048, radii 6 .. 102), directly and replayed,
    and both equal the oracle's Algorithm 2; the persistent plan's graph holds far fewer
    kernels."""
    b = _binding()
    lens = (128, 256, 512, 1024, 2048)
    nrows = {128: 300, 256: 300, 512: 250, 1024: 200, 2048: 150}
    dbs = {m: synth.random_walk(nrows[m], m, seed=m + 21) for m in lens}
    cfgs = {m: dict(W=m // 8, delta=3, n=n, K=K, L=25, band=0.05, seed=0) for m in lens}
    idxs, refs = [], {}
    try:
        for m in lens:
            ix = _index(cfgs[m])
            ix.add(dbs[m])
            idxs.append(ix)
            refs[m] = oracle.OracleIndex(**cfgs[m])
            refs[m].add(dbs[m])
        k = 10
        kernels = {}
        with b.SSHBatch(idxs, max_queries=40, k=k) as bt:
            for rep in range(2):
                qs, qlens = _mixed(dbs, lens, 30 + 5 * rep, seed=60 + rep)
                rows = {}
                for persistent in (True, False):
                    bt.set_persistent(persistent)
                    for _ in range(2):  # the first batch after the switch runs directly, the second replays
                        rows[persistent] = _run_batch(bt, qs, qlens, k)
                    kernels[persistent] = bt.stats()["graph_kernels"]
                for x, y in zip(rows[True], rows[False]):
                    assert np.array_equal(x, y)
                ids, dd, which = rows[True]
                for i, (q, m) in enumerate(zip(qs, qlens)):
                    assert which[i] == lens.index(m)
                    oi, od = refs[m].query(q, k)
                    assert_topk_match(q, ids[i], dd[i], oi, od, lambda j: dbs[m][j], oracle.band_radius(0.05, m))
        assert kernels[True] < kernels[False] and kernels[True] <= 30, kernels
    finally:
        for ix in idxs:
            ix.close()
