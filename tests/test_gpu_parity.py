"""GPU parity: the CUDA library (through the C ABI) against the FP64 CPU oracle
on the same seeded inputs.

Bars: sketch bits, shingle ids/counts, minhash (k*, t*) and bucket keys are
bit-exact; DTW and LB_Keogh distances agree to 1e-5 relative (FP32 kernels vs
FP64 oracle); top-k ids agree exactly except where two oracle distances lie
within that tolerance of each other, in which case either order is accepted
and each returned distance is checked against the oracle's DTW of that id.
"""
import numpy as np
import pytest

import oracle
from paper_1610_07328_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

RTOL = 1e-5

CFG1 = dict(W=32, delta=3, n=8, K=4, L=16, band=0.05, seed=0)          # tiny: m=128
CFG2 = dict(W=80, delta=3, n=15, K=4, L=25, band=0.05, seed=0)         # scale: m=512
CFG3 = dict(W=120, delta=5, n=15, K=4, L=50, band=0.10, seed=0)        # ECG-like: m=1024


def _binding():
    from paper_1610_07328_gb300 import binding
    return binding


def _index(cfg):
    return _binding().SSHIndex(cfg["W"], cfg["delta"], cfg["n"], cfg["K"], cfg["L"], cfg["band"], cfg["seed"])


def _unpack_bits(words, nb):
    out = np.zeros(nb, np.uint8)
    for i in range(nb):
        out[i] = (int(words[i // 32]) >> (31 - i % 32)) & 1
    return out


def gpu_hash(idx, x: np.ndarray):
    b = _binding()
    N, m = x.shape
    W, delta, n, KL, L = idx.W, idx.delta, idx.n, idx.K * idx.L, idx.L
    nb = (m - W) // delta + 1
    nw = (nb + 31) // 32
    S = nb - n + 1
    dev = "cuda"
    d_x = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    bits = torch.zeros((N, nw), dtype=torch.int32, device=dev)
    ids = torch.zeros((N, S), dtype=torch.int32, device=dev)
    cnt = torch.zeros((N, S), dtype=torch.int32, device=dev)
    nnz = torch.zeros(N, dtype=torch.int32, device=dev)
    ks = torch.zeros((N, KL), dtype=torch.int32, device=dev)
    ts = torch.zeros((N, KL), dtype=torch.int32, device=dev)
    keys = torch.zeros((L, N), dtype=torch.int64, device=dev)
    b.ssh_hash_device(idx.handle, d_x, m, N, bits, ids, cnt, nnz, ks, ts, keys)
    torch.cuda.synchronize()
    u32 = lambda t: t.cpu().numpy().view(np.uint32)
    return dict(bits=u32(bits), ids=u32(ids), cnt=u32(cnt), nnz=nnz.cpu().numpy(), ks=u32(ks), ts=u32(ts),
                keys=keys.cpu().numpy().view(np.uint64), nb=nb)


def check_hash_parity(cfg, x, rows=None, generic=False, force_fp64=False, minhash=0):
    idx = _index(cfg)
    try:
        idx.set_hash_kernel(generic)
        idx.set_cws_fp64(force_fp64)
        idx.set_minhash(minhash)
        g = gpu_hash(idx, x)
        r = oracle.filter_r(cfg["seed"], cfg["W"])
        assert np.array_equal(idx.filter, r)
        KL = cfg["K"] * cfg["L"]
        for i in (range(len(x)) if rows is None else rows):
            bits = oracle.sketch(x[i], r, cfg["delta"])
            assert np.array_equal(_unpack_bits(g["bits"][i], g["nb"]), bits), f"bits of row {i}"
            sid, scnt = oracle.shingle(bits, cfg["n"])
            k = int(g["nnz"][i])
            assert k == len(sid), f"nnz of row {i}"
            assert np.array_equal(g["ids"][i, :k], sid) and np.array_equal(g["cnt"][i, :k], scnt), f"shingles {i}"
            ks, ts = (oracle.doph if minhash else oracle.cws)(cfg["seed"], KL, sid, scnt)
            assert np.array_equal(g["ks"][i], ks), f"kstar of row {i}"
            assert np.array_equal(g["ts"][i], ts), f"tstar of row {i}"
            for l in range(cfg["L"]):
                assert int(g["keys"][l, i]) == oracle.bucket_key(cfg["seed"], l, cfg["K"], ks, ts), f"key {l},{i}"
        return idx.stats()
    finally:
        idx.close()


# ------------------------------------------------------------ hashing stages

KERNELS = pytest.mark.parametrize("generic", [False, True], ids=["specialised", "generic"])


@KERNELS
def test_hash_parity_tiny_config(generic):
    x = synth.random_walk(400, 128, seed=0)
    check_hash_parity(CFG1, x, generic=generic)


@KERNELS
def test_hash_parity_scale_config(generic):
    x = synth.random_walk(250, 512, seed=3)
    check_hash_parity(CFG2, x, generic=generic)


@KERNELS
def test_hash_parity_ecg_config(generic):
    x = synth.ecg_like(120, 1024, seed=5)
    check_hash_parity(CFG3, x, generic=generic)


@KERNELS
@pytest.mark.parametrize("m", [128, 256, 512, 1024, 2048])
def test_hash_parity_batched_lengths(m, generic):
    # per-length sub-indexes of the batched workload: W = m/8, delta 3, n 15, K 4, L 25
    cfg = dict(W=m // 8, delta=3, n=15, K=4, L=25, band=0.05, seed=0)
    x = synth.random_walk(60 if m >= 1024 else 120, m, seed=m)
    check_hash_parity(cfg, x, generic=generic)


@KERNELS
def test_hash_parity_ecg_like_scale_params(generic):
    # repeated-shingle heavy input (periodic beats): exercises the FP32 interval track
    x = synth.ecg_like(200, 512, seed=9)
    check_hash_parity(CFG2, x, generic=generic)


def test_hash_parity_ragged_and_minimum_length():
    # m = W + (n-1)*delta gives exactly one shingle; odd lengths exercise unaligned rows
    cfg = dict(W=16, delta=3, n=6, K=3, L=5, band=0.1, seed=7)
    for m in [16 + 5 * 3, 16 + 5 * 3 + 1, 67, 101]:
        x = synth.random_walk(70, m, seed=m)
        check_hash_parity(cfg, x)


@KERNELS
def test_sketch_fp64_path_on_near_zero_projections(generic):
    """Windows made orthogonal to r have |r.x| at rounding level: the FP64 path decides them."""
    cfg = dict(CFG1)
    r = oracle.filter_r(cfg["seed"], cfg["W"]).astype(np.float64)
    rng = np.random.default_rng(11)
    rows = []
    for t in range(64):
        x = rng.standard_normal(128)
        for start in range(0, 128 - 32 + 1, 33):  # windows at multiples of delta that do not overlap
            start -= start % 3
            v = x[start:start + 32]
            x[start:start + 32] = v - (r @ v) / (r @ r) * r
        rows.append(x)
    rows.append(np.zeros(128))            # every dot product exactly 0 -> bit 1
    rows.append(np.full(128, 1e-3))
    x = np.array(rows, np.float32)
    stats = check_hash_parity(cfg, x, generic=generic)
    assert stats["sketch_fp64"] > 0


@KERNELS
def test_cws_many_series_exact(generic):
    # enough series that near ties in FP32 occur; every hash must still match
    x = synth.random_walk(3000, 512, seed=21)
    check_hash_parity(CFG2, x, rows=range(0, 3000, 11), generic=generic)


@KERNELS
@pytest.mark.parametrize("data", ["random_walk", "ecg_like"])
def test_cws_fp64_recomputation_is_exact(generic, data):
    """Every minhash decided by the FP64 recomputation (the path taken on near ties)."""
    x = synth.random_walk(150, 512, seed=5) if data == "random_walk" else synth.ecg_like(150, 512, seed=6)
    stats = check_hash_parity(CFG2, x, generic=generic, force_fp64=True)
    assert stats["cws_fp64"] == 150 * CFG2["K"] * CFG2["L"]


# ------------------------------------------------------------- DTW, LB_Keogh

def _pairs(nA, nB, npairs, seed):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, nA, size=npairs).astype(np.int64)
    b = rng.integers(0, nB, size=npairs).astype(np.int64)
    return a, b


@pytest.mark.parametrize("m,rb", [(128, 6), (512, 25), (1024, 102), (256, 12), (2048, 102), (1024, 51),
                                  (64, 63), (100, 0), (37, 5), (200, 30), (300, 140)])
def test_dtw_parity(m, rb):
    b = _binding()
    A = synth.random_walk(12, m, seed=m + 1)
    B = synth.random_walk(40, m, seed=m + 2)
    ai, bi = _pairs(len(A), len(B), 60, seed=m)
    out = torch.zeros(len(ai), dtype=torch.float32, device="cuda")
    b.ssh_dtw_device(torch.from_numpy(A).cuda(), torch.from_numpy(ai).cuda(), torch.from_numpy(B).cuda(),
                     torch.from_numpy(bi).cuda(), m, rb, out)
    got = out.cpu().numpy()
    want = np.array([oracle.dtw(A[i], B[j], rb) for i, j in zip(ai, bi)])
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=0)


TILINGS = [(8, 0), (14, 0), (26, 0)]


@pytest.mark.parametrize("m,rb", [(128, 6), (512, 25), (1024, 102), (2048, 102), (1024, 51), (64, 63),
                                  (100, 0), (37, 5), (300, 140), (13, 1)])
def test_dtw_every_tiling_matches_the_oracle_and_each_other(m, rb):
    """Every compiled tiling (slots per lane S, kernel variant) computes each cell from the same
    three values with the same operations, so all give identical distances, within 1e-5 of the
    oracle; a tiling that needs more than 32 lanes per pair is refused."""
    b = _binding()
    A = synth.random_walk(6, m, seed=m + 3)
    B = synth.random_walk(30, m, seed=m + 4)
    ai, bi = _pairs(len(A), len(B), 90, seed=m + 5)
    want = np.array([oracle.dtw(A[i], B[j], rb) for i, j in zip(ai, bi)])
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dai, dbi = torch.from_numpy(ai).cuda(), torch.from_numpy(bi).cuda()
    results = {}
    for S, variant in TILINGS:
        out = torch.full((len(ai),), -1.0, dtype=torch.float32, device="cuda")
        if (2 * rb + 2 + S - 1) // S > 32:
            with pytest.raises(b.SSHError) as e:
                b.ssh_dtw_device_tiled(dA, dai, dB, dbi, m, rb, S, variant, out)
            assert e.value.status == b.SSH_ENOTSUP
            continue
        b.ssh_dtw_device_tiled(dA, dai, dB, dbi, m, rb, S, variant, out)
        results[(S, variant)] = out.cpu().numpy()
        np.testing.assert_allclose(results[(S, variant)], want, rtol=RTOL, atol=0, err_msg=str((S, variant)))
    first = next(iter(results.values()))
    for key, got in results.items():
        assert np.array_equal(got, first), key
    for S, variant in ((10, 0), (14, 1)):  # not compiled
        with pytest.raises(b.SSHError) as e:
            b.ssh_dtw_device_tiled(dA, dai, dB, dbi, m, rb, S, variant, torch.empty(len(ai), device="cuda"))
        assert e.value.status == b.SSH_ENOTSUP


def test_dtw_identity_and_band0():
    b = _binding()
    m = 512
    A = synth.random_walk(8, m, seed=9)
    idx = torch.arange(8, dtype=torch.int64, device="cuda")
    out = torch.zeros(8, dtype=torch.float32, device="cuda")
    d_a = torch.from_numpy(A).cuda()
    b.ssh_dtw_device(d_a, idx, d_a, idx, m, 25, out)
    assert (out.cpu().numpy() == 0).all()
    rev = torch.flip(idx, [0]).contiguous()
    b.ssh_dtw_device(d_a, idx, d_a, rev, m, 0, out)
    want = ((A.astype(np.float64) - A[::-1].astype(np.float64)) ** 2).sum(axis=1)
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=RTOL)


@pytest.mark.parametrize("m,rb", [(128, 6), (512, 25), (1024, 102), (37, 5)])
def test_lb_keogh_parity(m, rb):
    b = _binding()
    A = synth.random_walk(10, m, seed=m + 5)
    B = synth.random_walk(30, m, seed=m + 6)
    ai, bi = _pairs(len(A), len(B), 50, seed=m + 1)
    out = torch.zeros(len(ai), dtype=torch.float32, device="cuda")
    b.ssh_lb_keogh_device(torch.from_numpy(A).cuda(), torch.from_numpy(ai).cuda(), torch.from_numpy(B).cuda(),
                          torch.from_numpy(bi).cuda(), m, rb, out)
    got = out.cpu().numpy()
    want = np.array([oracle.lb_keogh(A[i], B[j], rb) for i, j in zip(ai, bi)])
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=1e-6)


@pytest.mark.parametrize("m,rb", [(128, 6), (512, 25), (1024, 102), (37, 5), (64, 0), (50, 49)])
def test_lb_bound_kinds_parity(m, rb):
    """The cascade's bounds through ssh_lb_bound_device against the oracle: kind 0 LB_Keogh,
    1 LB_Keogh with the LB_Kim endpoint costs, 2 the reversed LB_Keogh (candidate envelope)."""
    b = _binding()
    A = synth.random_walk(10, m, seed=m + 15)
    B = synth.random_walk(30, m, seed=m + 16)
    ai, bi = _pairs(len(A), len(B), 50, seed=m + 2)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dai, dbi = torch.from_numpy(ai).cuda(), torch.from_numpy(bi).cuda()
    refs = (oracle.lb_keogh, oracle.lb_keogh_kim, oracle.lb_keogh_rev)
    for kind, ref in enumerate(refs):
        out = torch.full((len(ai),), -1.0, dtype=torch.float32, device="cuda")
        b.ssh_lb_bound_device(dA, dai, dB, dbi, m, rb, kind, out)
        got = out.cpu().numpy()
        want = np.array([ref(A[i], B[j], rb) for i, j in zip(ai, bi)])
        np.testing.assert_allclose(got, want, rtol=RTOL, atol=1e-6, err_msg=f"kind {kind}")
    with pytest.raises(b.SSHError) as e:
        b.ssh_lb_bound_device(dA, dai, dB, dbi, m, rb, 3, out)
    assert e.value.status == b.SSH_EINVAL


@pytest.mark.parametrize("exact", [False, True])
def test_lb_cascade_changes_no_result(exact):
    """The cascade (LB_Kim endpoints, reversed LB_Keogh) only skips DTWs that cannot reach the
    top-k: ids and distances are identical with it on and off, and with pruning off."""
    cfg = CFG2
    db = synth.random_walk(3000, 512, seed=21)
    qs, _ = synth.perturbed_queries(db, 12, seed=22)
    res = {}
    with _index(cfg) as idx:
        idx.add(db)
        idx.set_exact_scan(exact)
        for name, prune, cascade in (("off", False, 0), ("lb", True, 0), ("kim", True, 1), ("cascade", True, 2)):
            idx.set_lb_prune(prune)
            idx.set_lb_cascade(cascade)
            idx.reset_stats()
            ids, d = idx.query(qs, 10)
            res[name] = (ids, d, idx.stats())
    for name in ("lb", "kim", "cascade"):
        assert np.array_equal(res[name][0], res["off"][0]) and np.array_equal(res[name][1], res["off"][1]), name
    st_lb, st_c = res["lb"][2], res["cascade"][2]
    assert st_lb["lb2_pruned"] == 0 and res["kim"][2]["lb2_pruned"] == 0
    assert st_c["dtw_computed"] <= res["kim"][2]["dtw_computed"]  # the reversed bound only removes survivors
    if exact:
        assert st_c["lb2_pruned"] > 0 and st_c["dtw_computed"] < res["kim"][2]["dtw_computed"]
    assert st_c["lb_pruned"] == st_c["candidates"] - st_c["dtw_computed"]


# ------------------------------------------------------------- end to end

def assert_topk_match(q, ids_g, d_g, ids_o, d_o, db_by_id, rb):
    k = len(ids_o)
    real = ids_o >= 0
    assert np.array_equal(ids_g >= 0, real)
    # the sorted distance lists agree
    np.testing.assert_allclose(d_g[real], d_o[real], rtol=RTOL, atol=0)
    for t in np.nonzero(real)[0]:
        if ids_g[t] != ids_o[t]:
            # a near tie: the returned id's exact distance must equal the oracle's t-th distance
            dd = oracle.dtw(q, db_by_id(int(ids_g[t])), rb)
            assert abs(dd - d_o[t]) <= RTOL * d_o[t], (t, ids_g[t], ids_o[t], dd, d_o[t])
    assert len(set(ids_g[real].tolist())) == int(real.sum())


@pytest.mark.parametrize("prune", [True, False])
def test_end_to_end_tiny_config(prune):
    cfg = CFG1
    db = synth.random_walk(1000, 128, seed=0)
    qs, _ = synth.perturbed_queries(db, 10, seed=1)
    ref = oracle.OracleIndex(**cfg)
    ref.add(db)
    with _index(cfg) as idx:
        idx.set_lb_prune(prune)
        assert idx.add(db) == 0
        assert len(idx) == 1000
        ids, d = idx.query(qs, 5)
        st = idx.stats()
    rb = oracle.band_radius(cfg["band"], 128)
    for i, q in enumerate(qs):
        oi, od = ref.query(q, 5)
        assert_topk_match(q, ids[i], d[i], oi, od, lambda j: db[j], rb)
    assert st["queries"] == 10
    assert st["candidates"] == sum(len(ref.candidates(q)) for q in qs)


def test_end_to_end_device_path_and_borrow():
    cfg = CFG1
    db = synth.random_walk(600, 128, seed=4)
    qs, _ = synth.perturbed_queries(db, 8, seed=5)
    ref = oracle.OracleIndex(**cfg)
    ref.add(db)
    d_db = torch.from_numpy(db).cuda()
    with _index(cfg) as idx:
        idx.add_device(d_db, borrow=True)
        d_q = torch.from_numpy(qs).cuda()
        ids = torch.empty((8, 7), dtype=torch.int64, device="cuda")
        dd = torch.empty((8, 7), dtype=torch.float32, device="cuda")
        idx.query_device(d_q, 7, ids, dd)
        torch.cuda.synchronize()
        ids, dd = ids.cpu().numpy(), dd.cpu().numpy()
    rb = oracle.band_radius(cfg["band"], 128)
    for i, q in enumerate(qs):
        oi, od = ref.query(q, 7)
        assert_topk_match(q, ids[i], dd[i], oi, od, lambda j: db[j], rb)


def test_end_to_end_mixed_lengths_and_incremental_adds():
    cfg = dict(W=16, delta=2, n=8, K=3, L=12, band=0.1, seed=3)
    lens = [64, 96, 128]
    parts = {m: synth.random_walk(150, m, seed=m) for m in lens}
    ref = oracle.OracleIndex(**cfg)
    with _index(cfg) as idx:
        # interleave lengths inside one call (ragged), then a second call
        order = [(m, i) for i in range(100) for m in lens]
        series = [parts[m][i] for m, i in order]
        ref.add(series)
        first = idx.add(np.concatenate(series), np.array([len(s) for s in series], np.int32))
        assert first == 0
        more = [parts[m][i] for m in lens for i in range(100, 150)]
        ref.add(more)
        first = idx.add(np.concatenate(more), np.array([len(s) for s in more], np.int32))
        assert first == len(series)
        allrows = series + more
        qs = []
        for m in lens:
            q, _ = synth.perturbed_queries(parts[m], 4, seed=m + 1)
            qs.extend(list(q))
        qlens = np.array([len(q) for q in qs], np.int32)
        ids, d = idx.query(np.concatenate(qs), 6, lengths=qlens)
    for i, q in enumerate(qs):
        oi, od = ref.query(q, 6)
        rb = oracle.band_radius(cfg["band"], len(q))
        assert_topk_match(q, ids[i], d[i], oi, od, lambda j: allrows[j], rb)


def test_scale_config_end_to_end_small_db():
    cfg = CFG2
    db = synth.random_walk(400, 512, seed=2)
    qs, _ = synth.perturbed_queries(db, 5, seed=3)
    ref = oracle.OracleIndex(**cfg)
    ref.add(db)
    with _index(cfg) as idx:
        idx.add(db)
        ids, d = idx.query(qs, 10)
    rb = oracle.band_radius(cfg["band"], 512)
    for i, q in enumerate(qs):
        oi, od = ref.query(q, 10)
        assert_topk_match(q, ids[i], d[i], oi, od, lambda j: db[j], rb)


def test_fewer_candidates_than_k_fill_with_minus_one():
    cfg = CFG1
    db = synth.random_walk(50, 128, seed=8)
    with _index(cfg) as idx:
        idx.add(db)
        ids, d = idx.query(db[:3], 64)
    ref = oracle.OracleIndex(**cfg)
    ref.add(db)
    for i in range(3):
        n = len(ref.candidates(db[i]))
        assert (ids[i, n:] == -1).all() and np.isinf(d[i, n:]).all()
        assert ids[i, 0] == i and d[i, 0] == 0.0


def test_errors_are_status_codes():
    b = _binding()
    with b.SSHIndex(32, 3, 17, 4, 16, 0.05, 0) as ix17:  # n up to 32: draws computed on the fly
        assert ix17.n == 17
        with pytest.raises(b.SSHError) as e:
            ix17.set_minhash(1)  # the one-permutation option tabulates n <= 16 only
        assert e.value.status == b.SSH_ENOTSUP
    for bad_n in (0, 33):
        with pytest.raises(b.SSHError) as e:
            b.SSHIndex(32, 3, bad_n, 4, 16, 0.05, 0)
        assert e.value.status == b.SSH_EINVAL
    with _index(CFG1) as idx:
        with pytest.raises(b.SSHError) as e:
            idx.add(np.zeros((2, 52), np.float32))  # shorter than W + (n-1) delta = 53
        assert e.value.status == b.SSH_ELENGTH
        assert len(idx) == 0
        idx.add(synth.random_walk(10, 128, seed=0))
        with pytest.raises(b.SSHError) as e:
            idx.query(np.zeros((1, 100), np.float32), 3)
        assert e.value.status == b.SSH_ELENGTH
        with pytest.raises(b.SSHError) as e:
            idx.query(np.zeros((1, 128), np.float32), 0)
        assert e.value.status == b.SSH_EINVAL
        idx.clear()
        assert len(idx) == 0
        idx.add(synth.random_walk(10, 128, seed=1))
        ids, _ = idx.query(synth.random_walk(10, 128, seed=1)[:1], 1)
        assert ids[0, 0] == 0


def test_group_query_routes_mixed_lengths_to_per_length_indexes():
    """Per-length filter W = m/8 (one index per length); queries of mixed lengths in one call."""
    b = _binding()
    lens = [128, 256, 512]
    dbs = {m: synth.random_walk(150, m, seed=m + 3) for m in lens}
    idxs, refs = [], {}
    try:
        for m in lens:
            cfg = dict(W=m // 8, delta=3, n=15, K=4, L=25, band=0.05, seed=0)
            ix = _index(cfg)
            ix.add(dbs[m])
            idxs.append(ix)
            refs[m] = oracle.OracleIndex(**cfg)
            refs[m].add(dbs[m])
        qs, qlens = [], []
        rng = np.random.default_rng(0)
        for t in range(12):
            m = lens[int(rng.integers(0, 3))]
            q, _ = synth.perturbed_queries(dbs[m], 1, seed=100 + t)
            qs.append(q[0])
            qlens.append(m)
        k = 5
        d_q = torch.from_numpy(np.concatenate(qs)).cuda()
        ids = torch.empty((len(qs), k), dtype=torch.int64, device="cuda")
        dd = torch.empty((len(qs), k), dtype=torch.float32, device="cuda")
        which = torch.full((len(qs),), -1, dtype=torch.int32, device="cuda")
        b.ssh_group_query_device([ix.handle for ix in idxs], d_q, np.array(qlens, np.int32), k, ids, dd, which)
        torch.cuda.synchronize()
        ids, dd, which = ids.cpu().numpy(), dd.cpu().numpy(), which.cpu().numpy()
        for i, (q, m) in enumerate(zip(qs, qlens)):
            assert which[i] == lens.index(m)
            oi, od = refs[m].query(q, k)
            assert_topk_match(q, ids[i], dd[i], oi, od, lambda j: dbs[m][j], oracle.band_radius(0.05, m))
        bad_ids = torch.empty((1, k), dtype=torch.int64, device="cuda")
        bad_d = torch.empty((1, k), dtype=torch.float32, device="cuda")
        with pytest.raises(b.SSHError) as e:
            b.ssh_group_query_device([ix.handle for ix in idxs], torch.zeros((1, 100), device="cuda"),
                                     np.array([100], np.int32), k, bad_ids, bad_d)
        assert e.value.status == b.SSH_ELENGTH
    finally:
        for ix in idxs:
            ix.close()


# ------------------------------------------------------------- batch plans

def _batch_setup(lens=(128, 256, 512), n=150):
    dbs = {m: synth.random_walk(n, m, seed=m + 5) for m in lens}
    cfgs = {m: dict(W=m // 8, delta=3, n=15, K=4, L=25, band=0.05, seed=0) for m in lens}
    idxs = []
    for m in lens:
        ix = _index(cfgs[m])
        ix.add(dbs[m])
        idxs.append(ix)
    return dbs, cfgs, idxs


def _mixed_queries(dbs, lens, nq, seed):
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
    b = _binding()
    d_q = torch.from_numpy(np.concatenate(qs)).cuda()
    ids = torch.empty((len(qs), k), dtype=torch.int64, device="cuda")
    dd = torch.empty((len(qs), k), dtype=torch.float32, device="cuda")
    which = torch.full((len(qs),), -1, dtype=torch.int32, device="cuda")
    b.ssh_group_query_device([ix.handle for ix in idxs], d_q, qlens, k, ids, dd, which)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dd.cpu().numpy(), which.cpu().numpy()


def test_batch_plan_matches_oracle_and_replays_graph():
    """Mixed-length batches through one plan: the first runs directly, later ones replay the captured graph."""
    b = _binding()
    lens = (128, 256, 512)
    dbs, cfgs, idxs = _batch_setup(lens)
    try:
        refs = {}
        for m in lens:
            refs[m] = oracle.OracleIndex(**cfgs[m])
            refs[m].add(dbs[m])
        k = 5
        with b.SSHBatch(idxs, max_queries=64, k=k) as bt:
            for rep in range(3):  # rep 0 runs directly, reps 1-2 replay the graph
                qs, qlens = _mixed_queries(dbs, lens, 20 + 7 * rep, seed=rep + 1)
                ids, dd, which = _run_batch(bt, qs, qlens, k)
                for i, (q, m) in enumerate(zip(qs, qlens)):
                    assert which[i] == lens.index(m)
                    oi, od = refs[m].query(q, k)
                    assert_topk_match(q, ids[i], dd[i], oi, od, lambda j: dbs[m][j], oracle.band_radius(0.05, m))
                # the same kernels answer the per-length group path: identical results
                gi, gd, gw = _run_group(idxs, qs, qlens, k)
                assert np.array_equal(ids, gi) and np.array_equal(dd, gd) and np.array_equal(which, gw)
            st = bt.stats()
            assert st["graph_kernels"] > 10
            assert st["pairs"] > 0 and 0 < st["dtw"] <= st["pairs"]
    finally:
        for ix in idxs:
            ix.close()


def test_batch_plan_grows_pair_buffers_and_follows_adds():
    b = _binding()
    lens = (128, 256)
    dbs, cfgs, idxs = _batch_setup(lens, n=200)
    try:
        k = 4
        with b.SSHBatch(idxs, max_queries=16, k=k, max_pairs=8) as bt:
            qs, qlens = _mixed_queries(dbs, lens, 12, seed=9)
            ids, dd, which = _run_batch(bt, qs, qlens, k)
            gi, gd, gw = _run_group(idxs, qs, qlens, k)
            assert np.array_equal(ids, gi) and np.array_equal(dd, gd)
            assert bt.stats()["pair_capacity"] > 8  # grown past the first capacity
            # an add to one index: the next batch sees the new rows (the plan is rebuilt)
            more = synth.random_walk(50, 256, seed=77)
            first = idxs[1].add(more)
            q = more[3:4] + np.float32(0.0)
            ids2, dd2, _ = _run_batch(bt, [q[0]], np.array([256], np.int32), k)
            assert ids2[0, 0] == first + 3 and dd2[0, 0] == 0.0
            # errors
            d_q = torch.zeros((17, 128), device="cuda")
            bad_ids = torch.empty((17, k), dtype=torch.int64, device="cuda")
            bad_d = torch.empty((17, k), dtype=torch.float32, device="cuda")
            with pytest.raises(b.SSHError) as e:
                bt.query(d_q, np.full(17, 128, np.int32), bad_ids, bad_d)
            assert e.value.status == b.SSH_EINVAL
            with pytest.raises(b.SSHError) as e:
                bt.query(d_q[:1, :100].contiguous(), np.array([100], np.int32), bad_ids[:1], bad_d[:1])
            assert e.value.status == b.SSH_ELENGTH
    finally:
        for ix in idxs:
            ix.close()


def test_small_adds_go_to_delta_tables_then_merge():
    """Adds of up to an eighth of the binned rows go to the delta tables; results and candidate
    sets must equal the oracle's after each add, and after the merge that a large add triggers."""
    cfg = CFG1
    rng_db = synth.random_walk(800, 128, seed=41)
    ref = oracle.OracleIndex(**cfg)
    with _index(cfg) as idx:
        chunks = [(0, 400), (400, 430), (430, 470), (470, 800)]  # full, delta, delta, merge
        for a, b in chunks:
            assert idx.add(rng_db[a:b]) == a
            ref.add(rng_db[a:b])
            qs, _ = synth.perturbed_queries(rng_db[:b], 6, seed=b)
            qs[0] = rng_db[b - 1]  # an exact copy of the newest row: its own top-1
            idx.reset_stats()
            ids, d = idx.query(qs, 5)
            st = idx.stats()
            assert st["candidates"] == sum(len(ref.candidates(q)) for q in qs)
            assert ids[0, 0] == b - 1 and d[0, 0] == 0.0
            rb = oracle.band_radius(cfg["band"], 128)
            for i, q in enumerate(qs):
                oi, od = ref.query(q, 5)
                assert_topk_match(q, ids[i], d[i], oi, od, lambda j: rng_db[j], rb)


@pytest.mark.parametrize("prune", [True, False])
def test_exact_scan_equals_brute_force_topk(prune):
    """SSH_OPT_EXACT_SCAN: every stored series is a candidate; the top-k must be the oracle's
    brute-force banded-DTW top-k (LB_Keogh pruning and early abandoning change nothing)."""
    cfg = CFG1
    db = synth.random_walk(700, 128, seed=13)
    qs, _ = synth.perturbed_queries(db, 7, seed=14)
    ref = oracle.OracleIndex(**cfg)
    ref.add(db)
    with _index(cfg) as idx:
        idx.add(db)
        idx.set_exact_scan(True)
        idx.set_lb_prune(prune)
        idx.reset_stats()
        ids, d = idx.query(qs, 6)
        st = idx.stats()
    assert st["candidates"] == 7 * 700
    if prune:
        assert 0 < st["dtw_computed"] < st["candidates"]
    rb = oracle.band_radius(cfg["band"], 128)
    for i, q in enumerate(qs):
        oi, od = ref.exact_topk(q, 6)
        assert_topk_match(q, ids[i], d[i], oi, od, lambda j: db[j], rb)


def _check_large_table_candidates(db, src):
    """Every query's candidate count must equal the size of the union over tables of the rows
    whose bucket key equals the query's (computed here from the keys ssh_hash_device returns),
    and the stored series db[src[:3]] must find themselves at distance 0."""
    b = _binding()
    N, m = db.shape
    with _index(CFG1) as idx:
        idx.add(db)
        L = idx.L
        d_db = torch.from_numpy(db).cuda()
        keys = torch.zeros((L, N), dtype=torch.int64, device="cuda")
        b.ssh_hash_device(idx.handle, d_db, m, N, d_keys=keys)
        torch.cuda.synchronize()
        keys = keys.cpu().numpy()
        qs = np.concatenate([db[src[:3]], synth.perturbed_queries(db, 3, seed=9)[0]])
        qkeys = torch.zeros((L, len(qs)), dtype=torch.int64, device="cuda")
        b.ssh_hash_device(idx.handle, torch.from_numpy(qs).cuda(), m, len(qs), d_keys=qkeys)
        torch.cuda.synchronize()
        qkeys = qkeys.cpu().numpy()
        for i in range(len(qs)):
            want = np.zeros(N, bool)
            for l in range(L):
                want |= keys[l] == qkeys[l, i]
            idx.reset_stats()
            ids, d = idx.query(qs[i:i + 1], 3)
            assert idx.stats()["candidates"] == int(want.sum())
            if i < 3:
                assert d[0, 0] == 0.0 and np.array_equal(db[ids[0, 0]], db[src[i]])


def test_large_tables_two_pass_partition_candidates():
    """Tables of >= 65,536 rows are binned in two passes (buckets of the top key bits, then the
    bins inside each bucket, placed in shared memory)."""
    db = synth.random_walk(70_000, 128, seed=71)
    _check_large_table_candidates(db, np.random.default_rng(5).integers(0, len(db), 6))


def test_large_tables_with_an_oversized_bucket():
    """5,000 copies of one series share its bucket key in every table, so that bucket holds more
    entries than a block places in shared memory and the second pass takes its tile-by-tile path;
    the candidate sets must still be the exact key matches."""
    db = synth.random_walk(70_000, 128, seed=72)
    db[10_000:15_000] = db[3]
    _check_large_table_candidates(db, np.array([3, 12_345, 40_000, 0, 0, 0]))


def test_read_probe_runs_and_rejects_bad_sizes():
    """The measurement helper reads a buffer and refuses sizes it cannot read in 16-byte words."""
    from paper_1610_07328_gb300 import binding
    x = torch.ones(1 << 20, dtype=torch.float32, device="cuda")
    binding.ssh_read_device(x, 4)
    torch.cuda.synchronize()
    assert float(x.sum()) == float(1 << 20)  # only read
    with pytest.raises(binding.SSHError) as e:
        binding.ssh_read_device(x[:3], 1)
    assert e.value.status == binding.SSH_EINVAL
    with pytest.raises(binding.SSHError):
        binding.ssh_read_device(x, 0)


# the paper's Random Walk parameters (Sec. 5.1: W = 30, delta = 5, n = 15, one hash per table, 20 tables)
CFG_RW = dict(W=30, delta=5, n=15, K=1, L=20, band=0.05, seed=0)


@pytest.mark.parametrize("cfg,step,generic", [(CFG1, 1, False), (CFG1, 7, False), (CFG1, 1, True),
                                              (CFG1, 40, False), (CFG_RW, 1, False), (CFG_RW, 3, True)],
                         ids=["cfg1-step1", "cfg1-step7", "cfg1-step1-rows", "cfg1-step40-rows", "rw-step1",
                              "rw-step3-rows"])
def test_windows_of_one_stream_equal_the_oracle_over_the_same_windows(cfg, step, generic):
    """Sec. 5.1's workload: every length-t window of one long series (offsets 0, step, ...),
    added without copies; queries must return the oracle's top-k over the same windows added
    one by one as series, and a window used as the query finds itself at distance 0. Steps
    below N_B take the shared-stream sketch; larger steps and the generic-kernel knob hash the
    windows as rows."""
    b = _binding()
    stream = synth.random_walk(1, 2400, seed=31)[0]
    t = 128
    starts = list(range(0, len(stream) - t + 1, step))
    windows = np.stack([stream[p:p + t] for p in starts])
    d_stream = torch.from_numpy(stream).cuda()
    extra = synth.random_walk(3, t, seed=33)  # ids of the windows follow these
    ref = oracle.OracleIndex(**cfg)
    ref.add(extra)
    ref.add(windows)
    rows = np.concatenate([extra, windows])
    qs, _ = synth.perturbed_queries(windows, 5, seed=32)
    qs = np.concatenate([qs, windows[len(windows) // 3][None]])
    with _index(cfg) as idx:
        idx.set_hash_kernel(generic)
        idx.add(extra)
        first = idx.add_windows_device(d_stream, t, step)
        assert first == 3 and len(idx) == 3 + len(starts)
        ids, d = idx.query(qs, 5)
        with pytest.raises(b.SSHError) as e:
            idx.add_windows_device(d_stream, t, 0)
        assert e.value.status == b.SSH_EINVAL
        with pytest.raises(b.SSHError) as e:
            idx.add_windows_device(d_stream[:100], t, 1)
        assert e.value.status == b.SSH_EINVAL
        with pytest.raises(b.SSHError) as e:
            idx.add_windows_device(d_stream, 40, 1)  # shorter than W + (n-1) delta (53 or 100)
        assert e.value.status == b.SSH_ELENGTH
        assert len(idx) == 3 + len(starts)
    rb = oracle.band_radius(cfg["band"], t)
    for i, q in enumerate(qs):
        oi, od = ref.query(q, 5)
        assert_topk_match(q, ids[i], d[i], oi, od, lambda j: rows[j], rb)
    assert ids[-1][0] == 3 + len(windows) // 3 and d[-1][0] == 0.0


@pytest.mark.parametrize("m,K,L", [(128, 8, 10), (512, 12, 20), (77, 4, 6)])
def test_srp_baseline_matches_the_oracle(m, K, L):
    """The SRP baseline (ssh_create_srp): every query's candidate set (rows sharing a table key)
    has the oracle's size, and the top-k equals the oracle's over it."""
    b = _binding()
    db = synth.random_walk(500, m, seed=m + 40)
    qs, _ = synth.perturbed_queries(db, 6, seed=m + 41)
    ref = oracle.OracleIndex(1, 1, 1, K, L, 0.05, 3, family="srp")
    ref.add(db)
    idx = b.SSHIndex.srp(K, L, 0.05, 3)
    try:
        idx.add(db)
        idx.reset_stats()
        ids, d = idx.query(qs, 5)
        st = idx.stats()
    finally:
        idx.close()
    assert st["candidates"] == sum(len(ref.candidates(q)) for q in qs)
    rb = oracle.band_radius(0.05, m)
    for i, q in enumerate(qs):
        oi, od = ref.query(q, 5)
        assert_topk_match(q, ids[i], d[i], oi, od, lambda j: db[j], rb)


def test_srp_near_zero_projections_take_the_fp64_path():
    """Series made orthogonal to projections 0..3 (up to FP32 rounding) put those products at
    rounding level: the FP64 recomputation decides them, and the candidate sets stay exact."""
    b = _binding()
    m, K, L = 96, 4, 3
    R = np.stack([oracle.srp_projection(9, m, j) for j in range(K * L)]).astype(np.float64)
    rng = np.random.default_rng(42)
    rows = []
    for t in range(200):
        x = rng.standard_normal(m)
        for j in range(4):
            x = x - (R[j] @ x) / (R[j] @ R[j]) * R[j]
        rows.append(x)
    db = np.array(rows, np.float32)
    ref = oracle.OracleIndex(1, 1, 1, K, L, 0.05, 9, family="srp")
    ref.add(db)
    idx = b.SSHIndex.srp(K, L, 0.05, 9)
    try:
        idx.add(db)
        ids, d = idx.query(db[:8], 3)
        st = idx.stats()
        idx.reset_stats()
        idx.query(db[8:16], 3)
        st2 = idx.stats()
        with pytest.raises(b.SSHError) as e:
            b.SSHBatch([idx], max_queries=4, k=3)
        assert e.value.status == b.SSH_ENOTSUP
    finally:
        idx.close()
    assert st["sketch_fp64"] > 0
    assert st2["candidates"] == sum(len(ref.candidates(q)) for q in db[8:16])
    rb = oracle.band_radius(0.05, m)
    for i in range(8):
        oi, od = ref.query(db[i], 3)
        assert_topk_match(db[i], ids[i], d[i], oi, od, lambda j: db[j], rb)


@pytest.mark.parametrize("cfg,m", [(CFG1, 128), (CFG2, 512), (CFG3, 1024)])
def test_doph_minhash_parity(cfg, m):
    """SSH_OPT_MINHASH 1: the densified one-permutation minhash of every series equals the
    oracle's, (k*, t*) and bucket keys bit for bit (random walks and repeated-shingle-heavy
    ECG-like beats)."""
    x = synth.random_walk(150, m, seed=m + 50) if m != 1024 else synth.ecg_like(80, m, seed=51)
    check_hash_parity(cfg, x, minhash=1)


def test_doph_end_to_end_and_option_rules():
    b = _binding()
    cfg = CFG1
    db = synth.random_walk(800, 128, seed=52)
    qs, _ = synth.perturbed_queries(db, 8, seed=53)
    ref = oracle.OracleIndex(**cfg, family="ssh-doph")
    ref.add(db)
    with _index(cfg) as idx:
        idx.set_minhash(1)
        idx.add(db)
        ids, d = idx.query(qs, 5)
        with pytest.raises(b.SSHError) as e:
            idx.set_minhash(0)  # the stored keys are one-permutation keys
        assert e.value.status == b.SSH_EBUSY
    rb = oracle.band_radius(cfg["band"], 128)
    for i, q in enumerate(qs):
        oi, od = ref.query(q, 5)
        assert_topk_match(q, ids[i], d[i], oi, od, lambda j: db[j], rb)
    with b.SSHIndex(40, 3, 10, 4, 8, 0.05, 0) as idx:  # no compiled sketch shape for W = 40
        idx.set_minhash(1)
        with pytest.raises(b.SSHError) as e:
            idx.add(synth.random_walk(5, 128, seed=54))
        assert e.value.status == b.SSH_ENOTSUP


def test_limits_and_empty_calls():
    """k at its maximum (1024) returns every candidate in order and fills the rest with
    (-1, +inf); k above it is refused; empty adds and empty query batches are no-ops; the
    option values outside their ranges are refused."""
    b = _binding()
    cfg = CFG1
    db = synth.random_walk(300, 128, seed=60)
    with _index(cfg) as idx:
        assert idx.add(np.zeros((0, 128), np.float32)) == 0 and len(idx) == 0
        idx.add(db)
        ids, d = idx.query(db[:2], 1024)
        for i in range(2):
            real = ids[i] >= 0
            n = int(real.sum())
            assert real[:n].all() and not real[n:].any() and np.isinf(d[i, n:]).all()
            pairs = list(zip(d[i, :n].tolist(), ids[i, :n].tolist()))
            assert pairs == sorted(pairs) and ids[i, 0] == i and d[i, 0] == 0.0
        with pytest.raises(b.SSHError) as e:
            idx.query(db[:1], 1025)
        assert e.value.status == b.SSH_EINVAL
        ids0, d0 = idx.query(np.zeros((0, 128), np.float32), 5)
        assert ids0.shape == (0, 5)
        for opt, bad in ((b.SSH_OPT_LB_CASCADE, 3), (b.SSH_OPT_MINHASH, 2), (b.SSH_OPT_HASH_KERNEL, 2)):
            with pytest.raises(b.SSHError) as e:
                b.ssh_set_option(idx.handle, opt, bad)
            assert e.value.status == b.SSH_EINVAL
