"""Plain FP64 CPU oracle for the SSH (Sketch, Shingle & Hash) index and query path.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. It shares no code with the CUDA library (``paper_1610_07328_gb300``):
the arithmetic lives in ``ssh_oracle.c`` (its own Philox, its own key mixing,
FP64 throughout, compiled with ``-ffp-contract=off``) and this module only
marshals numpy arrays and keeps the bucket dictionaries.

Paper: Luo & Shrivastava, "SSH (Sketch, Shingle, & Hash) for Indexing
Massive-Scale Time Series", arXiv:1610.07328.

* Sec. 4.1 (sliding-window sign sketch, worked example Eq. eq1) -> ``sketch``
* Sec. 4.2 (shingles, Eq. set and its worked example) -> ``shingle``
* Sec. 4.3 with Sec. 2.3 Eqs. WJaccardDef / CollProb (weighted minhash, read as
  Ioffe's Improved Consistent Sampling) -> ``cws``
* Algorithm 1 (pre-processing into d = L hash tables, each keyed by K hashes)
  -> ``OracleIndex.add``
* Algorithm 2 (probe every table, union the buckets, top-k by DTW)
  -> ``OracleIndex.query``
* Sec. 2.1 (DTW by dynamic programming) -> ``dtw``; Sec. 3 (LB_Keogh) -> ``lb_keogh``,
  with the UCR suite's cascade the paper prunes with: ``lb_kim_fl``, ``lb_keogh_kim``,
  ``lb_keogh_rev``
* Sec. 5.3 (precision of the top-k against the exact DTW top-k) -> ``recall_at_k``;
  (NDCG of the ranking) -> ``ndcg_at_k``
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ssh_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libssh_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ssh_oracle.c into oracle/_build/libssh_oracle.so with gcc."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                          os.path.getmtime(os.path.join(_HERE, "ssh_oracle.h"))))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        f32p = ctypes.POINTER(ctypes.c_float)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        f64p = ctypes.POINTER(ctypes.c_double)
        sig = {
            "ssh_oracle_philox4x32_10": (None, [u32p, u32p, u32p]),
            "ssh_oracle_uniform": (ctypes.c_double, [ctypes.c_uint32]),
            "ssh_oracle_filter": (None, [ctypes.c_uint64, ctypes.c_int, f32p]),
            "ssh_oracle_srp_projection": (None, [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, f32p]),
            "ssh_oracle_srp_bits": (None, [f32p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, u32p]),
            "ssh_oracle_num_bits": (ctypes.c_int, [ctypes.c_int] * 3),
            "ssh_oracle_sketch": (None, [f32p, ctypes.c_int, f32p, ctypes.c_int, ctypes.c_int, u8p]),
            "ssh_oracle_window_dot": (ctypes.c_double, [f32p, f32p, ctypes.c_int, ctypes.c_int]),
            "ssh_oracle_shingle": (ctypes.c_int, [u8p, ctypes.c_int, ctypes.c_int, u32p, u32p]),
            "ssh_oracle_cws_draw": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, f64p, f64p, f64p]),
            "ssh_oracle_cws_log_a": (ctypes.c_double, [ctypes.c_double] * 3 + [ctypes.c_uint32, f64p]),
            "ssh_oracle_ln": (ctypes.c_double, [ctypes.c_double]),
            "ssh_oracle_cws": (None, [ctypes.c_uint64, ctypes.c_int, u32p, u32p, ctypes.c_int, u32p, u32p]),
            "ssh_oracle_bucket_key": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, u32p, u32p]),
            "ssh_oracle_doph": (None, [ctypes.c_uint64, ctypes.c_int, u32p, u32p, ctypes.c_int, u32p, u32p]),
            "ssh_oracle_hash_series": (ctypes.c_int, [f32p, ctypes.c_int, f32p, ctypes.c_int, ctypes.c_int,
                                                      ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                                      u32p, u32p]),
            "ssh_oracle_band_radius": (ctypes.c_int, [ctypes.c_float, ctypes.c_int]),
            "ssh_oracle_dtw": (ctypes.c_double, [f32p, f32p, ctypes.c_int, ctypes.c_int]),
            "ssh_oracle_lb_keogh": (ctypes.c_double, [f32p, f32p, ctypes.c_int, ctypes.c_int]),
            "ssh_oracle_lb_kim_fl": (ctypes.c_double, [f32p, f32p, ctypes.c_int]),
            "ssh_oracle_lb_keogh_kim": (ctypes.c_double, [f32p, f32p, ctypes.c_int, ctypes.c_int]),
            "ssh_oracle_topk_dtw": (None, [f32p, f32p, i64p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, i64p, f64p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


# ----------------------------------------------------------------- primitives

def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    _load().ssh_oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def uniform(x: int) -> float:
    return _load().ssh_oracle_uniform(int(x) & 0xFFFFFFFF)


def filter_r(seed: int, W: int) -> np.ndarray:
    """Sec. 4.1: the Gaussian filter r (FP32 values)."""
    out = np.zeros(W, dtype=np.float32)
    _load().ssh_oracle_filter(int(seed), int(W), _ptr(out, ctypes.c_float))
    return out


def srp_projection(seed: int, m: int, j: int) -> np.ndarray:
    """The SRP baseline's projection j for series of length m (FP32 normals)."""
    out = np.zeros(m, dtype=np.float32)
    _load().ssh_oracle_srp_projection(int(seed), int(m), int(j), _ptr(out, ctypes.c_float))
    return out


def srp_bits(x, seed: int, nhash: int) -> np.ndarray:
    """Sign random projections (the paper's SRP baseline, Sec. 5.2): bit j = [r_j . x >= 0]."""
    x = _f32(x)
    out = np.zeros(nhash, dtype=np.uint32)
    _load().ssh_oracle_srp_bits(_ptr(x, ctypes.c_float), len(x), int(seed), int(nhash), _ptr(out, ctypes.c_uint32))
    return out


def num_bits(m: int, W: int, delta: int) -> int:
    return _load().ssh_oracle_num_bits(int(m), int(W), int(delta))


def sketch(x, r, delta: int) -> np.ndarray:
    """Sec. 4.1: the sign bits (0/1, uint8) of one series."""
    x = _f32(x)
    r = _f32(r)
    nb = num_bits(len(x), len(r), delta)
    out = np.zeros(max(nb, 1), dtype=np.uint8)
    _load().ssh_oracle_sketch(_ptr(x, ctypes.c_float), len(x), _ptr(r, ctypes.c_float), len(r), int(delta),
                              _ptr(out, ctypes.c_uint8))
    return out[:nb]


def window_dot(x, r, start: int) -> float:
    x = _f32(x)
    r = _f32(r)
    return _load().ssh_oracle_window_dot(_ptr(x, ctypes.c_float), _ptr(r, ctypes.c_float), len(r), int(start))


def shingle(bits, n: int):
    """Sec. 4.2: (ids ascending, counts) of the weighted shingle set."""
    b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8))
    nb = len(b)
    ids = np.zeros(max(nb, 1), dtype=np.uint32)
    counts = np.zeros(max(nb, 1), dtype=np.uint32)
    nnz = _load().ssh_oracle_shingle(_ptr(b, ctypes.c_uint8) if nb else None, nb, int(n),
                                     _ptr(ids, ctypes.c_uint32), _ptr(counts, ctypes.c_uint32))
    return ids[:nnz].copy(), counts[:nnz].copy()


def ln(x: float) -> float:
    """The oracle's natural logarithm (a fixed sequence of FP64 operations; Sec. 4.3 draws)."""
    return _load().ssh_oracle_ln(float(x))


def cws_draw(seed: int, j: int, k: int):
    r, c, beta = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().ssh_oracle_cws_draw(int(seed), int(j), int(k), ctypes.byref(r), ctypes.byref(c), ctypes.byref(beta))
    return r.value, c.value, beta.value


def cws_log_a(r: float, c: float, beta: float, S: int):
    t = ctypes.c_double()
    la = _load().ssh_oracle_cws_log_a(float(r), float(c), float(beta), int(S), ctypes.byref(t))
    return la, t.value


def cws(seed: int, nhash: int, ids, counts):
    """Sec. 4.3: (kstar, tstar) of hash functions 0 .. nhash-1 over a weighted set."""
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32))
    counts = np.ascontiguousarray(np.asarray(counts, dtype=np.uint32))
    ks = np.zeros(nhash, dtype=np.uint32)
    ts = np.zeros(nhash, dtype=np.uint32)
    _load().ssh_oracle_cws(int(seed), int(nhash), _ptr(ids, ctypes.c_uint32), _ptr(counts, ctypes.c_uint32),
                           len(ids), _ptr(ks, ctypes.c_uint32), _ptr(ts, ctypes.c_uint32))
    return ks, ts


def doph(seed: int, nhash: int, ids, counts):
    """Densified one-permutation weighted minhash (a faster variant of Sec. 4.3's weighted
    minhash): (kstar, tstar) = (shingle id, copy index) of hash functions 0 .. nhash-1."""
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32))
    counts = np.ascontiguousarray(np.asarray(counts, dtype=np.uint32))
    ks = np.zeros(nhash, dtype=np.uint32)
    ts = np.zeros(nhash, dtype=np.uint32)
    _load().ssh_oracle_doph(int(seed), int(nhash), _ptr(ids, ctypes.c_uint32), _ptr(counts, ctypes.c_uint32),
                            len(ids), _ptr(ks, ctypes.c_uint32), _ptr(ts, ctypes.c_uint32))
    return ks, ts


def bucket_key(seed: int, l: int, K: int, kstar, tstar) -> int:
    ks = np.ascontiguousarray(np.asarray(kstar, dtype=np.uint32))
    ts = np.ascontiguousarray(np.asarray(tstar, dtype=np.uint32))
    return _load().ssh_oracle_bucket_key(int(seed), int(l), int(K), _ptr(ks, ctypes.c_uint32),
                                         _ptr(ts, ctypes.c_uint32))


def band_radius(band: float, m: int) -> int:
    return _load().ssh_oracle_band_radius(ctypes.c_float(band), int(m))


def dtw(a, b, rb: int) -> float:
    """Sec. 2.1: banded DTW (sum of squared costs, no square root), FP64."""
    a = _f32(a)
    b = _f32(b)
    assert len(a) == len(b)
    return _load().ssh_oracle_dtw(_ptr(a, ctypes.c_float), _ptr(b, ctypes.c_float), len(a), int(rb))


def lb_keogh(q, c, rb: int) -> float:
    """Sec. 3: LB_Keogh, the envelope (radius rb) of q against the samples of c."""
    q = _f32(q)
    c = _f32(c)
    return _load().ssh_oracle_lb_keogh(_ptr(q, ctypes.c_float), _ptr(c, ctypes.c_float), len(q), int(rb))


def lb_kim_fl(q, c) -> float:
    """LB_Kim's endpoint bound (the UCR suite's first stage, which Sec. 3 relies on):
    the costs of the first and last cells, which every warping path contains."""
    q = _f32(q)
    c = _f32(c)
    return _load().ssh_oracle_lb_kim_fl(_ptr(q, ctypes.c_float), _ptr(c, ctypes.c_float), len(q))


def lb_keogh_kim(q, c, rb: int) -> float:
    """LB_Keogh with the terms of c's first and last samples replaced by the exact
    first and last cell costs (LB_Kim folded into LB_Keogh)."""
    q = _f32(q)
    c = _f32(c)
    return _load().ssh_oracle_lb_keogh_kim(_ptr(q, ctypes.c_float), _ptr(c, ctypes.c_float), len(q), int(rb))


def lb_keogh_rev(q, c, rb: int) -> float:
    """LB_Keogh with the roles reversed: the envelope of the candidate c against the
    samples of q (the UCR suite's second LB_Keogh stage)."""
    return lb_keogh(c, q, rb)


def topk_dtw(q, rows, ids, rb: int, k: int):
    """Exact top-k by DTW over the rows of a [n, m] array."""
    q = _f32(q)
    rows = _f32(rows)
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.int64))
    n, m = rows.shape
    out_ids = np.zeros(k, dtype=np.int64)
    out_d = np.zeros(k, dtype=np.float64)
    _load().ssh_oracle_topk_dtw(_ptr(q, ctypes.c_float), _ptr(rows, ctypes.c_float), _ptr(ids, ctypes.c_int64),
                                n, m, int(rb), int(k), _ptr(out_ids, ctypes.c_int64), _ptr(out_d, ctypes.c_double))
    return out_ids, out_d


def hash_series(x, r, delta: int, n: int, seed: int, K: int, L: int):
    """Sec. 4.1-4.3 for one series: (kstar, tstar) with K*L entries, or None if too short."""
    x = _f32(x)
    r = _f32(r)
    ks = np.zeros(K * L, dtype=np.uint32)
    ts = np.zeros(K * L, dtype=np.uint32)
    nnz = _load().ssh_oracle_hash_series(_ptr(x, ctypes.c_float), len(x), _ptr(r, ctypes.c_float), len(r),
                                         int(delta), int(n), int(seed), int(K), int(L),
                                         _ptr(ks, ctypes.c_uint32), _ptr(ts, ctypes.c_uint32))
    if nnz < 0:
        return None
    return ks, ts


def recall_at_k(returned_ids, exact_ids) -> float:
    """Sec. 5.3 precision: |returned top-k  ∩  exact top-k| / |exact top-k|. Entries of -1 are
    empty slots (fewer than k series to return); the exact list then holds min(k, N) ids, and
    a result that returns all of them scores 1 (as an empty exact list does)."""
    exact = [int(i) for i in exact_ids if int(i) >= 0]
    got = {int(i) for i in returned_ids if int(i) >= 0}
    if not exact:
        return 1.0
    return sum(1 for i in exact if i in got) / float(len(exact))


def ndcg_at_k(returned_ids, gold_ids) -> float:
    """Sec. 5.3's NDCG of a returned top-k against the gold (exact DTW) top-k, k = len(gold_ids).
    The printed DCG divides by log2(i) for positions i = 1..k, which is 0 at i = 1, and gives
    R_i = k - i: read as the standard DCG, sum over result positions i = 1..k of
    rel / log2(i + 1), with a result's graded relevance k - g + 1 where g (1..k) is its rank in
    the gold list (k for the gold first, 1 for the gold k-th, 0 outside it); IDCG is the DCG
    of the gold list itself."""
    gold = [int(i) for i in gold_ids]
    k = len(gold)
    if k == 0:
        return 1.0
    rel = {g: k - r for r, g in enumerate(gold) if g >= 0}  # r = g - 1: relevance k .. 1
    dcg = 0.0
    for pos, i in enumerate(list(returned_ids)[:k]):
        dcg += rel.get(int(i), 0) / np.log2(pos + 2.0)
    idcg = sum((k - r) / np.log2(r + 2.0) for r, g in enumerate(gold) if g >= 0)
    return dcg / idcg if idcg > 0 else 1.0


# ------------------------------------------------------------------ the index

class OracleIndex:
    """Algorithms 1 and 2 with plain dictionaries.

    One table per l in [0, L); table l maps the K-tuple of (kstar, tstar) pairs
    of hashes l*K .. l*K+K-1 to the list of ids hashed there. Ids are assigned
    from 0 in insertion order. Series of different lengths live in separate
    per-length collections, and a query only sees series of its own length.
    """

    def __init__(self, W: int, delta: int, n: int, K: int, L: int, band: float, seed: int, family: str = "ssh"):
        if W < 1 or delta < 1 or n < 1 or n > 32 or K < 1 or L < 1 or not band >= 0:
            raise ValueError("invalid SSH parameters")
        if family not in ("ssh", "srp", "ssh-doph"):
            raise ValueError("family is 'ssh', 'srp' or 'ssh-doph'")
        # "srp": the paper's baseline, K sign random projections of the whole series per
        # table (hash values (bit, 0) in the same key fold); W, delta and n are unused.
        # "ssh-doph": SSH with the densified one-permutation minhash in place of ICWS
        self.family = family
        self.W, self.delta, self.n, self.K, self.L = W, delta, n, K, L
        self.band = float(np.float32(band))
        self.seed = int(seed)
        self.r = filter_r(seed, W)
        self.tables = [dict() for _ in range(L)]
        self.rows = {}        # length -> list of float32 arrays
        self.row_ids = {}     # length -> list of ids
        self.hashes = {}      # id -> (kstar, tstar)
        self.next_id = 0

    def min_length(self) -> int:
        return 1 if self.family == "srp" else self.W + (self.n - 1) * self.delta

    def tuples(self, kstar, tstar):
        K = self.K
        return [tuple((int(kstar[l * K + i]), int(tstar[l * K + i])) for i in range(K)) for l in range(self.L)]

    def hash(self, x):
        if self.family == "srp":
            bits = srp_bits(x, self.seed, self.K * self.L)
            return bits, np.zeros_like(bits)
        if self.family == "ssh-doph":  # Sec. 4.1-4.2, then the densified one-permutation minhash
            x = _f32(x)
            if len(x) < self.min_length():
                raise ValueError(f"series of length {len(x)} is shorter than {self.min_length()}")
            ids, counts = shingle(sketch(x, self.r, self.delta), self.n)
            return doph(self.seed, self.K * self.L, ids, counts)
        h = hash_series(x, self.r, self.delta, self.n, self.seed, self.K, self.L)
        if h is None:
            raise ValueError(f"series of length {len(x)} is shorter than W + (n-1)*delta = {self.min_length()}")
        return h

    def add(self, series_list) -> int:
        first = self.next_id
        for x in series_list:
            x = _f32(x)
            ks, ts = self.hash(x)
            i = self.next_id
            self.next_id += 1
            self.hashes[i] = (ks, ts)
            for l, tup in enumerate(self.tuples(ks, ts)):
                self.tables[l].setdefault(tup, []).append(i)
            self.rows.setdefault(len(x), []).append(x)
            self.row_ids.setdefault(len(x), []).append(i)
        return first

    def candidates(self, q) -> np.ndarray:
        """Algorithm 2: the union R of the buckets probed in every table (ids ascending)."""
        q = _f32(q)
        ks, ts = self.hash(q)
        found = set()
        length_ids = set(self.row_ids.get(len(q), []))
        for l, tup in enumerate(self.tuples(ks, ts)):
            for i in self.tables[l].get(tup, []):
                if i in length_ids:
                    found.add(i)
        return np.array(sorted(found), dtype=np.int64)

    def row_of(self, m: int):
        ids = np.array(self.row_ids.get(m, []), dtype=np.int64)
        rows = np.stack(self.rows[m]) if ids.size else np.zeros((0, m), np.float32)
        return ids, rows

    def query(self, q, k: int):
        """Algorithm 2: top-k of R by DTW (exact, no pruning): (ids, distances)."""
        q = _f32(q)
        m = len(q)
        cand = self.candidates(q)
        ids, rows = self.row_of(m)
        pos = {int(i): p for p, i in enumerate(ids)}
        sel = np.array([pos[int(c)] for c in cand], dtype=np.int64)
        sub = rows[sel] if sel.size else np.zeros((0, m), np.float32)
        return topk_dtw(q, sub, cand, band_radius(self.band, m), k)

    def exact_topk(self, q, k: int):
        """Brute-force DTW top-k over every stored series of the query's length."""
        q = _f32(q)
        ids, rows = self.row_of(len(q))
        return topk_dtw(q, rows, ids, band_radius(self.band, len(q)), k)
