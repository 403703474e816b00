#!/usr/bin/env python
"""Benchmark of the SSH index and query path on one GB300 (or N, one per rank).

One step = the whole hot path over one batch: build the index of N resident
series (sketch, shingle, weighted minhash, bucket keys, table sort) and answer
the query batch (hash, probe + union, LB_Keogh, banded DTW, top-k). The JSON
line reports series hashed per second of step time (value), the query-phase
throughput, recall@10 against exact DTW, single-query latency, the roofline
of the dominant kernel group, an end-to-end figure through host buffers, and
the CPU oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ssh|reference] [--small]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1610_07328_gb300 import synth  # noqa: E402

METRIC = "series hashed/s; queries/s at recall@10≥0.9 vs exact DTW; p50/p99 latency"

# Plain SSH at scale: 1M random-walk series of length 512 (z-normalised, FP32),
# W=80, delta=3, n=15, K=4, L=25, band 5% of m, 100 queries, top-10; recall
# against brute-force DTW on a 10k-series subset.
SCALE = dict(name="plain SSH at scale", N=1_000_000, m=512, W=80, delta=3, n=15, K=4, L=25, band=0.05, seed=0,
             nq=100, k=10, recall_subset=10_000)
# Plain SSH, tiny (a quick run): 1000 series x 128, W=32, delta=3, n=8, K=4, L=16, 10 queries, top-5.
TINY = dict(name="plain SSH tiny", N=1000, m=128, W=32, delta=3, n=8, K=4, L=16, band=0.05, seed=0, nq=10, k=5,
            recall_subset=1000)

FP32_LANES_PER_SM = 128


def workload_desc(w):
    return (f"{w['name']}: {w['N']:,} random-walk series x {w['m']} (FP32, z-normalised), W={w['W']} "
            f"delta={w['delta']} n={w['n']} K={w['K']} L={w['L']} band={w['band']} of m, {w['nq']} perturbed "
            f"queries, top-{w['k']}")


def peaks():
    """HBM copy bandwidth and the maximum SM clock measured on the GB300s
    (MEASURED_PEAKS.json), else the recipe's fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return dict(hbm_gbs=float(p["hbm_gbs"]), sm_max_mhz=float(p.get("sm_max_mhz") or 2070.0),
                    source="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


def l2_read_gbs(torch, dev, binding):
    """L2 read bandwidth measured here: one launch of the library's L1-bypassing read kernel
    (ssh_read_device) over a 32 MB buffer that stays in L2 (129 MB), 64 passes, timed with
    CUDA events on the launching stream; best of 5 launches after 3 warm-up launches."""
    x = torch.ones(8 << 20, dtype=torch.float32, device=dev)
    passes = 64
    st = torch.cuda.current_stream()
    for _ in range(3):
        binding.ssh_read_device(x, passes, st)
    best = float("inf")
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        binding.ssh_read_device(x, passes, st)
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return x.numel() * 4 * passes / (best / 1000.0) / 1e9


_FP32_PEAK = {}


def set_fp32_peak(num_sms, sm_max_mhz):
    _FP32_PEAK.update(sms=int(num_sms), mhz=float(sm_max_mhz))


def fp32_peak_tflops():
    """The device's SM count x 128 FP32 lanes x 2 FLOP (FMA) x the measured maximum SM clock."""
    return _FP32_PEAK["sms"] * FP32_LANES_PER_SM * 2 * _FP32_PEAK["mhz"] * 1e6 / 1e12


def fp32_peak_source():
    return "derived: %d SMs x %d FP32 lanes x 2 x %.0f MHz" % (_FP32_PEAK["sms"], FP32_LANES_PER_SM,
                                                                _FP32_PEAK["mhz"])


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                 r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def host_rss_bytes():
    """Resident set size of this process (Linux /proc), 0 where unavailable."""
    try:
        with open("/proc/self/status") as f:
            for line in f:
                if line.startswith("VmRSS:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def h2d_copy_gbs(torch, h_src, d_dst):
    """Host-to-device copy bandwidth from pinned memory: one copy of the whole series buffer,
    timed with CUDA events on the current stream, best of 3 after one warm-up."""
    st = torch.cuda.current_stream()
    d_dst.copy_(h_src, non_blocking=True)
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        d_dst.copy_(h_src, non_blocking=True)
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return h_src.numel() * h_src.element_size() / (best / 1000.0) / 1e9


def gpu_bus_id(torch, dev):
    try:
        p = torch.cuda.get_device_properties(dev)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


# -------------------------------------------------------------- CPU oracle

def oracle_sample(w, n_sample: int, n_queries: int, row0: int = 0):
    """Time the oracle on a bounded sample of the workload and extrapolate the
    step time: N * (hash time per series) + nq * (query time at n_sample) * N / n_sample
    (the candidate set, hence the rerank, grows in proportion to the index)."""
    import oracle
    db = synth.random_walk(row0 + n_sample, w["m"], seed=w["seed"])[row0:]
    qs, _ = synth.perturbed_queries(db, n_queries, seed=1)
    idx = oracle.OracleIndex(w["W"], w["delta"], w["n"], w["K"], w["L"], w["band"], w["seed"])
    t0 = time.perf_counter()
    idx.add(db)
    t1 = time.perf_counter()
    for q in qs:
        idx.query(q, w["k"])
    t2 = time.perf_counter()
    t_hash = (t1 - t0) / n_sample
    t_query = (t2 - t1) / n_queries
    step = w["N"] * t_hash + w["nq"] * t_query * (w["N"] / n_sample)
    return dict(value=w["N"] / step, seconds=t2 - t0, t_hash=t_hash, t_query=t_query,
                sample=(f"oracle indexed {n_sample} series and answered {n_queries} queries on them; step time "
                        f"extrapolated as N*t_hash + nq*t_query*N/{n_sample}"))


_ORACLE_WORKER = {}


def _oracle_worker_init(w, n_sample, n_queries):
    db = synth.random_walk(n_sample, w["m"], seed=w["seed"])
    qs, _ = synth.perturbed_queries(db, n_queries, seed=1)
    _ORACLE_WORKER.update(w=w, db=db, qs=qs, idx=None)


def _oracle_index(rows):
    import oracle
    w = _ORACLE_WORKER["w"]
    ix = oracle.OracleIndex(w["W"], w["delta"], w["n"], w["K"], w["L"], w["band"], w["seed"])
    ix.add(rows)
    return ix


def _oracle_hash_slice(bounds):
    a, b = bounds
    _oracle_index(_ORACLE_WORKER["db"][a:b])
    return b - a


def _oracle_build(_):
    if _ORACLE_WORKER["idx"] is None:
        _ORACLE_WORKER["idx"] = _oracle_index(_ORACLE_WORKER["db"])
    return os.getpid()


def _oracle_query(i):
    if _ORACLE_WORKER["idx"] is None:  # a worker that got no build task builds here (slower, never faster)
        _oracle_build(0)
    return _ORACLE_WORKER["idx"].query(_ORACLE_WORKER["qs"][i], _ORACLE_WORKER["w"]["k"])[0].tolist()


def oracle_sample_all_cores(w, n_sample: int, n_queries: int, timeout: float = 300.0):
    """oracle_sample with one spawned process per host core: the sample's series hashed in
    slices across the processes (wall time), then the queries spread over processes that each
    hold the sample's index (built before the timed query phase); same extrapolation."""
    import multiprocessing as mp
    P = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(P, initializer=_oracle_worker_init, initargs=(w, n_sample, n_queries)) as pool:
        pool.map_async(_oracle_hash_slice, [(0, 2)] * P, chunksize=1).get(timeout)  # warm-up
        step = (n_sample + P - 1) // P
        slices = [(a, min(n_sample, a + step)) for a in range(0, n_sample, step)]
        t0 = time.perf_counter()
        pool.map_async(_oracle_hash_slice, slices, chunksize=1).get(timeout)
        t1 = time.perf_counter()
        pool.map_async(_oracle_build, range(2 * P), chunksize=1).get(timeout)
        t2 = time.perf_counter()
        pool.map_async(_oracle_query, range(n_queries), chunksize=1).get(timeout)
        t3 = time.perf_counter()
    t_hash = (t1 - t0) / n_sample
    t_query = (t3 - t2) / n_queries
    step_s = w["N"] * t_hash + w["nq"] * t_query * (w["N"] / n_sample)
    return dict(value=w["N"] / step_s, cores=P, seconds=(t1 - t0) + (t3 - t2),
                sample=(f"{P} processes: the oracle hashed {n_sample} series in slices (wall time) and answered "
                        f"{n_queries} queries on their index spread over the processes; step time extrapolated "
                        f"as N*t_hash + nq*t_query*N/{n_sample}"))


def run_reference(args, w):
    """The oracle as it stands, on the host cores, each step a bounded sample of the workload:
    index an n_s-series slice and answer all nq queries on that slice's index. The query phase
    of the full step grows with N (candidate sets grow in proportion to the index), so a step
    over n_s series costs n_s/N of the full step under that model; value = n_s / step time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    n_s = 1000 if not args.small else 200
    n_slices = 5
    slices = []
    all_rows = synth.random_walk(n_slices * n_s, w["m"], seed=w["seed"])
    for s in range(n_slices):
        db = all_rows[s * n_s:(s + 1) * n_s]
        qs, _ = synth.perturbed_queries(db, w["nq"], seed=1 + s)
        slices.append((db, qs))
    step_s = []
    for s in range(args.warmup + args.steps):
        db, qs = slices[s % n_slices]
        t0 = time.perf_counter()
        idx = oracle.OracleIndex(w["W"], w["delta"], w["n"], w["K"], w["L"], w["band"], w["seed"])
        idx.add(db)
        for q in qs:
            idx.query(q, w["k"])
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            step_s.append(dt)
    ms_per_step = 1000.0 * statistics.mean(step_s)
    value = n_s / (ms_per_step / 1000.0)
    sample = (f"each step: the oracle indexes a {n_s}-series slice of the workload (one of {n_slices}) and answers "
              f"{w['nq']} perturbed queries on it, one core")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "series/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"sample of {workload_desc(w)}: {n_s} series + {w['nq']} queries per step",
                   "parallelism": "single process, CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "series/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "series/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "extrapolated_full_step_ms": 1000.0 * w["N"] / value,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def source_digest(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


CSRC = "paper_1610_07328_gb300/csrc/"
KERNEL_SOURCES = {
    "sketch": [CSRC + "hash_split.cu"],
    "sketch_fixup": [CSRC + "hash_split.cu"],
    "shingle": [CSRC + "hash_split.cu"],
    "cws": [CSRC + "hash_split.cu", CSRC + "hash_common.cuh"],
    "hash_generic": [CSRC + "hash_kernels.cu", CSRC + "hash_common.cuh"],
    "table_sort": [CSRC + "sort_kernels.cu"],
    "probe_union": [CSRC + "query_kernels.cu"],
    "lb_keogh": [CSRC + "query_kernels.cu"],
    "dtw": [CSRC + "query_kernels.cu"],
    "topk": [CSRC + "sort_kernels.cu", CSRC + "capi.cu"],
}


def traffic_for(group, field="bytes_per_launch"):
    """DRAM bytes (or another field) per launch from a committed ncu summary, if taken on the
    current source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    stage = group.split(".", 1)[-1]
    if not os.path.exists(path) or stage not in KERNEL_SOURCES:
        return None
    with open(path) as f:
        t = json.load(f)
    e = t.get(group)
    if not e or e.get("source_digest") != source_digest(KERNEL_SOURCES[stage]):
        return None
    return e.get(field)


def algorithmic(w, stage):
    """(bound, bytes or FLOP per unit) of a kernel group; units are series unless noted."""
    m, L, W, delta, n = w["m"], w["L"], w["W"], w["delta"], w["n"]
    nb = (m - W) // delta + 1
    nwords = (nb + 31) // 32
    S = nb - n + 1
    if stage == "sketch":       # series read once, sign bits written
        return "hbm", 4 * m + 4 * nwords
    if stage == "shingle":      # bits read, weighted set written (at most S slots)
        return "hbm", 4 * nwords + 4 * S
    if stage == "cws":          # weighted set read, L bucket keys written
        return "hbm", 4 * S + 8 * L
    if stage == "hash_generic":
        return "hbm", 4 * m + 8 * L
    if stage == "table_sort":   # per table entry: the key read once, (key, row) written once
        return "hbm", 20
    if stage == "lb_keogh":     # per candidate sample read
        return "hbm", 4
    if stage == "dtw":          # per DTW cell: difference and fused square-add (3 FLOP)
        return "alu", 3
    return None, None


def kernel_rooflines(w, times, pk):
    """Achieved vs peak for each kernel group, from the library's CUDA-event times."""
    out = {}
    total = sum(v["total_ms"] for v in times.values()) or 1.0
    for name, v in times.items():
        stage = name.split(".", 1)[-1]
        calls = max(v["calls"], 1)
        avg_ms = v["total_ms"] / calls
        units_per_call = v["units"] / calls
        e = dict(ms_total=v["total_ms"], calls=v["calls"], launches=v["launches"], avg_ms=avg_ms,
                 share=v["total_ms"] / total, units_per_call=units_per_call)
        bound, per = algorithmic(w, stage)
        if bound == "hbm":
            e.update(bound="hbm", unit="GB/s", achieved=units_per_call * per / (avg_ms * 1e-3) / 1e9,
                     peak=pk["hbm_gbs"])
        elif bound == "alu":
            e.update(bound="alu", unit="TFLOP/s", achieved=units_per_call * per / (avg_ms * 1e-3) / 1e12,
                     peak=fp32_peak_tflops())
        else:
            e.update(bound=None, unit=None, achieved=None, peak=None)
        if e.get("achieved") is not None:
            e["frac"] = e["achieved"] / e["peak"]
        out[name] = e
    # the hash pipeline of Sec. 4.1-4.3 as a whole: series read once, keys written once
    parts = [n for n in out if n.startswith("add.") and n.split(".", 1)[1] in
             ("sketch", "sketch_fixup", "shingle", "cws", "hash_generic")]
    if parts:
        ms = sum(out[n]["avg_ms"] for n in parts)
        units = out[parts[0]]["units_per_call"]
        ach = units * (4 * w["m"] + 8 * w["L"]) / (ms * 1e-3) / 1e9
        out["add.hash_pipeline"] = dict(ms_per_call=ms, series_per_call=units, bound="hbm", unit="GB/s",
                                        achieved=ach, peak=pk["hbm_gbs"], frac=ach / pk["hbm_gbs"],
                                        series_per_s=units / (ms * 1e-3))
    return out


def exact_topk_gpu(binding, torch, d_q, d_db, rows, m, rb, k):
    """Brute-force DTW top-k of each query over the given rows (parity-checked DTW kernel)."""
    nq = d_q.shape[0]
    out_ids = np.zeros((nq, k), np.int64)
    rows_t = torch.as_tensor(rows, dtype=torch.int64, device="cuda")
    for i in range(nq):
        a_idx = torch.full((len(rows),), i, dtype=torch.int64, device="cuda")
        d = torch.empty(len(rows), dtype=torch.float32, device="cuda")
        binding.ssh_dtw_device(d_q, a_idx, d_db, rows_t, m, rb, d)
        dd = d.cpu().numpy().astype(np.float64)
        order = np.lexsort((rows, dd))[:k]
        out_ids[i] = np.asarray(rows)[order]
    return out_ids


def recall(ids, exact):
    """Mean recall@k: returned ids found in the exact top-k over the exact list's valid (>= 0) ids."""
    r = []
    for a, b in zip(ids, exact):
        got = {int(x) for x in a if x >= 0}
        gold = [int(x) for x in b if x >= 0]
        r.append(sum(1 for x in gold if x in got) / len(gold) if gold else 1.0)
    return float(np.mean(r))


def ndcg(ids, exact):
    """Mean NDCG@k (Sec. 5.3, standard DCG): a returned id's relevance is k - g + 1 for gold
    rank g (1..k) in the exact top-k, 0 outside it; position i (1..k) is discounted by
    log2(i + 1); normalised by the DCG of the exact list."""
    out = []
    for a, b in zip(ids, exact):
        k = len(b)
        rel = {int(g): k - r for r, g in enumerate(b)}
        dcg = sum(rel.get(int(x), 0) / math.log2(p + 2) for p, x in enumerate(list(a)[:k]))
        idcg = sum((k - r) / math.log2(r + 2) for r in range(k))
        out.append(dcg / idcg if idcg > 0 else 1.0)
    return float(np.mean(out))


# Parameter sets tried for the recall operating point, from the most to the
# least selective; the operating point is the fastest one with recall@10 >= 0.9.
OPERATING_POINTS = [
    (80, 3, 15, 4, 25), (40, 3, 15, 4, 25), (40, 3, 12, 4, 25), (40, 3, 10, 4, 25),
    (40, 3, 8, 4, 25), (80, 3, 10, 2, 25), (80, 3, 12, 1, 25), (80, 3, 10, 1, 25),
]


def sweep_points(binding, torch, d_sub, d_q, exact, points, band, seed, k, n_plain=20, srp=False):
    """recall@10, candidate fraction and queries/s of each parameter set (W, delta, n, K, L) on a
    subset; the chosen point is the fastest with recall@10 >= 0.9 (else the one of highest recall).
    srp: the points are SRP baseline indexes (K, L used; W, delta, n ignored)."""
    n_sub, nq = d_sub.shape[0], d_q.shape[0]
    out = []
    for (W, delta, n, K, L) in points:
        make = (lambda: binding.SSHIndex.srp(K, L, band, seed)) if srp else \
            (lambda: binding.SSHIndex(W, delta, n, K, L, band, seed))
        with make() as ix:
            ix.add_device(d_sub)  # warm-up build (first use of the shapes)
            build = float("inf")
            for _ in range(2):
                ix.clear()
                b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                b0.record()
                ix.add_device(d_sub)
                b1.record()
                b1.synchronize()
                build = min(build, b0.elapsed_time(b1))
            ids = torch.empty((nq, k), dtype=torch.int64, device=d_q.device)
            dd = torch.empty((nq, k), dtype=torch.float32, device=d_q.device)
            ix.query_device(d_q, k, ids, dd)  # warm-up (and the DTW tiling's timing)
            torch.cuda.synchronize()
            ix.reset_stats()
            best = float("inf")
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ix.query_device(d_q, k, ids, dd)
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            st = ix.stats()
            r10 = recall(ids.cpu().numpy(), exact)
            one_i = torch.empty((1, k), dtype=torch.int64, device=d_q.device)
            one_d = torch.empty((1, k), dtype=torch.float32, device=d_q.device)
            lat = []
            for i in range(min(nq, n_plain)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ix.query_device(d_q[i:i + 1], k, one_i, one_d)
                e1.record()
                e1.synchronize()
                lat.append(e0.elapsed_time(e1))
        out.append({"W": W, "delta": delta, "n": n, "K": K, "L": L, "recall_at_10": r10,
                    "ndcg_at_10": ndcg(ids.cpu().numpy(), exact), "index_ms": build,
                    "candidate_fraction": st["candidates"] / (3 * nq) / n_sub,
                    "queries_per_s": nq / (best / 1000.0),
                    "plain_gpu_path_queries_per_s": 1000.0 / statistics.mean(lat) if lat else None})
    ok = [p for p in out if p["recall_at_10"] >= 0.9]
    chosen = max(ok, key=lambda p: p["queries_per_s"]) if ok else max(out, key=lambda p: p["recall_at_10"])
    return {"subset": n_sub, "queries": nq, "points": out, "chosen": chosen,
            "meets_recall_0_9": chosen["recall_at_10"] >= 0.9}


def recall_operating_point(binding, torch, d_sub, d_q, exact, w, k):
    """The OPERATING_POINTS sweep on the recall subset of the scale workload."""
    return sweep_points(binding, torch, d_sub, d_q, exact, OPERATING_POINTS, w["band"], w["seed"], k)


# Sec. 5.5's parameter study on the scale workload's recall subset: the window W,
# the step delta and the shingle length n, one at a time around (80, 3, 15), K=4, L=25.
STUDY_POINTS = {
    "W": [(W, 3, 15, 4, 25) for W in (40, 80, 120, 160)],
    "delta": [(80, d, 15, 4, 25) for d in (1, 2, 3, 5, 8)],
    "n": [(80, 3, n, 4, 25) for n in (8, 10, 12, 15)],
}


# The paper's SRP baseline (Sec. 5.2) on the same subset: K sign random projections of the
# whole series per table, 25 tables.
SRP_POINTS = [(1, 1, 1, K, 25) for K in (16, 8, 4, 2)]


def srp_baseline(binding, torch, d_sub, d_q, exact, w, k):
    """recall@10, NDCG@10, candidate fraction and queries/s of the SRP baseline on the recall subset."""
    sw = sweep_points(binding, torch, d_sub, d_q, exact, SRP_POINTS, w["band"], w["seed"], k, n_plain=0, srp=True)
    return {"subset": int(d_sub.shape[0]), "queries": int(d_q.shape[0]),
            "points": [{key: p[key] for key in ("K", "L", "recall_at_10", "ndcg_at_10", "candidate_fraction",
                                                 "index_ms", "queries_per_s")} for p in sw["points"]]}


def minhash_variants(binding, torch, d_db, d_sub, d_q, exact, w, k):
    """SSH_OPT_MINHASH 0 (ICWS) against 1 (densified one-permutation hashing): the index build of
    the whole workload (N series, borrowed; best of 3) with its minhash kernel's time, and
    recall@10 / NDCG@10 / candidate fraction on the recall subset at n = 15, 10, 8."""
    out = {}
    for mh, name in ((0, "icws"), (1, "doph")):
        entry = {}
        with binding.SSHIndex(w["W"], w["delta"], w["n"], w["K"], w["L"], w["band"], w["seed"]) as ix:
            ix.set_minhash(mh)
            best = float("inf")
            for rep in range(4):
                ix.clear()
                if rep == 3:
                    ix.reset_stats()
                    ix.set_kernel_timing(True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                ix.add_device(d_db, borrow=True)
                e1.record()
                e1.synchronize()
                if rep < 3:
                    best = min(best, e0.elapsed_time(e1))
            kt = ix.kernel_times()
            ix.set_kernel_timing(False)
        entry["index_ms"] = best
        entry["series_hashed_per_s_index_phase"] = d_db.shape[0] / (best / 1000.0)
        if "add.cws" in kt:
            entry["minhash_kernel_ms"] = kt["add.cws"]["total_ms"] / max(kt["add.cws"]["calls"], 1)
        pts = [(w["W"], w["delta"], n, w["K"], w["L"]) for n in (15, 10, 8)]
        sw = []
        for (W, delta, n, K, L) in pts:
            with binding.SSHIndex(W, delta, n, K, L, w["band"], w["seed"]) as ix:
                ix.set_minhash(mh)
                ix.add_device(d_sub)
                ids, ms, st = _timed_query(torch, ix, d_q, k)
                sw.append({"n": n, "recall_at_10": recall(ids.cpu().numpy(), exact),
                           "ndcg_at_10": ndcg(ids.cpu().numpy(), exact),
                           "candidate_fraction": st["candidates"] / max(st["queries"], 1) / d_sub.shape[0],
                           "queries_per_s": d_q.shape[0] / (ms / 1000.0)})
        entry["subset_points"] = sw
        out[name] = entry
    return out


def parameter_study(binding, torch, d_sub, d_q, exact, w, k):
    """recall@10, NDCG@10, candidate fraction, index build time and queries/s as W, delta and n vary."""
    out = {}
    for name, pts in STUDY_POINTS.items():
        sw = sweep_points(binding, torch, d_sub, d_q, exact, pts, w["band"], w["seed"], k, n_plain=0)
        out[name] = [{key: p[key] for key in ("W", "delta", "n", "recall_at_10", "ndcg_at_10", "candidate_fraction",
                                              "index_ms", "queries_per_s")} for p in sw["points"]]
    out["subset"] = int(d_sub.shape[0])
    out["queries"] = int(d_q.shape[0])
    return out


def _timed_query(torch, ix, d_q, k, reps=3):
    ids = torch.empty((d_q.shape[0], k), dtype=torch.int64, device=d_q.device)
    dd = torch.empty((d_q.shape[0], k), dtype=torch.float32, device=d_q.device)
    ix.query_device(d_q, k, ids, dd)  # warm-up
    torch.cuda.synchronize()
    ix.reset_stats()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ix.query_device(d_q, k, ids, dd)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    st = ix.stats()
    return ids, best, st


def cascade_modes(torch, ix, d_q, k, reps=1):
    """Queries/s and pruned fractions of each SSH_OPT_LB_CASCADE mode (0 LB_Keogh, 1 with the LB_Kim
    endpoints, 2 with the reversed LB_Keogh too); the index is left in mode 1 (the default)."""
    out = {}
    for mode in (0, 1, 2):
        ix.set_lb_cascade(mode)
        _, ms, st = _timed_query(torch, ix, d_q, k, reps=reps)
        out[str(mode)] = {"queries_per_s": d_q.shape[0] / (ms / 1000.0),
                          "lb_pruned_fraction": 1.0 - st["dtw_computed"] / max(st["candidates"], 1),
                          "reversed_lb_pruned_fraction": st["lb2_pruned"] / max(st["candidates"], 1)}
    ix.set_lb_cascade(1)
    return out


def exact_scan_measurement(binding, torch, d_sub, d_db, d_q, exact_sub, w, k, n_full):
    """The comparator without hashing (SSH_OPT_EXACT_SCAN): every stored series goes through the
    same LB_Keogh filter and early-abandoning DTW; on the recall subset and on the whole database."""
    out = {}
    for name, db, nq in (("subset", d_sub, d_q.shape[0]), ("full_db", d_db, n_full)):
        with binding.SSHIndex(w["W"], w["delta"], w["n"], w["K"], w["L"], w["band"], w["seed"]) as ix:
            ix.add_device(db, borrow=True)
            ix.set_exact_scan(True)
            ids, ms, st = _timed_query(torch, ix, d_q[:nq].contiguous(), k, reps=3 if name == "subset" else 1)
            entry = {"rows": int(db.shape[0]), "queries": int(nq), "queries_per_s": nq / (ms / 1000.0),
                     "lb_pruned_fraction": 1.0 - st["dtw_computed"] / max(st["candidates"], 1),
                     "reversed_lb_pruned_fraction": st["lb2_pruned"] / max(st["candidates"], 1),
                     "by_cascade_mode": cascade_modes(torch, ix, d_q[:nq].contiguous(), k,
                                                      reps=3 if name == "subset" else 1)}
            if name == "subset":
                entry["recall_at_10"] = recall(ids.cpu().numpy(), exact_sub)
            out[name] = entry
    return out


def dtw_full_load_measurement(binding, torch, d_db, d_q, w, rows=40_000, nq=10):
    """The banded DTW kernel at full load: an exact scan with LB pruning off ranks every one of
    `rows` stored series for each of `nq` queries, so one DTW launch runs rows * nq complete
    pairs (no abandoning); its CUDA-event time gives cells/s and the FP32 fraction at 3 FLOP
    per cell. The query path's own DTW passes are short (seeds, then survivors cut by the bound)
    and are reported apart as query.dtw."""
    try:
        with binding.SSHIndex(w["W"], w["delta"], w["n"], w["K"], w["L"], w["band"], w["seed"]) as ix:
            ix.add_device(d_db[:rows].contiguous(), borrow=True)
            ix.set_exact_scan(True)
            ix.set_lb_prune(False)
            q = d_q[:nq].contiguous()
            _timed_query(torch, ix, q, w["k"], reps=1)
            ix.set_kernel_timing(True)
            ix.reset_stats()
            _timed_query(torch, ix, q, w["k"], reps=3)
            t = ix.kernel_times()["query.dtw"]
            ix.set_kernel_timing(False)
        ms = t["total_ms"] / t["calls"]
        cells = t["units"] / t["calls"]
        tflops = 3.0 * cells / (ms * 1e-3) / 1e12
        return {"pairs_per_launch": rows * nq, "cells_per_launch": cells, "ms_per_launch": ms,
                "cells_per_s": cells / (ms * 1e-3), "tflops": tflops, "peak_tflops": fp32_peak_tflops(),
                "frac": tflops / fp32_peak_tflops(), "peak_source": fp32_peak_source()}
    except Exception as e:  # a measurement block: report, never lose the bench line
        return {"error": "%s: %s" % (type(e).__name__, e)}


BATCH_LENGTHS = (128, 256, 512, 1024, 2048)


def batched_measurement(args, binding, torch, dev):
    """Mixed-length queries over per-length indexes (W = m/8) through one batch plan (a CUDA graph),
    against the plain path of one query per call; recall@10 against exact DTW on a sample."""
    small = args.small
    N4, nq4, k = (2000, 256, 10) if small else (200_000, 4096, 10)
    rng = np.random.default_rng(4)
    t0 = time.perf_counter()
    hosts = {m: synth.random_walk(N4, m, seed=40 + m) for m in BATCH_LENGTHS}
    data = {m: torch.from_numpy(hosts[m]).to(dev) for m in BATCH_LENGTHS}
    qlens = rng.choice(np.array(BATCH_LENGTHS, np.int32), size=nq4)
    qs = []
    for i, m in enumerate(qlens):
        q, _ = synth.perturbed_queries(hosts[m], 1, seed=1000 + i)
        qs.append(q[0])
    d_q = torch.from_numpy(np.concatenate(qs)).to(dev)
    gen_s = time.perf_counter() - t0
    idxs = [binding.SSHIndex(m // 8, 3, 15, 4, 25, 0.05, 0) for m in BATCH_LENGTHS]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for ix, m in zip(idxs, BATCH_LENGTHS):
        ix.add_device(data[m], borrow=True)
    e1.record()
    e1.synchronize()
    build_ms = e0.elapsed_time(e1)
    ids = torch.empty((nq4, k), dtype=torch.int64, device=dev)
    dd = torch.empty((nq4, k), dtype=torch.float32, device=dev)
    which = torch.empty((nq4,), dtype=torch.int32, device=dev)
    out = {"workload": "5 per-length indexes x %d random walks, m in %s, W = m/8, delta=3, n=15, K=4, L=25, "
                       "band 5%%; %d queries of uniformly mixed lengths, top-%d" % (N4, list(BATCH_LENGTHS), nq4, k),
           "index_build_series_per_s": 5 * N4 / (build_ms / 1000.0)}
    with binding.SSHBatch(idxs, max_queries=nq4, k=k) as bt:
        modes = {}
        # the rerank as one persistent launch, as per-class kernels, then by batch size (the default)
        for persistent in (True, False, None):
            bt.set_persistent(persistent)
            for _ in range(2):  # the first batch runs directly and captures the graph
                bt.query(d_q, qlens, ids, dd, which)
            torch.cuda.synchronize()
            steps = max(3, min(args.steps, 5))
            e0.record()
            for _ in range(steps):
                bt.query(d_q, qlens, ids, dd, which)
            e1.record()
            e1.synchronize()
            modes[persistent] = (e0.elapsed_time(e1) / steps, bt.stats())
        batch_ms, st = modes[None]
    out.update({"batched_queries_per_s": nq4 / (batch_ms / 1000.0), "ms_per_batch": batch_ms,
                "graph_kernels": st["graph_kernels"],
                "rerank": "by batch size (persistent launch up to 512 queries, per-class kernels above)",
                "persistent_rerank": {"queries_per_s": nq4 / (modes[True][0] / 1000.0), "ms_per_batch": modes[True][0],
                                      "graph_kernels": modes[True][1]["graph_kernels"]},
                "per_class_kernels": {"queries_per_s": nq4 / (modes[False][0] / 1000.0),
                                      "ms_per_batch": modes[False][0],
                                      "graph_kernels": modes[False][1]["graph_kernels"]},
                "candidates_per_query": st["pairs"] / nq4, "dtw_per_query": st["dtw"] / nq4})
    # small batches of the same mix (the serving loop's regime), both rerank forms
    small = []
    for nsm in (64, 256, 1024):
        offs_s = np.concatenate([[0], np.cumsum(qlens[:nsm])])
        d_qs = d_q[: int(offs_s[-1])].contiguous()
        row = {"queries": nsm}
        with binding.SSHBatch(idxs, max_queries=nsm, k=k) as bs:
            for persistent, key in ((True, "persistent"), (False, "per_class")):
                bs.set_persistent(persistent)
                for _ in range(3):
                    bs.query(d_qs, qlens[:nsm], ids[:nsm], dd[:nsm])
                torch.cuda.synchronize()
                e0.record()
                for _ in range(5):
                    bs.query(d_qs, qlens[:nsm], ids[:nsm], dd[:nsm])
                e1.record()
                e1.synchronize()
                ms = e0.elapsed_time(e1) / 5
                row[key] = {"ms_per_batch": ms, "queries_per_s": nsm / (ms / 1000.0),
                            "graph_kernels": bs.stats()["graph_kernels"]}
        small.append(row)
    out["small_batches"] = small
    # plain path: one query per call on the query's own index
    n_plain = min(nq4, 256)
    one_i = torch.empty((1, k), dtype=torch.int64, device=dev)
    one_d = torch.empty((1, k), dtype=torch.float32, device=dev)
    offs = np.concatenate([[0], np.cumsum(qlens)])
    for i in range(min(n_plain, 8)):  # warm-up
        m = int(qlens[i])
        idxs[BATCH_LENGTHS.index(m)].query_device(d_q[offs[i]:offs[i] + m].view(1, m), k, one_i, one_d)
    torch.cuda.synchronize()
    e0.record()
    for i in range(n_plain):
        m = int(qlens[i])
        idxs[BATCH_LENGTHS.index(m)].query_device(d_q[offs[i]:offs[i] + m].view(1, m), k, one_i, one_d)
    e1.record()
    e1.synchronize()
    out["plain_gpu_path_queries_per_s"] = n_plain / (e0.elapsed_time(e1) / 1000.0)
    out["plain_sample"] = n_plain
    # recall@10 against exact DTW over the whole per-length collection, a few queries per length
    res = ids.cpu().numpy()
    rec = []
    per_len = 2 if small else 4
    for m in BATCH_LENGTHS:
        sel = [i for i in range(nq4) if qlens[i] == m][:per_len]
        if not sel:
            continue
        d_sel = torch.stack([d_q[offs[i]:offs[i] + m] for i in sel]).contiguous()
        rb = min(int(math.floor(np.float32(0.05) * np.float64(m))), m - 1)
        ex = exact_topk_gpu(binding, torch, d_sel, data[m], np.arange(N4, dtype=np.int64), m, rb, k)
        rec.append(recall(res[sel], ex))
    out["recall_at_10"] = float(np.mean(rec)) if rec else None
    out["recall_queries"] = per_len * len(BATCH_LENGTHS)
    # pruning and speed against length (the exact scan of each collection; a Table 4 analog)
    per_length = []
    for ix, m in zip(idxs, BATCH_LENGTHS):
        sel = [i for i in range(nq4) if qlens[i] == m][:8]
        d_sel = torch.stack([d_q[offs[i]:offs[i] + m] for i in sel]).contiguous()
        _, ms_h, st_h = _timed_query(torch, ix, d_sel, k, reps=1)
        ix.set_exact_scan(True)
        _, ms_e, st_e = _timed_query(torch, ix, d_sel, k, reps=1)
        by_mode = cascade_modes(torch, ix, d_sel, k)
        ix.set_exact_scan(False)
        per_length.append({"m": m, "ssh_queries_per_s": len(sel) / (ms_h / 1000.0),
                           "ssh_candidate_fraction": st_h["candidates"] / max(st_h["queries"], 1) / N4,
                           "ssh_filtered_by_hashing": 1.0 - st_h["candidates"] / max(st_h["queries"], 1) / N4,
                           "exact_queries_per_s": len(sel) / (ms_e / 1000.0),
                           "exact_lb_pruned_fraction": 1.0 - st_e["dtw_computed"] / max(st_e["candidates"], 1),
                           "exact_reversed_lb_pruned_fraction": st_e["lb2_pruned"] / max(st_e["candidates"], 1),
                           "exact_by_cascade_mode": by_mode})
    out["per_length"] = per_length
    out["setup_s"] = gen_s
    for ix in idxs:
        ix.close()
    out["at_recall"] = batched_at_recall(args, binding, torch, dev, data, qlens, d_q, offs, k)
    return out


def recall_points_for(m):
    """Parameter sets tried per length for recall@10 >= 0.9 (the scale workload's sweep, W scaled
    with m): narrower windows and shorter shingles, then one hash per table."""
    w1, w2 = max(8, m * 5 // 64), m // 8
    return [(w1, 3, 10, 4, 25), (w1, 3, 8, 4, 25), (w2, 3, 10, 1, 25), (w2, 3, 8, 1, 25)]


def batched_at_recall(args, binding, torch, dev, data, qlens, d_q, offs, k):
    """The batched workload at parameters that reach recall@10 >= 0.9: per length, the fastest
    point of recall_points_for(m) with recall >= 0.9 on the first 10,000 rows (20 queries), then
    the five indexes at those parameters through one batch plan on 1,024 of the mixed-length
    queries, against one query per call, and recall@10 over the whole per-length collections."""
    small = args.small
    n_sub, n_sweep, nq_r, n_plain, per_len = (1000, 8, 128, 16, 2) if small else (10_000, 20, 1024, 64, 4)
    N4 = int(next(iter(data.values())).shape[0])
    chosen, sweeps = {}, []
    for m in BATCH_LENGTHS:
        sel = [i for i in range(len(qlens)) if qlens[i] == m][:n_sweep]
        d_sel = torch.stack([d_q[offs[i]:offs[i] + m] for i in sel]).contiguous()
        d_sub = data[m][:n_sub].contiguous()
        rb = min(int(math.floor(np.float32(0.05) * np.float64(m))), m - 1)
        ex = exact_topk_gpu(binding, torch, d_sel, d_sub, np.arange(n_sub, dtype=np.int64), m, rb, k)
        sw = sweep_points(binding, torch, d_sub, d_sel, ex, recall_points_for(m), 0.05, 0, k, n_plain=0)
        chosen[m] = sw["chosen"]
        sweeps.append({"m": m, **{key: sw["chosen"][key] for key in ("W", "delta", "n", "K", "L", "recall_at_10",
                                                                   "candidate_fraction")}})
    idxs = [binding.SSHIndex(chosen[m]["W"], chosen[m]["delta"], chosen[m]["n"], chosen[m]["K"], chosen[m]["L"],
                             0.05, 0) for m in BATCH_LENGTHS]
    for ix, m in zip(idxs, BATCH_LENGTHS):
        ix.add_device(data[m], borrow=True)
    ql = np.asarray(qlens[:nq_r])
    nfloat = int(offs[nq_r])
    d_qr = d_q[:nfloat].contiguous()
    ids = torch.empty((nq_r, k), dtype=torch.int64, device=dev)
    dd = torch.empty((nq_r, k), dtype=torch.float32, device=dev)
    which = torch.empty((nq_r,), dtype=torch.int32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with binding.SSHBatch(idxs, max_queries=nq_r, k=k) as bt:
        for _ in range(2):  # the first batch runs directly (growing the pair buffers) and captures the graph
            bt.query(d_qr, ql, ids, dd, which)
        torch.cuda.synchronize()
        steps = 3
        e0.record()
        for _ in range(steps):
            bt.query(d_qr, ql, ids, dd, which)
        e1.record()
        e1.synchronize()
        batch_ms = e0.elapsed_time(e1) / steps
        st = bt.stats()
    one_i = torch.empty((1, k), dtype=torch.int64, device=dev)
    one_d = torch.empty((1, k), dtype=torch.float32, device=dev)
    for i in range(4):  # warm-up
        m = int(ql[i])
        idxs[BATCH_LENGTHS.index(m)].query_device(d_qr[offs[i]:offs[i] + m].view(1, m), k, one_i, one_d)
    torch.cuda.synchronize()
    e0.record()
    for i in range(n_plain):
        m = int(ql[i])
        idxs[BATCH_LENGTHS.index(m)].query_device(d_qr[offs[i]:offs[i] + m].view(1, m), k, one_i, one_d)
    e1.record()
    e1.synchronize()
    plain_qps = n_plain / (e0.elapsed_time(e1) / 1000.0)
    res = ids.cpu().numpy()
    rec = []
    for m in BATCH_LENGTHS:
        sel = [i for i in range(nq_r) if ql[i] == m][:per_len]
        if not sel:
            continue
        d_sel = torch.stack([d_qr[offs[i]:offs[i] + m] for i in sel]).contiguous()
        rb = min(int(math.floor(np.float32(0.05) * np.float64(m))), m - 1)
        ex = exact_topk_gpu(binding, torch, d_sel, data[m], np.arange(N4, dtype=np.int64), m, rb, k)
        rec.append(recall(res[sel], ex))
    for ix in idxs:
        ix.close()
    return {"params_per_length": sweeps, "sweep_subset": n_sub, "sweep_queries_per_length": n_sweep,
            "queries": nq_r, "batched_queries_per_s": nq_r / (batch_ms / 1000.0), "ms_per_batch": batch_ms,
            "candidates_per_query": st["pairs"] / nq_r, "dtw_per_query": st["dtw"] / nq_r,
            "plain_gpu_path_queries_per_s": plain_qps, "plain_sample": n_plain,
            "recall_at_10": float(np.mean(rec)) if rec else None, "recall_queries": per_len * len(BATCH_LENGTHS)}


def ecg_like_gpu(torch, N, m, seed, dev, chunk=65536):
    """The ECG-like recipe of synth.ecg_like generated on the GPU with torch's generator
    (the serving index is too large for the host generator): beats of P/QRS/T Gaussian bumps
    (sigma 8/3/12, amplitude 0.15/1.0/0.3 at -0.2/0/+0.3 period), periods uniform 180-260,
    first beat offset uniform 0-64, wander 0.1 sin(2 pi t / T_w + phi) with T_w uniform
    700-1200, noise N(0, 0.05^2); not z-normalised."""
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    out = torch.empty((N, m), dtype=torch.float32, device=dev)
    t = torch.arange(m, dtype=torch.float32, device=dev)[None, :]
    nb = m // 180 + 3
    for a in range(0, N, chunk):
        n = min(chunk, N - a)
        per = torch.rand((n, nb), generator=g, device=dev) * 80.0 + 180.0
        off = torch.rand((n, 1), generator=g, device=dev) * 64.0
        cen = off + torch.cat([torch.zeros((n, 1), device=dev), torch.cumsum(per[:, :-1], 1)], 1)
        x = torch.zeros((n, m), device=dev)
        for b in range(nb):
            c0, p = cen[:, b:b + 1], per[:, b:b + 1]
            for rel, sig, amp in ((-0.2, 8.0, 0.15), (0.0, 3.0, 1.0), (0.3, 12.0, 0.3)):
                x += amp * torch.exp(-0.5 * ((t - (c0 + rel * p)) / sig) ** 2)
        tw = torch.rand((n, 1), generator=g, device=dev) * 500.0 + 700.0
        phi = torch.rand((n, 1), generator=g, device=dev) * (2.0 * math.pi)
        x += 0.1 * torch.sin(2.0 * math.pi * t / tw + phi)
        x += 0.05 * torch.randn((n, m), generator=g, device=dev)
        out[a:a + n] = x
    return out


SERVE_RATES = (1000, 5000, 20000, 50000)


def subsequence_measurement(args, binding, torch, dev):
    """Sec. 5.1's workload: every length-128 window (step 1) of one long random-walk stream,
    indexed with the paper's Random Walk parameters (W=30, delta=5, n=15, one hash per table,
    20 tables) through ssh_index_add_windows_device (windows borrowed, sketch positions shared);
    the same windows hashed as rows for comparison; queries/s and recall@10 against the exact scan
    of the same windows."""
    small = args.small
    n_s, t, nq, k = ((1 << 18) if small else (1 << 24)), 128, 100, 10
    W, delta, n, K, L, band = 30, 5, 15, 1, 20, 0.05
    t0 = time.perf_counter()
    stream = synth.random_walk(1, n_s, seed=90)[0]
    d_s = torch.from_numpy(stream).to(dev)
    starts = np.random.default_rng(91).integers(0, n_s - t, nq)
    qs, _ = synth.perturbed_queries(np.stack([stream[p:p + t] for p in starts]), nq, seed=92)
    d_q = torch.from_numpy(qs).to(dev)
    gen_s = time.perf_counter() - t0
    nwin = n_s - t + 1
    out = {"workload": "windows of length %d at every offset of a %d-sample random-walk stream (%d windows), "
                       "W=%d, delta=%d, n=%d, K=%d, L=%d, band 5%%, %d queries (perturbed windows), top-%d"
                       % (t, n_s, nwin, W, delta, n, K, L, nq, k), "setup_s": gen_s}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with binding.SSHIndex(W, delta, n, K, L, band, 0) as ix:
        for generic in (True, False):  # rows first (the stream path's index stays for the queries)
            ix.set_hash_kernel(generic)
            best = float("inf")
            for _ in range(3):
                ix.clear()
                torch.cuda.synchronize()
                e0.record()
                ix.add_windows_device(d_s, t, 1)
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out["rows_path" if generic else "stream_path"] = {"index_ms": best,
                                                              "windows_per_s": nwin / (best / 1000.0)}
        ix.set_hash_kernel(False)
        ids, ms, st = _timed_query(torch, ix, d_q, k)
        out.update({"queries_per_s": nq / (ms / 1000.0),
                    "candidate_fraction": st["candidates"] / max(st["queries"], 1) / nwin})
        nrec = 4 if small else 10
        ix.set_exact_scan(True)
        ex_ids, ms_e, _ = _timed_query(torch, ix, d_q[:nrec].contiguous(), k, reps=1)
        ix.set_exact_scan(False)
        out["recall_at_10"] = recall(ids.cpu().numpy()[:nrec], ex_ids.cpu().numpy())
        out["recall_queries"] = nrec
        out["exact_scan_queries_per_s"] = nrec / (ms_e / 1000.0)
    return out


def serve_rates(srv, rates, dur, q_host, ins_pool, m, rng):
    """Open-loop serving phases: per offered rate, Poisson arrivals for `dur` seconds (queries
    drawn from q_host) while 100 random walks are inserted every 10 ms; served queries/s, p50/p99
    latency from each query's scheduled arrival to its rows on the host, batch sizes, inserts/s."""
    import threading
    pool = len(q_host)
    # warm-up: every slot's first batch runs directly and captures its graph
    for _ in range(3):
        tk = srv.submit(q_host[:256], np.full(min(256, pool), m, np.int32))
        srv.wait(tk[-1], 120.0)
    srv.flush(120.0)
    res = []
    for rate in rates:
        n = max(1, int(rate * dur))
        arr = np.cumsum(rng.exponential(1.0 / rate, n))
        qidx = rng.integers(0, pool, n)
        got = []
        done_evt = threading.Event()

        def collector():
            while len(got) < n:
                tk, _, _, lat, stt = srv.collect(4096, 0.01)
                got.extend(zip(lat.tolist(), stt.tolist()))
            done_evt.set()

        while len(srv.collect(4096, 0.0)[0]):  # results of earlier phases
            pass
        st0 = srv.stats()
        th = threading.Thread(target=collector, daemon=True)
        th.start()
        start = srv.now() + 0.02
        arr_abs = start + arr
        ins_t, ins_i, i = start, 0, 0
        while i < n:
            now = srv.now()
            j = int(np.searchsorted(arr_abs, now, side="right"))
            if j > i:
                sel = qidx[i:j]
                srv.submit(q_host[sel], np.full(j - i, m, np.int32), arr_abs[i:j])
                i = j
            while ins_t <= now:  # 100 random walks every 10 ms
                a = (ins_i * 100) % (len(ins_pool) - 100)
                srv.insert(ins_pool[a:a + 100], np.full(100, m, np.int32))
                ins_t += 0.01
                ins_i += 1
            time.sleep(0.0002)
        done_evt.wait(300.0)
        t_end = srv.now()
        srv.flush(300.0)
        st1 = srv.stats()
        lat = np.array([l for l, sc in got])
        ok = sum(1 for _, sc in got if sc == 0)
        span = max(t_end - start, 1e-9)
        res.append({
            "offered_qps": rate, "queries": n, "completed_ok": ok,
            "served_qps": ok / span,
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "mean_batch": (st1["queries_done"] - st0["queries_done"]) / max(st1["batches"] - st0["batches"], 1),
            "batches": st1["batches"] - st0["batches"],
            "max_inflight": st1["max_inflight"],
            "inserts_per_s": (st1["inserts_applied"] - st0["inserts_applied"]) / span,
        })
    return res


def serving_measurement(args, binding, torch, dev):
    """Poisson query arrivals at several rates against a served ECG-like index while random
    walks are inserted at 10k/s; open-loop latency from each query's scheduled arrival."""
    small = args.small
    N5, m, k = (20_000, 1024, 10) if small else (2_000_000, 1024, 10)
    dur = 0.3 if small else 1.0
    t0 = time.perf_counter()
    db = ecg_like_gpu(torch, N5, m, 3, dev)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    pool = 4096
    src = torch.randint(0, N5, (pool,), generator=g, device=dev)
    qd = db[src] + 0.1 * torch.randn((pool, m), generator=g, device=dev)
    shifts = torch.randint(0, 9, (pool,), generator=g, device=dev).cpu().numpy()
    q_host = np.stack([np.roll(r, int(sft)) for r, sft in zip(qd.cpu().numpy(), shifts)]).astype(np.float32)
    ins_pool = synth.random_walk(2000, m, seed=77)
    gen_s = time.perf_counter() - t0
    ix = binding.SSHIndex(120, 5, 15, 4, 50, 0.10, 0)
    ix.add_device(db, borrow=True)
    torch.cuda.synchronize()
    out = {"workload": "ECG-like index of %d x %d (W=120, delta=5, n=15, K=4, L=50, band 10%%), top-%d; "
                       "Poisson arrivals, random walks inserted at 10k/s" % (N5, m, k),
           "rates": []}
    with binding.SSHServer([ix], k=k, max_batch=256, max_slots=4, reserve_bytes=2 << 30) as srv:
        out["rates"] = serve_rates(srv, SERVE_RATES, dur, q_host, ins_pool, m, np.random.default_rng(8))
        st = srv.stats()
        out["slots"] = st["slots"]
        out["insert_mean_latency_ms"] = st["insert_latency_ms_sum"] / max(st["insert_batches"], 1)
    # recall@10 of the served configuration against exact DTW over the whole index (a sample)
    nrec = 4 if small else 12
    d_qs = torch.from_numpy(q_host[:nrec]).to(dev)
    ids = torch.empty((nrec, k), dtype=torch.int64, device=dev)
    dd = torch.empty((nrec, k), dtype=torch.float32, device=dev)
    ix.clear()
    ix.add_device(db, borrow=True)  # without the inserted walks: exact top-k over the same rows
    ix.query_device(d_qs, k, ids, dd)
    rb = min(int(math.floor(np.float32(0.10) * np.float64(m))), m - 1)
    ex = exact_topk_gpu(binding, torch, d_qs, db, np.arange(N5, dtype=np.int64), m, rb, k)
    out["recall_at_10"] = recall(ids.cpu().numpy(), ex)
    out["recall_queries"] = nrec
    out["setup_s"] = gen_s
    ix.close()
    out["at_recall"] = served_at_recall(args, binding, torch, dev, db, q_host, ins_pool, m, k)
    del db
    return out


# Parameter sets tried on the ECG-like index for recall@10 >= 0.9 (m = 1024, band 10%).
ECG_RECALL_POINTS = [(60, 5, 10, 4, 50), (60, 5, 8, 4, 50), (120, 5, 10, 1, 50), (120, 5, 8, 1, 50)]


def served_at_recall(args, binding, torch, dev, db, q_host, ins_pool, m, k):
    """The served workload at parameters that reach recall@10 >= 0.9: the fastest point of
    ECG_RECALL_POINTS with recall >= 0.9 on the first 10,000 rows (20 queries); its batched
    capacity (one call of 256 queries) and recall@10 over the whole index; then the serving loop
    at 25%, 50% and 90% of that capacity for 3 s each, inserts at 10k/s as before."""
    small = args.small
    n_sub, n_sweep, nrec = (2000, 8, 4) if small else (10_000, 20, 8)
    N5 = int(db.shape[0])
    rb = min(int(math.floor(np.float32(0.10) * np.float64(m))), m - 1)
    d_sub = db[:n_sub].contiguous()
    d_sw = torch.from_numpy(q_host[:n_sweep]).to(dev)
    ex = exact_topk_gpu(binding, torch, d_sw, d_sub, np.arange(n_sub, dtype=np.int64), m, rb, k)
    sw = sweep_points(binding, torch, d_sub, d_sw, ex, ECG_RECALL_POINTS, 0.10, 0, k, n_plain=0)
    c = sw["chosen"]
    out = {"params": {key: c[key] for key in ("W", "delta", "n", "K", "L")},
           "sweep": [{key: p[key] for key in ("W", "delta", "n", "K", "L", "recall_at_10", "candidate_fraction",
                                              "queries_per_s")} for p in sw["points"]],
           "sweep_subset": n_sub, "sweep_queries": n_sweep}
    ix = binding.SSHIndex(c["W"], c["delta"], c["n"], c["K"], c["L"], 0.10, 0)
    ix.add_device(db, borrow=True)
    ncap = min(256, len(q_host))
    d_cap = torch.from_numpy(q_host[:ncap]).to(dev)
    ids, ms, _ = _timed_query(torch, ix, d_cap, k, reps=1)
    cap_qps = ncap / (ms / 1000.0)
    ex = exact_topk_gpu(binding, torch, d_cap[:nrec].contiguous(), db, np.arange(N5, dtype=np.int64), m, rb, k)
    out.update({"capacity_queries_per_s": cap_qps, "recall_at_10": recall(ids.cpu().numpy()[:nrec], ex),
                "recall_queries": nrec})
    one_i = torch.empty((1, k), dtype=torch.int64, device=dev)
    one_d = torch.empty((1, k), dtype=torch.float32, device=dev)
    lat = []
    for i in range(8):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ix.query_device(d_cap[i:i + 1], k, one_i, one_d)
        e1.record()
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
    out["plain_gpu_path_queries_per_s"] = 1000.0 / statistics.mean(lat[1:])
    rates = [max(1.0, round(f * cap_qps, 1)) for f in (0.25, 0.5, 0.9)]
    with binding.SSHServer([ix], k=k, max_batch=64, max_slots=4, reserve_bytes=4 << 30) as srv:
        out["rates"] = serve_rates(srv, rates, 1.0 if small else 3.0, q_host, ins_pool, m,
                                   np.random.default_rng(9))
        st = srv.stats()
        out["slots"] = st["slots"]
    ix.close()
    return out


def run_gpu(args, w):
    import torch

    from paper_1610_07328_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    set_fp32_peak(torch.cuda.get_device_properties(dev).multi_processor_count, peaks()["sm_max_mhz"])
    N, m, nq, k = w["N"], w["m"], w["nq"], w["k"]

    # inputs: each rank holds its own N-series shard (weak scaling), pinned on the host and resident on the GPU
    t_gen = time.perf_counter()
    h_db = torch.empty((N, m), dtype=torch.float32, pin_memory=True)
    synth.random_walk(N, m, seed=w["seed"] + rank, out=h_db.numpy())
    sub = synth.random_walk(w["recall_subset"], m, seed=w["seed"])  # rank 0's first rows: query sources
    h_q_np, src = synth.perturbed_queries(sub, nq, seed=1)
    h_q = torch.from_numpy(h_q_np).pin_memory()
    d_db = h_db.to(dev, non_blocking=False)
    d_q = h_q.to(dev)
    d_ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
    d_dists = torch.empty((nq, k), dtype=torch.float32, device=dev)
    gen_s = time.perf_counter() - t_gen

    rss0 = host_rss_bytes()
    t_create = time.perf_counter()
    idx = binding.SSHIndex(w["W"], w["delta"], w["n"], w["K"], w["L"], w["band"], w["seed"])
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t_create
    create_rss = host_rss_bytes() - rss0
    stream = torch.cuda.current_stream()

    lengths = np.full(N, m, np.int32)
    qlengths = np.full(nq, m, np.int32)

    def exchange():
        """N > 1: the one exchange step of a sharded query (all-gather of every shard's
        top-k with global ids, merged on every rank)."""
        if not dist:
            return None
        from paper_1610_07328_gb300 import shard
        g_ids = torch.where(d_ids >= 0, d_ids + rank * N, d_ids)
        return shard.allgather_topk(g_ids, d_dists, k)

    def step():
        idx.clear()
        idx.add_device(d_db, lengths, borrow=True)
        idx.query_device(d_q, k, d_ids, d_dists, lengths=qlengths)
        exchange()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # per-kernel-group device times from three extra untimed steps: the events of
    # every group would add host work to the timed steps
    idx.reset_stats()
    idx.set_kernel_timing(True)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    times = idx.kernel_times()
    idx.set_kernel_timing(False)
    if dist:
        dist.barrier()
    idx.reset_stats()
    sampler = ClockSampler(gpu_bus_id(torch, dev))
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * args.steps + 2)]
    ev[0].record(stream)
    for s in range(args.steps):
        ev[1 + 3 * s].record(stream)
        idx.clear()
        idx.add_device(d_db, lengths, borrow=True)
        ev[2 + 3 * s].record(stream)
        idx.query_device(d_q, k, d_ids, d_dists, lengths=qlengths)
        exchange()
        ev[3 + 3 * s].record(stream)
    ev[-1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = ev[0].elapsed_time(ev[-1])
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    index_ms = statistics.mean(ev[1 + 3 * s].elapsed_time(ev[2 + 3 * s]) for s in range(args.steps))
    query_ms = statistics.mean(ev[2 + 3 * s].elapsed_time(ev[3 + 3 * s]) for s in range(args.steps))
    stats = idx.stats()
    ms_per_step = total_ms / args.steps
    value = N * world / (ms_per_step / 1000.0)

    # results of the last timed step, recall against exact DTW (untimed)
    res_ids = d_ids.cpu().numpy()
    rb = int(math.floor(np.float32(w["band"]) * np.float64(m)))
    rb = min(rb, m - 1)
    subset_rows = np.arange(w["recall_subset"], dtype=np.int64)
    extra = {}
    if rank == 0 and not args.no_recall:
        d_sub = d_db[: w["recall_subset"]] if w["seed"] + rank == w["seed"] else torch.from_numpy(sub).to(dev)
        with binding.SSHIndex(w["W"], w["delta"], w["n"], w["K"], w["L"], w["band"], w["seed"]) as sidx:
            sidx.add_device(d_sub.contiguous())
            s_ids = torch.empty_like(d_ids)
            s_d = torch.empty_like(d_dists)
            sidx.query_device(d_q, k, s_ids, s_d)
            s_ids = s_ids.cpu().numpy()
        exact_sub = exact_topk_gpu(binding, torch, d_q, d_sub.contiguous(), subset_rows, m, rb, k)
        extra["recall_at_10"] = recall(s_ids, exact_sub)
        extra["ndcg_at_10"] = ndcg(s_ids, exact_sub)
        extra["recall_at_1"] = float(np.mean([s_ids[i, 0] == exact_sub[i, 0] for i in range(nq)]))
        extra["recall_operating_point"] = recall_operating_point(binding, torch, d_sub.contiguous(), d_q,
                                                                 exact_sub, w, k)
        extra["parameter_study"] = parameter_study(binding, torch, d_sub.contiguous(), d_q, exact_sub, w, k)
        extra["srp_baseline"] = srp_baseline(binding, torch, d_sub.contiguous(), d_q, exact_sub, w, k)
        extra["minhash_variants"] = minhash_variants(binding, torch, d_db, d_sub.contiguous(), d_q, exact_sub, w, k)
        extra["dtw_full_load"] = dtw_full_load_measurement(binding, torch, d_db, d_q, w)
        extra["exact_scan"] = exact_scan_measurement(binding, torch, d_sub.contiguous(), d_db, d_q, exact_sub, w, k,
                                                     n_full=4 if args.small else 10)
        if not args.fast:
            n_full = min(nq, 20)
            exact_full = exact_topk_gpu(binding, torch, d_q[:n_full].contiguous(), d_db,
                                        np.arange(N, dtype=np.int64), m, rb, k)
            extra["recall_at_10_full_db"] = recall(res_ids[:n_full], exact_full)
            extra["recall_full_db_queries"] = n_full

    # single-query latency: the plain one-query-per-call path
    lat = []
    one_ids = torch.empty((1, k), dtype=torch.int64, device=dev)
    one_d = torch.empty((1, k), dtype=torch.float32, device=dev)
    for i in range(nq):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        idx.query_device(d_q[i:i + 1], k, one_ids, one_d)
        e1.record(stream)
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
    lat_sorted = sorted(lat)
    p50 = lat_sorted[len(lat) // 2]
    p99 = lat_sorted[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]

    # end to end through the public host API: H2D of the series and queries, D2H of the results
    h_db_np = h_db.numpy()
    h_q_np2 = h_q.numpy()
    qlen = qlengths
    e2e_steps = args.steps
    # warm-up: the first host add allocates the index's 2 GB staging copy, later
    # adds reuse it (ssh_index_clear keeps the buffer for the next add)
    for _ in range(max(1, min(args.warmup, 2))):
        idx.clear()
        binding.ssh_index_add(idx.handle, h_db_np, lengths)
        binding.ssh_query(idx.handle, h_q_np2, qlen, k)
    idx.clear()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        idx.clear()
        binding.ssh_index_add(idx.handle, h_db_np, lengths)
        ids_h, dists_h = binding.ssh_query(idx.handle, h_q_np2, qlen, k)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1000.0 / e2e_steps
    if dist:
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    idx.close()
    h2d_peak = h2d_copy_gbs(torch, h_db, d_db)

    pk = peaks()
    roofs = kernel_rooflines(w, times, pk)
    dominant = max((n for n in roofs if roofs[n].get("achieved") is not None and "ms_total" in roofs[n]),
                   key=lambda n: roofs[n]["ms_total"])
    d = roofs[dominant]
    roofline = {"kernel": dominant, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"],
                "unit": d["unit"], "frac": d["frac"], "traffic": traffic_for(dominant),
                "peak_source": pk["source"] if d["unit"] == "GB/s" else fp32_peak_source()}
    l2b = traffic_for(dominant, "l2_read_bytes_per_launch")
    if l2b:
        # the minhash kernel's binding resource: its L2 reads (rank-row gathers) per launch from the
        # ncu capture, over its CUDA-event time, against the L2 read bandwidth measured in this run
        l2_peak = l2_read_gbs(torch, dev, binding)
        ach = l2b / (d["avg_ms"] / 1000.0) / 1e9
        roofline["binding"] = {"resource": "L2 reads (gathers)", "bytes_per_launch": l2b, "achieved": ach,
                               "peak": l2_peak, "unit": "GB/s", "frac": ach / l2_peak,
                               "peak_source": "measured here: L1-bypassing reads of a 32 MB L2-resident buffer (ssh_read_device)"}

    line = {
        "metric": METRIC, "value": value, "unit": "series/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_desc(w), "N_per_gpu": N, "m": m, "W": w["W"], "delta": w["delta"],
                   "n": w["n"], "K": w["K"], "L": w["L"], "band": w["band"], "queries": nq, "k": k,
                   "parallelism": "one index shard per GPU" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (series %.2f GB per step)" % (N * m * 4 / 1e9),
                   "step": "index build of N series + one batch of nq queries"},
        "index_ms": index_ms, "query_ms": query_ms,
        "series_hashed_per_s_index_phase": N * world / (index_ms / 1000.0),
        "queries_per_s": nq / (query_ms / 1000.0),
        "latency_ms": {"p50": p50, "p99": p99, "mode": "one query per call on the built index"},
        "plain_gpu_path_queries_per_s": 1000.0 / statistics.mean(lat),
        "candidates_per_query": stats["candidates"] / max(stats["queries"], 1),
        "candidate_fraction": stats["candidates"] / max(stats["queries"], 1) / N,
        "dtw_per_query": stats["dtw_computed"] / max(stats["queries"], 1),
        "fp64_fallbacks": {"sketch_windows": stats["sketch_fp64"], "minhashes": stats["cws_fp64"]},
        "gpu_launches": stats["kernel_launches"],
        "roofline": roofline,
        "kernels": roofs,
        "e2e": {"value": N * world / (e2e_ms / 1000.0), "unit": "series/s",
                "h2d_bytes_per_step": N * m * 4 + nq * m * 4,
                "d2h_bytes_per_step": nq * k * 12, "steps": e2e_steps, "warmup": max(1, min(args.warmup, 2)),
                "ms_per_step": e2e_ms,
                "h2d_gbs": (N * m * 4 + nq * m * 4) / (e2e_ms / 1000.0) / 1e9,
                "h2d_peak_gbs": h2d_peak, "h2d_frac": (N * m * 4 + nq * m * 4) / (e2e_ms / 1000.0) / 1e9 / h2d_peak,
                "h2d_peak_source": "measured here: one pinned host-to-device copy of the series (best of 3)",
                "api": "ssh_index_clear + ssh_index_add(host) + ssh_query(host)"},
        "clocks": clocks,
        "setup_s": {"inputs": gen_s},
        "ssh_create": {"seconds": create_s, "host_rss_growth_bytes": create_rss,
                       "what": "ssh_create at n=%d, K*L=%d: filter on the host, draw tables built on the GPU"
                               % (w["n"], w["K"] * w["L"])},
        **extra,
    }
    if rank == 0 and world == 1 and not args.no_batched:
        line["batched"] = batched_measurement(args, binding, torch, dev)
    if rank == 0 and world == 1 and not args.no_served:
        line["served"] = serving_measurement(args, binding, torch, dev)
    if rank == 0 and world == 1 and not args.no_subsequence:
        line["subsequence"] = subsequence_measurement(args, binding, torch, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_s = 10000 if not args.small else 300
        r = oracle_sample(w, n_s, 10 if not args.small else 3)
        line["cpu_baseline"] = {"value": r["value"], "unit": "series/s", "cores": 1, "kind": "oracle",
                                "sample": r["sample"], "seconds": r["seconds"]}
        try:
            ra = oracle_sample_all_cores(w, n_s, 32 if not args.small else 8)
            line["cpu_baseline"]["all_cores"] = {"value": ra["value"], "unit": "series/s", "cores": ra["cores"],
                                                 "sample": ra["sample"], "seconds": ra["seconds"]}
        except Exception as e:  # reported, never fatal to the line
            line["cpu_baseline"]["all_cores"] = {"error": repr(e)[:200]}
    if rank == 0:
        detail = args.detail_out or os.path.join(ROOT, "gpurun_out", "bench_detail_n%d.json" % world)
        try:
            os.makedirs(os.path.dirname(detail), exist_ok=True)
            with open(detail, "w") as f:
                json.dump(line, f, indent=1)
        except OSError as e:  # the headline below still carries every contract key
            detail = "not written: %r" % (e,)
        print(json.dumps(headline(line, detail)), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------- fixed cases for ncu captures
#
#   python bench.py --profile-case hash 200000
#       hashes 200,000 random walks of length 512 with the scale parameters (W=80, delta=3,
#       n=15, K=4, L=25) through ssh_hash_device twice: the sketch, FP64 fix-up, shingle and
#       minhash kernels run once per call.
#   python bench.py --profile-case dtw 512:25 [reps]
#       banded DTW of 100 queries against 2,000,000 / m random candidates each (rows of a
#       random-walk table larger than L2) through ssh_dtw_device; prints the fastest call.
#   python bench.py --profile-case tables 262144
#       an index of 262,144 random walks of length 512 with the scale parameters, added twice.
#   python bench.py --profile-case batch 50000 1024
#       five per-length indexes (m = 128 .. 2048, W = m/8, delta=3, n=15, K=4, L=25) of 50,000
#       random walks each and three batches of 1,024 mixed-length queries through one plan.

def profile_hash(n: int) -> None:
    import torch
    from paper_1610_07328_gb300 import binding
    m = 512
    x = torch.from_numpy(synth.random_walk(n, m, seed=0)).cuda()
    with binding.SSHIndex(80, 3, 15, 4, 25, 0.05, 0) as idx:
        keys = torch.empty((25, n), dtype=torch.int64, device="cuda")
        for _ in range(2):
            binding.ssh_hash_device(idx.handle, x, m, n, d_keys=keys)
        torch.cuda.synchronize()
        print("hashed", n, "series twice;", idx.stats())


def profile_dtw(spec: str, reps: int) -> None:
    import torch
    from paper_1610_07328_gb300 import binding
    for case in spec.split(","):
        m, rb = (int(v) for v in case.split(":"))
        nb = max(20000, 400_000_000 // (4 * m))
        b = torch.from_numpy(synth.random_walk(nb, m, seed=1)).cuda()
        a = torch.from_numpy(synth.random_walk(100, m, seed=2)).cuda()
        cand = max(200, 2_000_000 // m)
        rng = np.random.default_rng(0)
        ai = torch.from_numpy(np.repeat(np.arange(100), cand).astype(np.int64)).cuda()
        bi = torch.from_numpy(rng.integers(0, nb, 100 * cand).astype(np.int64)).cuda()
        out = torch.empty(100 * cand, device="cuda")
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            binding.ssh_dtw_device(a, ai, b, bi, m, rb, out)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        cells = 100 * cand * (m * (2 * rb + 1) - rb * (rb + 1))
        print(f"m={m} rb={rb} pairs={100 * cand} call_ms={best:.3f} cells={cells}")


def profile_batch(n: int, nq: int) -> None:
    import torch
    from paper_1610_07328_gb300 import binding
    lens = (128, 256, 512, 1024, 2048)
    hosts = {m: synth.random_walk(n, m, seed=40 + m) for m in lens}
    idxs = [binding.SSHIndex(m // 8, 3, 15, 4, 25, 0.05, 0) for m in lens]
    data = {m: torch.from_numpy(hosts[m]).cuda() for m in lens}
    for ix, m in zip(idxs, lens):
        ix.add_device(data[m], borrow=True)
    rng = np.random.default_rng(4)
    qlens = rng.choice(np.array(lens, np.int32), size=nq)
    qs = [synth.perturbed_queries(hosts[m], 1, seed=1000 + i)[0][0] for i, m in enumerate(qlens)]
    d_q = torch.from_numpy(np.concatenate(qs)).cuda()
    ids = torch.empty((nq, 10), dtype=torch.int64, device="cuda")
    dd = torch.empty((nq, 10), dtype=torch.float32, device="cuda")
    with binding.SSHBatch(idxs, max_queries=nq, k=10) as bt:
        for _ in range(3):
            bt.query(d_q, qlens, ids, dd)
        torch.cuda.synchronize()
        print("batches done;", bt.stats())
    for ix in idxs:
        ix.close()


def profile_tables(n: int) -> None:
    import torch
    from paper_1610_07328_gb300 import binding
    x = torch.from_numpy(synth.random_walk(n, 512, seed=0)).cuda()
    with binding.SSHIndex(80, 3, 15, 4, 25, 0.05, 0) as idx:
        for _ in range(2):
            idx.clear()
            idx.add_device(x, borrow=True)
        torch.cuda.synchronize()
        print("built twice;", len(idx), "rows")



def run_profile_case(argv):
    if len(argv) >= 2 and argv[0] == "hash":
        profile_hash(int(argv[1]))
    elif len(argv) >= 2 and argv[0] == "tables":
        profile_tables(int(argv[1]))
    elif len(argv) >= 3 and argv[0] == "batch":
        profile_batch(int(argv[1]), int(argv[2]))
    elif len(argv) >= 2 and argv[0] == "dtw":
        profile_dtw(argv[1], int(argv[2]) if len(argv) > 2 else 3)
    else:
        raise SystemExit("unknown --profile-case %r" % (argv,))


def _r(x, nd=4):
    """Round a float for the headline (significant digits), leave other values alone."""
    if isinstance(x, float) and math.isfinite(x) and x != 0.0:
        return float("%.*g" % (nd, x))
    return x


def headline(line, detail_path):
    """The one short JSON line printed last: the contract keys plus the few figures that the
    detail file (every block of the run) summarises."""
    keep = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
            "scaling", "vs_baseline", "dtype", "data", "gpu_launches", "clocks")
    h = {k: line[k] for k in keep if k in line}
    h["value"] = float(line["value"])
    h["ms_per_step"] = _r(float(line["ms_per_step"]), 5)
    c = line["config"]
    h["config"] = {k: c[k] for k in ("workload", "parallelism", "l2") if k in c}
    r = line["roofline"]
    h["roofline"] = {k: _r(r[k]) for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "traffic")}
    if r.get("binding"):
        b = r["binding"]
        h["roofline"]["binding"] = {"resource": b["resource"], "achieved": _r(b["achieved"]), "peak": _r(b["peak"]),
                                    "frac": _r(b["frac"])}
    kr = line.get("kernels", {})
    if "add.hash_pipeline" in kr:
        h["hash_pipeline_hbm_frac"] = _r(kr["add.hash_pipeline"]["frac"])
    if "query.dtw" in kr:
        h["dtw_fp32_frac"] = _r(kr["query.dtw"].get("frac"))
    if isinstance(line.get("dtw_full_load"), dict) and "frac" in line["dtw_full_load"]:
        h["dtw_fp32_frac_full_load"] = _r(line["dtw_full_load"]["frac"])
    if "cpu_baseline" in line:
        cb = line["cpu_baseline"]
        h["cpu_baseline"] = {"value": _r(cb["value"]), "unit": cb["unit"], "cores": cb["cores"], "kind": cb["kind"],
                             "sample": cb["sample"]}
        if isinstance(cb.get("all_cores"), dict) and "value" in cb["all_cores"]:
            h["cpu_baseline"]["all_cores"] = {"value": _r(cb["all_cores"]["value"]),
                                              "cores": cb["all_cores"]["cores"]}
    e = line["e2e"]
    h["e2e"] = {k: _r(e[k]) for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step", "steps",
                                      "h2d_gbs", "h2d_peak_gbs", "h2d_frac") if k in e}
    h["queries_per_s"] = _r(line["queries_per_s"])
    if "ssh_create" in line:
        h["ssh_create_s"] = _r(line["ssh_create"]["seconds"])
    h["latency_ms"] = {"p50": _r(line["latency_ms"]["p50"]), "p99": _r(line["latency_ms"]["p99"])}
    for k in ("recall_at_10", "ndcg_at_10"):
        if k in line:
            h[k] = _r(line[k])
    rop = line.get("recall_operating_point", {}).get("chosen")
    if rop:
        h["at_recall_0_9"] = {"queries_per_s": _r(rop["queries_per_s"]), "recall_at_10": _r(rop["recall_at_10"]),
                              "params": "W=%d delta=%d n=%d K=%d L=%d" % (rop["W"], rop["delta"], rop["n"],
                                                                          rop["K"], rop["L"])}
    if "batched" in line:
        b = line["batched"]
        h["batched_queries_per_s"] = _r(b["batched_queries_per_s"])
        h["batched_graph_kernels"] = b.get("graph_kernels")
        if b.get("at_recall"):
            h["batched_at_recall_queries_per_s"] = _r(b["at_recall"]["batched_queries_per_s"])
    h["detail"] = os.path.relpath(detail_path, ROOT) if os.path.isabs(detail_path) else detail_path
    return h


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ssh", choices=["ssh", "reference"])
    ap.add_argument("--small", action="store_true", help="the tiny configuration (quick check)")
    ap.add_argument("--fast", action="store_true", help="skip the full-database recall")
    ap.add_argument("--no-recall", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the mixed-length batch-plan measurement")
    ap.add_argument("--no-served", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--no-subsequence", action="store_true", help="skip the sliding-window index measurement")
    ap.add_argument("--detail-out", default=None,
                    help="where the full measurement JSON goes (default gpurun_out/bench_detail_nN.json)")
    ap.add_argument("--profile-case", nargs="+", default=None,
                    help="run one fixed small case for an ncu capture (hash N | dtw m:rb[,m:rb] [reps] | "
                         "tables N | batch N nq) and exit")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    w = TINY if args.small else SCALE
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
