"""The benchmark's last stdout line: a short headline with the contract's keys, whatever the
run's clock record holds (the full measurement goes to the detail file)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _full_line():
    """A full measurement line of the scale workload, with the longest strings the bench writes."""
    sample = ("oracle indexed 10000 series and answered 10 queries on them; step time extrapolated as "
              "N*t_hash + nq*t_query*N/10000")
    return {
        "metric": bench.METRIC, "value": 186495018.55175248, "unit": "series/s", "n_gpus": 1, "steps": 10,
        "warmup": 3, "ms_per_step": 5.362073516845703, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "gpu_launches": 340,
        "clocks": {"sm_mhz": 1965.0, "sm_max_mhz": 2070.0,
                   "reasons": ["sw_power_cap", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"],
                   "samples": 2},
        "config": {"workload": bench.workload_desc(bench.SCALE), "parallelism": "single GPU",
                   "l2": "inputs larger than L2 (series 2.05 GB per step)", "recall_subset": 10000},
        "roofline": {"kernel": "add.cws", "bound": "hbm", "achieved": 295.4832, "peak": 6790.0, "unit": "GB/s",
                     "frac": 0.043517, "traffic": 714453760.0, "peak_source": "measured",
                     "binding": {"resource": "L2 reads (gathers)", "bytes_per_launch": 23231502560.0,
                                 "achieved": 9481.93, "peak": 19168.48, "unit": "GB/s", "frac": 0.49466,
                                 "peak_source": "measured here: L1-bypassing reads of a 32 MB L2-resident buffer"}},
        "kernels": {"add.hash_pipeline": {"frac": 0.086093}, "query.dtw": {"frac": 0.062119}},
        "cpu_baseline": {"value": 764.0447, "unit": "series/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "seconds": 11.9, "all_cores": {"value": 9748.85, "unit": "series/s", "cores": 16,
                                                        "sample": sample, "seconds": 0.85}},
        "e2e": {"value": 84106303.9, "unit": "series/s", "h2d_bytes_per_step": 2048204800, "d2h_bytes_per_step": 12000,
                "steps": 10, "warmup": 2, "ms_per_step": 11.89, "h2d_gbs": 172.26, "h2d_peak_gbs": 211.47,
                "h2d_frac": 0.8146, "h2d_peak_source": "measured here", "api": "ssh_index_add(host) + ssh_query(host)"},
        "queries_per_s": 115277.07, "ssh_create": {"seconds": 0.0068},
        "latency_ms": {"p50": 0.40864, "p99": 0.59648, "mode": "one query per call on the built index"},
        "recall_at_10": 0.009, "ndcg_at_10": 0.02703,
        "recall_operating_point": {"chosen": {"W": 40, "delta": 3, "n": 10, "K": 4, "L": 25, "recall_at_10": 0.925,
                                              "queries_per_s": 90503.63}},
        "batched": {"batched_queries_per_s": 12936.91, "graph_kernels": 56,
                    "at_recall": {"batched_queries_per_s": 3285.26}},
        "served": {"rates": [{"offered_qps": q, "p50_ms": 1.5, "p99_ms": 9.9} for q in (1000, 5000, 20000, 50000)]},
        "dtw_full_load": {"frac": 0.27123, "tflops": 21.71, "cells_per_s": 7.24e12},
    }


def test_headline_is_short_and_carries_the_contract_keys():
    h = bench.headline(_full_line(), "gpurun_out/bench_detail_n1.json")
    text = json.dumps(h)
    assert len(text) < 2048
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "gpu_launches", "clocks", "roofline", "cpu_baseline", "e2e"):
        assert key in h, key
    assert h["config"]["workload"].startswith("plain SSH at scale")
    assert h["value"] == 186495018.55175248
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in h["roofline"], key
    for key in ("value", "unit", "cores", "kind", "sample"):
        assert key in h["cpu_baseline"], key
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in h["e2e"], key
    assert json.loads(text) == h


def test_algorithmic_bytes_per_series_follow_the_sketch_geometry():
    """Per-series bytes of the hash kernels at the scale shape (m=512, W=80, delta=3, n=15, L=25):
    N_B = floor((m - W) / delta) + 1 = 145 sign bits (5 words), S = N_B - n + 1 = 131 shingles."""
    w = bench.SCALE
    assert bench.algorithmic(w, "sketch") == ("hbm", 4 * 512 + 4 * 5)
    assert bench.algorithmic(w, "shingle") == ("hbm", 4 * 5 + 4 * 131)
    assert bench.algorithmic(w, "cws") == ("hbm", 4 * 131 + 8 * 25)
    assert bench.algorithmic(w, "table_sort") == ("hbm", 20)
    assert bench.algorithmic(w, "dtw") == ("alu", 3)
    assert bench.algorithmic(w, "probe_union") == (None, None)


def test_kernel_rooflines_divide_algorithmic_work_by_the_event_time():
    bench.set_fp32_peak(152, 2070.0)
    times = {"add.cws": {"total_ms": 3 * 2.45, "calls": 3, "launches": 3, "units": 3e6},
             "query.dtw": {"total_ms": 2.0, "calls": 2, "launches": 2, "units": 2e9},
             "query.probe_union": {"total_ms": 0.5, "calls": 2, "launches": 4, "units": 50.0}}
    out = bench.kernel_rooflines(bench.SCALE, times, {"hbm_gbs": 6790.0})
    cws = out["add.cws"]
    assert cws["avg_ms"] == 2.45 and cws["units_per_call"] == 1e6
    assert abs(cws["achieved"] - 1e6 * 724 / 2.45e-3 / 1e9) < 1e-9
    assert abs(cws["frac"] - cws["achieved"] / 6790.0) < 1e-12
    dtw = out["query.dtw"]
    assert dtw["unit"] == "TFLOP/s" and abs(dtw["achieved"] - 3.0) < 1e-12
    assert abs(dtw["peak"] - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9
    assert out["query.probe_union"]["achieved"] is None
    pipe = out["add.hash_pipeline"]  # only the minhash was timed here: the series read + keys written
    assert abs(pipe["achieved"] - 1e6 * (4 * 512 + 8 * 25) / 2.45e-3 / 1e9) < 1e-9


def test_reference_arm_prints_its_contract_line():
    """`bench.py --impl reference` times the CPU oracle on a slice of the workload per step and
    prints one JSON line last, with the step it actually timed as ms_per_step."""
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    last = r.stdout.strip().splitlines()[-1]
    assert len(last) < 2048
    line = json.loads(last)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["unit"] == "series/s" and line["steps"] == 1 and line["warmup"] == 0
    series, queries = 1000, 100
    assert "%d series + %d queries per step" % (series, queries) in line["config"]["workload"]
    assert abs(line["value"] - series / (line["ms_per_step"] / 1000.0)) <= 1e-6 * line["value"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
