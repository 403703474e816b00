"""Small, fixed workloads for profiling single kernels under ncu.

    python -m paper_1610_07328_gb300.profile_cases hash 200000
        hashes 200,000 random walks of length 512 with the scale parameters
        (W=80, delta=3, n=15, K=4, L=25) through ssh_hash_device twice: the
        sketch, FP64 fix-up, shingle and minhash kernels run once per call.
    python -m paper_1610_07328_gb300.profile_cases dtw 512:25 [reps]
        banded DTW of 100 queries against 2,000,000 / m random candidates
        each (rows of a random-walk table larger than L2) through
        ssh_dtw_device; prints the call time of the fastest repetition.

    python -m paper_1610_07328_gb300.profile_cases tables 262144
        an index of 262,144 random walks of length 512 with the scale
        parameters, added twice (two table builds of 25 x 262,144 entries).
    python -m paper_1610_07328_gb300.profile_cases batch 50000 1024
        five per-length indexes (m = 128 .. 2048, W = m/8, delta=3, n=15, K=4,
        L=25) of 50,000 random walks each and three batches of 1,024 mixed-length
        queries through one batch plan: the first runs directly, the others
        replay the captured CUDA graph.

Every input is seeded and synthetic; nothing here is on the library's path.
"""
from __future__ import annotations

import sys

import numpy as np


def _hash(n: int) -> None:
    import torch
    from . import binding, synth
    m = 512
    x = torch.from_numpy(synth.random_walk(n, m, seed=0)).cuda()
    with binding.SSHIndex(80, 3, 15, 4, 25, 0.05, 0) as idx:
        keys = torch.empty((25, n), dtype=torch.int64, device="cuda")
        for _ in range(2):
            binding.ssh_hash_device(idx.handle, x, m, n, d_keys=keys)
        torch.cuda.synchronize()
        print("hashed", n, "series twice;", idx.stats())


def _dtw(spec: str, reps: int) -> None:
    import torch
    from . import binding, synth
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


def _batch(n: int, nq: int) -> None:
    import torch
    from . import binding, synth
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


def _tables(n: int) -> None:
    import torch
    from . import binding, synth
    x = torch.from_numpy(synth.random_walk(n, 512, seed=0)).cuda()
    with binding.SSHIndex(80, 3, 15, 4, 25, 0.05, 0) as idx:
        for _ in range(2):
            idx.clear()
            idx.add_device(x, borrow=True)
        torch.cuda.synchronize()
        print("built twice;", len(idx), "rows")


def main(argv: list[str]) -> None:
    if len(argv) >= 2 and argv[0] == "hash":
        _hash(int(argv[1]))
    elif len(argv) >= 2 and argv[0] == "tables":
        _tables(int(argv[1]))
    elif len(argv) >= 3 and argv[0] == "batch":
        _batch(int(argv[1]), int(argv[2]))
    elif len(argv) >= 2 and argv[0] == "dtw":
        _dtw(argv[1], int(argv[2]) if len(argv) > 2 else 3)
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    main(sys.argv[1:])
