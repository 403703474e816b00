"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only (no hashing, no DTW): the tests feed
the same arrays to the CUDA library and to the CPU oracle, and the benchmark
uses the same recipes. Random numbers come from numpy's PCG64 with explicit
seeds, generated in fixed-size chunks so a given (seed, N, m) always yields the
same array.

The paper evaluates on the UCR Random Walk and ECG collections (Sec. 5.1),
which are not available here; these generators stand in for them:

* ``random_walk``: cumulative sum of N(0,1) steps, z-normalised per series.
* ``ecg_like``: a train of beats, each the sum of three Gaussian bumps
  (P, QRS, T) with jittered period, plus baseline wander and noise.
* ``perturbed_queries``: a stored series plus N(0, sigma^2) noise, circularly
  shifted by a uniform 0..max_shift samples.
"""
from __future__ import annotations

import numpy as np

_CHUNK = 65536


def _chunks(N: int):
    for start in range(0, N, _CHUNK):
        yield start, min(N, start + _CHUNK)


def znorm(x: np.ndarray) -> np.ndarray:
    """Per-row z-normalisation (rows with zero spread are only centred)."""
    x = np.asarray(x, dtype=np.float64)
    mu = x.mean(axis=-1, keepdims=True)
    sd = x.std(axis=-1, keepdims=True)
    sd = np.where(sd > 0, sd, 1.0)
    return (x - mu) / sd


def random_walk(N: int, m: int, seed: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """[N, m] float32 random walks, z-normalised per series."""
    if out is None:
        out = np.empty((N, m), dtype=np.float32)
    for c, (a, b) in enumerate(_chunks(N)):
        rng = np.random.Generator(np.random.PCG64([seed, c]))
        steps = rng.standard_normal((b - a, m))
        out[a:b] = znorm(np.cumsum(steps, axis=1)).astype(np.float32)
    return out


def ecg_like(N: int, m: int, seed: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """[N, m] float32 ECG-like beat trains (not z-normalised).

    Beat = P (sigma 8, amp 0.15, at -0.2 period) + QRS (sigma 3, amp 1.0, at 0)
    + T (sigma 12, amp 0.3, at +0.3 period); periods uniform in [180, 260];
    first beat offset uniform in [0, 64]; baseline wander 0.1 sin(2 pi t / T_w + phi)
    with T_w uniform in [700, 1200]; noise N(0, 0.05^2).
    """
    if out is None:
        out = np.empty((N, m), dtype=np.float32)
    t = np.arange(m, dtype=np.float64)
    max_beats = m // 180 + 3
    for c, (a, b) in enumerate(_chunks(N)):
        rng = np.random.Generator(np.random.PCG64([seed, 1_000_003, c]))
        n = b - a
        periods = rng.uniform(180.0, 260.0, size=(n, max_beats))
        offset = rng.uniform(0.0, 64.0, size=(n, 1))
        centres = offset + np.concatenate([np.zeros((n, 1)), np.cumsum(periods[:, :-1], axis=1)], axis=1)
        x = np.zeros((n, m), dtype=np.float64)
        for beat in range(max_beats):
            c0 = centres[:, beat:beat + 1]
            p = periods[:, beat:beat + 1]
            for rel, sig, amp in ((-0.2, 8.0, 0.15), (0.0, 3.0, 1.0), (0.3, 12.0, 0.3)):
                mu = c0 + rel * p
                x += amp * np.exp(-0.5 * ((t[None, :] - mu) / sig) ** 2)
        tw = rng.uniform(700.0, 1200.0, size=(n, 1))
        phi = rng.uniform(0.0, 2.0 * np.pi, size=(n, 1))
        x += 0.1 * np.sin(2.0 * np.pi * t[None, :] / tw + phi)
        x += rng.normal(0.0, 0.05, size=(n, m))
        out[a:b] = x.astype(np.float32)
    return out


def perturbed_queries(db: np.ndarray, nq: int, seed: int = 1, noise: float = 0.1, max_shift: int = 8,
                      source_range: int | None = None):
    """Queries made from stored series: (queries [nq, m] float32, source row indices).

    Each query is row src of ``db`` plus N(0, noise^2) noise, circularly shifted
    by a uniform integer in [0, max_shift]; it is not re-normalised.
    ``source_range`` restricts the sources to rows [0, source_range).
    """
    rng = np.random.Generator(np.random.PCG64([seed, 7]))
    n_src = db.shape[0] if source_range is None else min(source_range, db.shape[0])
    src = rng.integers(0, n_src, size=nq)
    shifts = rng.integers(0, max_shift + 1, size=nq)
    q = db[src].astype(np.float64) + rng.normal(0.0, noise, size=(nq, db.shape[1]))
    for i in range(nq):
        q[i] = np.roll(q[i], int(shifts[i]))
    return q.astype(np.float32), src.astype(np.int64)
