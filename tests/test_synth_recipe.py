"""The seeded input recipe that stands in for the paper's Random Walk and ECG collections
(Sec. 5.1): shapes, normalisation, determinism and the query perturbation it states."""
import numpy as np

from paper_1610_07328_gb300 import synth


def test_random_walks_are_z_normalised_and_deterministic():
    x = synth.random_walk(200, 512, seed=5)
    assert x.shape == (200, 512) and x.dtype == np.float32
    assert np.abs(x.mean(axis=1)).max() < 1e-5
    assert np.abs(x.std(axis=1) - 1.0).max() < 1e-4
    assert np.array_equal(x, synth.random_walk(200, 512, seed=5))
    assert not np.array_equal(x, synth.random_walk(200, 512, seed=6))
    # rows are generated in fixed chunks: a prefix of a larger draw is the smaller draw
    assert np.array_equal(synth.random_walk(50, 512, seed=5), x[:50])
    # a random walk's increments are the (normalised) N(0, 1) steps: lag-1 correlation near 1
    r = [np.corrcoef(row[:-1], row[1:])[0, 1] for row in x[:50]]
    assert min(r) > 0.9


def test_ecg_like_beats_have_the_stated_periods():
    x = synth.ecg_like(40, 1024, seed=3)
    assert x.shape == (40, 1024) and x.dtype == np.float32
    assert np.array_equal(x, synth.ecg_like(40, 1024, seed=3))
    for row in x:
        # QRS peaks (amplitude 1.0 against P 0.15, T 0.3, wander 0.1, noise 0.05): local maxima above 0.6
        peaks = [i for i in range(3, len(row) - 3) if row[i] > 0.6 and row[i] == row[i - 3:i + 4].max()]
        gaps = np.diff(peaks)
        assert len(peaks) >= 3
        assert gaps.min() >= 170 and gaps.max() <= 270  # periods uniform in [180, 260], +- noise


def test_perturbed_queries_are_shifted_noisy_copies():
    db = synth.random_walk(100, 256, seed=1)
    q, src = synth.perturbed_queries(db, 30, seed=2)
    assert q.shape == (30, 256) and q.dtype == np.float32 and src.dtype == np.int64
    assert np.array_equal(q, synth.perturbed_queries(db, 30, seed=2)[0])
    for qi, s in zip(q, src):
        # the circular shift in 0..8 that best explains the query, and the residual's spread
        res = [np.std(qi.astype(np.float64) - np.roll(db[s], k)) for k in range(0, 9)]
        k = int(np.argmin(res))
        assert 0 <= k <= 8
        assert abs(res[k] - 0.1) < 0.03
    q2, src2 = synth.perturbed_queries(db, 30, seed=2, source_range=10)
    assert src2.max() < 10
