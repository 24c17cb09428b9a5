"""Input generators: determinism, thread invariance, alphabets, stationarity."""
import numpy as np

from paper_1612_01506_gb300 import synth


def test_uniform_deterministic_and_thread_invariant():
    a = synth.uniform(3_000_001, 4, seed=0, stream=9, threads=1)
    b = synth.uniform(3_000_001, 4, seed=0, stream=9, threads=7)
    c = synth.uniform(3_000_001, 4, seed=0, stream=10, threads=7)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert set(np.unique(a).tolist()) == set(b"ACGT")


def test_uniform_frequencies():
    for sigma in (2, 4, 20, 64, 256):
        t = synth.uniform(1 << 20, sigma, seed=1, stream=sigma)
        counts = np.bincount(t, minlength=256)[np.frombuffer(synth.ALPHABETS[sigma], np.uint8)]
        e = t.size / sigma
        assert np.all(np.abs(counts - e) < 6 * np.sqrt(e)), sigma


def test_markov_deterministic_and_stationary():
    n = 3 * 65536 + 1234
    a = synth.markov95(n, seed=0, stream=3, threads=1)
    b = synth.markov95(n, seed=0, stream=3, threads=5)
    assert np.array_equal(a, b)
    assert a.min() >= 0x20 and a.max() <= 0x7E
    t = synth.markov95(1 << 24, seed=0, stream=4)
    w = synth.markov95_weights(0).astype(np.float64)
    q = w / w.sum()
    f = np.bincount(t, minlength=256) / t.size
    assert np.abs(f - q).max() < 2e-3
    # Zipf(s=1) by rank with the space first
    ranked = np.sort(q[q > 0])[::-1]
    assert np.argmax(q) == 0x20
    zipf = 1.0 / np.arange(1, 96)
    zipf /= zipf.sum()
    assert np.abs(ranked - zipf).max() < 1e-3
    # neighbours are correlated but runs are rare
    assert np.mean(t[1:] == t[:-1]) < 0.1


def test_patterns():
    t = synth.uniform(10_000, 20, seed=0, stream=1)
    offs = synth.sample_offsets(t.size, 16, 50, 0, 2)
    pats = synth.sample_patterns(t, 16, 50, 0, 2)
    assert all(pats[i] == t[int(offs[i]):int(offs[i]) + 16].tobytes() for i in range(50))
    rp = synth.random_patterns(b"ACGT", 9, 20, 0, 3)
    assert all(len(p) == 9 and set(p) <= set(b"ACGT") for p in rp)
