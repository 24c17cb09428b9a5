"""The autotuner's host side without a GPU: buckets and the JSON cache."""
import numpy as np
import pytest

from paper_1612_01506_gb300 import sm, synth, tune


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return sm.load()


def test_buckets(lib):
    # m bucket = ceil(log2 m)
    h = np.zeros(256, np.uint64)
    h[ord("a")] = h[ord("b")] = 10
    for m, mb in ((1, 0), (2, 1), (3, 2), (4, 2), (5, 3), (64, 6), (65, 7), (4096, 12)):
        assert sm.sm_tune_bucket(h, m) == (mb, 0)
    # sigma bucket: <= 2 symbols, <= 4 symbols, then the effective alphabet 1 / sum p^2
    for text, sb in ((synth.uniform(1 << 16, 4, seed=0, stream=1), 1),
                     (np.random.default_rng(0).integers(97, 105, 1 << 16).astype(np.uint8), 2),
                     (synth.uniform(1 << 16, 20, seed=0, stream=1), 3),
                     (synth.uniform(1 << 16, 64, seed=0, stream=1), 4),
                     (synth.markov95(1 << 18, seed=0, stream=1), 3)):
        hist = np.bincount(text, minlength=256).astype(np.uint64)
        assert sm.sm_tune_bucket(hist, 8)[1] == sb
    with pytest.raises(sm.SmError):
        sm.sm_tune_bucket(h, 0)
    with pytest.raises(sm.SmError):
        sm.sm_tune_bucket(h, sm.SM_MAX_M + 1)


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    assert tune.read_entries(path, "gpu") == []
    a = [{"m_bucket": 1, "sigma_bucket": 3, "peel": 2, "stages": 0, "ctas_per_sm": 0, "ms": 0.2},
         {"m_bucket": 3, "sigma_bucket": 3, "peel": 0, "stages": 3, "ctas_per_sm": 2, "ms": 0.19}]
    tune.write_entries(path, "gpu", a)
    tune.write_entries(path, "other", a[:1])
    # a new entry for a bucket replaces the old one; other buckets and keys stay
    tune.write_entries(path, "gpu", [{"m_bucket": 1, "sigma_bucket": 3, "peel": 5, "stages": 2, "ctas_per_sm": 1,
                                      "ms": 0.18}])
    got = tune.read_entries(path, "gpu")
    assert [(e["m_bucket"], e["peel"], e["stages"], e["ctas_per_sm"]) for e in got] == [(1, 5, 2, 1), (3, 0, 3, 2)]
    assert len(tune.read_entries(path, "other")) == 1
    # malformed entries are skipped
    with open(path, "w") as f:
        f.write('{"gpu": [{"m_bucket": 1}, {"m_bucket": 2, "sigma_bucket": 4, "peel": "x"}]}')
    assert tune.read_entries(path, "gpu") == []
