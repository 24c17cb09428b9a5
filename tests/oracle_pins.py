"""Pins that tie the oracle to facts other than itself.

Each ``pin_*`` takes an ``oracle.Oracle`` and raises AssertionError when the
oracle disagrees with the paper's worked example, a closed form, a brute
force computed independently here (numpy sliding windows), or an invariant
of the problem. ``test_oracle.py`` runs every pin on the real oracle;
``test_oracle_mutants.py`` plants plausible mistakes in a copy of the oracle
and checks that some pin fails for each.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_kv(name):
    kv = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    return kv


def _rng_bytes(seed, n, sigma):
    r = np.random.default_rng(seed)
    return r.integers(0, sigma, size=n, dtype=np.uint8) if sigma < 256 else r.integers(0, 256, size=n, dtype=np.uint8)


def brute_positions(p: bytes, t: np.ndarray) -> np.ndarray:
    """All starts s with t[s:s+m] == p, via numpy sliding windows."""
    pa = np.frombuffer(p, dtype=np.uint8)
    m, n = pa.size, t.size
    if m > n:
        return np.zeros(0, dtype=np.uint64)
    win = np.lib.stride_tricks.sliding_window_view(t, m)
    return np.nonzero((win == pa).all(axis=1))[0].astype(np.uint64)


# ---------------------------------------------------------------- paper values

def pin_fig1(o):
    g = _golden_kv("fig1.txt")
    t, p = g["text"].encode(), g["pattern"].encode()
    want_pos = [int(x) for x in g["positions"].split()]
    assert o.naive_count(p, t) == int(g["count"])
    pos, c = o.naive_report(p, t)
    assert c == int(g["count"]) and list(pos) == want_pos
    assert o.kmp_count(p, t) == int(g["count"])
    assert o.memcmp_count(p, t) == int(g["count"])


def pin_order_h_golden(o):
    with open(os.path.join(GOLDEN, "order_h.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            m, order = line.split(":")
            want = [int(x) - 1 for x in order.split()]
            assert list(o.order_h(int(m))) == want, (m, list(o.order_h(int(m))))


# ---------------------------------------------------------------- closed forms

def pin_runs(o):
    # a^m in a^n occurs n-m+1 times (overlaps count), and 0 times when m > n
    for n in (0, 1, 2, 7, 64, 1000):
        t = b"a" * n
        for m in (1, 2, 3, 7, 64, 999, 1000, 1001):
            want = max(n - m + 1, 0)
            assert o.naive_count(b"a" * m, t) == want, (n, m)
            assert o.kmp_count(b"a" * m, t) == want, (n, m)
    assert o.naive_count(b"aaaa", b"aaaaaaa") == 4
    # (ab)^j in (ab)^k occurs k-j+1 times; (ab)^j b never
    for k in (1, 5, 40):
        for j in range(1, k + 1):
            assert o.naive_count(b"ab" * j, b"ab" * k) == k - j + 1
            assert o.naive_count(b"ab" * j + b"b", b"ab" * k) == 0


def pin_single_symbol_is_histogram(o):
    # m = 1: the count of pattern c equals the number of c bytes in t
    for seed, sigma, n in ((1, 2, 5000), (2, 4, 7777), (3, 256, 20000)):
        t = _rng_bytes(seed, n, sigma)
        h = o.histogram(t)
        ref = np.bincount(t, minlength=256).astype(np.uint64)
        assert np.array_equal(h, ref)
        assert int(h.sum()) == n
        for c in range(256):
            assert o.naive_count(bytes([c]), t) == int(ref[c]), c


def pin_all_patterns_partition(o):
    # every start matches exactly one of the sigma^m patterns of length m
    import itertools
    for seed, sigma, n, ms in ((4, 2, 300, (1, 2, 3, 4, 5, 6)), (5, 3, 257, (1, 2, 3, 4)), (6, 4, 500, (1, 2, 3, 4))):
        t = _rng_bytes(seed, n, sigma)
        for m in ms:
            total = sum(o.naive_count(bytes(w), t) for w in itertools.product(range(sigma), repeat=m))
            assert total == n - m + 1, (sigma, m, total)


# ---------------------------------------------------------------- brute force

def pin_brute_tiny(o):
    r = np.random.default_rng(7)
    for sigma in (1, 2, 4, 256):
        for n in (0, 1, 2, 3, 15, 16, 17, 63, 200):
            t = _rng_bytes(int(r.integers(1 << 30)), n, sigma) if sigma > 1 else np.zeros(n, np.uint8)
            for m in range(1, n + 2):
                if n and r.random() < 0.5 and m <= n:
                    s = int(r.integers(0, n - m + 1))
                    p = t[s:s + m].tobytes()
                else:
                    p = (_rng_bytes(int(r.integers(1 << 30)), m, sigma) if sigma > 1 else np.zeros(m, np.uint8)).tobytes()
                want = brute_positions(p, t)
                c = o.naive_count(p, t)
                assert c == want.size, (sigma, n, m)
                assert o.memcmp_count(p, t) == c
                assert o.kmp_count(p, t) == c
                pos, c2 = o.naive_report(p, t)
                assert c2 == c and np.array_equal(pos, want)


def pin_report_cap(o):
    t = np.frombuffer(b"ab" * 50, dtype=np.uint8)
    for cap in (0, 1, 7, 49, 50, 51, 100):
        pos, c = o.naive_report(b"ab", t, cap)
        assert c == 50
        assert list(pos) == [2 * i for i in range(min(cap, 50))]


def pin_sampled_patterns_found(o):
    t = _rng_bytes(11, 100_000, 4)
    r = np.random.default_rng(12)
    for m in (2, 8, 31, 64, 500):
        for _ in range(5):
            s = int(r.integers(0, t.size - m + 1))
            p = t[s:s + m].tobytes()
            pos, c = o.naive_report(p, t)
            assert c >= 1 and s in set(int(x) for x in pos)
            assert np.array_equal(pos, brute_positions(p, t))


def pin_threads(o):
    t = _rng_bytes(13, 1_000_003, 2)
    for m in (1, 2, 5, 17, 1000):
        p = t[777:777 + m].tobytes()
        c = o.naive_count(p, t)
        for th in (1, 3, 8, 64):
            assert o.count_threads(p, t, th) == c
        full, c1 = o.naive_report(p, t)
        for th, cap in ((4, c), (7, c // 2), (5, 0)):
            pos, c2 = o.report_threads(p, t, cap, th)
            assert c2 == c and np.array_equal(pos, full[:cap])


# ---------------------------------------------------------------- orders

def pin_order_freq(o):
    r = np.random.default_rng(21)
    h = np.zeros(256, dtype=np.uint64)
    assert list(o.order_freq(b"abcd", h)) == [0, 1, 2, 3]        # all ties: ascending position
    h[ord("a")], h[ord("b")], h[ord("c")] = 30, 10, 20
    assert list(o.order_freq(b"abcab", h)) == [1, 4, 2, 0, 3]    # b, b, c, a, a
    for m in (1, 2, 5, 64, 1000, 4096):
        hist = r.integers(0, 50, size=256).astype(np.uint64)
        p = r.integers(0, 256, size=m, dtype=np.uint8)
        pi = o.order_freq(p, hist).astype(np.int64)
        keys = hist[p].astype(np.int64)
        assert sorted(pi.tolist()) == list(range(m))
        assert np.array_equal(pi, np.lexsort((np.arange(m), keys)))


def pin_order_h(o):
    for m in range(1, 300):
        pi = o.order_h(m)
        assert sorted(pi.tolist()) == list(range(m))
        if m >= 2:
            assert pi[0] == 0 and pi[1] == m - 1


def pin_order_hs(o):
    r = np.random.default_rng(31)
    for m in (1, 2, 3, 10, 57, 200):
        p = r.choice(np.frombuffer(b"ab c", dtype=np.uint8), size=m)
        pi = o.order_hs(p).tolist()
        assert sorted(pi) == list(range(m))
        spaces = [q for q in range(m) if p[q] == 0x20]
        rest = [q for q in range(m) if p[q] != 0x20]
        assert pi[len(rest):] == spaces
        assert pi[:len(rest)] == [rest[i] for i in o.order_h(len(rest))]
    # no spaces: pi_hs is pi_h
    assert list(o.order_hs(b"abcdefghij")) == list(o.order_h(10))


# ---------------------------------------------------------------- batches

def pin_batch(o):
    r = np.random.default_rng(41)
    texts = [_rng_bytes(int(r.integers(1 << 30)), int(n), 4) for n in (0, 5, 100, 3000)]
    text_off = np.cumsum([0] + [t.size for t in texts]).astype(np.int64)
    flat = np.concatenate(texts) if texts else np.zeros(0, np.uint8)
    pats, pat_text = [], []
    for x, t in enumerate(texts):
        for m in (1, 2, 7):
            if t.size >= m:
                s = int(r.integers(0, t.size - m + 1))
                pats.append(t[s:s + m].tobytes())
            else:
                pats.append(b"A" * m)
            pat_text.append(x)
    pat_off = np.cumsum([0] + [len(p) for p in pats]).astype(np.int64)
    counts = o.batch_count(flat, text_off, np.frombuffer(b"".join(pats), np.uint8), pat_off, np.array(pat_text))
    for k, p in enumerate(pats):
        assert counts[k] == brute_positions(p, texts[pat_text[k]]).size


ALL_PINS = [pin_fig1, pin_order_h_golden, pin_runs, pin_single_symbol_is_histogram,
            pin_all_patterns_partition, pin_brute_tiny, pin_report_cap, pin_sampled_patterns_found,
            pin_threads, pin_order_freq, pin_order_h, pin_order_hs, pin_batch]
