"""GPU parity of histogram, count and report against the CPU oracle (bit-exact).

Every call goes through the C ABI (ctypes binding). Inputs are seeded and
synthetic; expected values come from the oracle only.
"""
import numpy as np
import pytest

import oracle
from paper_1612_01506_gb300 import sm, synth

pytestmark = pytest.mark.gpu

TILE = sm.SM_TILE_STARTS


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    import __graft_entry__
    __graft_entry__.build()
    return sm.sm_create(0)


def to_dev(torch, host: np.ndarray, offset: int = 0):
    """Copy host bytes to the device at a chosen misalignment."""
    buf = torch.zeros(host.size + offset + 64, dtype=torch.uint8, device="cuda")
    if host.size:
        buf[offset:offset + host.size] = torch.from_numpy(host).cuda()
    return buf[offset:offset + host.size]


def gpu_count(ctx, text, p, **kw):
    c = sm.sm_count(ctx, text, p, **kw)
    assert sm.sm_sync(ctx) == sm.SM_OK
    return int(c.item())


def gpu_report(ctx, text, p, cap, **kw):
    pos, c = sm.sm_report(ctx, text, p, cap, **kw)
    st = sm.sm_sync(ctx)
    n = int(c.item())
    return pos[: min(n, cap)].cpu().numpy().view(np.uint64), n, st


def host_text(kind, n, seed):
    if kind == "ones":
        return np.full(n, ord("a"), dtype=np.uint8)
    return synth.text(kind, n, seed=0, stream=seed)


def patterns_for(t, m, r, k=2):
    out = []
    for _ in range(k):
        if t.size >= m:
            s = int(r.integers(0, t.size - m + 1))
            out.append(t[s:s + m].tobytes())
    out.append(bytes(r.integers(0, 256, size=m, dtype=np.uint8)))
    return out


# ------------------------------------------------------------------ histogram

@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 1000, TILE + 5, (1 << 20) + 7])
@pytest.mark.parametrize("offset", [0, 1, 15])
def test_histogram(torch, ctx, n, offset):
    for kind in (2, 256):
        t = host_text(kind, n, n + offset)
        h = sm.sm_histogram(ctx, to_dev(torch, t, offset))
        assert sm.sm_sync(ctx) == sm.SM_OK
        assert np.array_equal(h.cpu().numpy().view(np.uint64), oracle.histogram(t))


# ------------------------------------------------------------------ count edges

EDGE_N = [1, 2, 15, 16, 17, 100, TILE - 1, TILE, TILE + 1, 3 * TILE + 777]
EDGE_M = [1, 2, 3, 4, 5, 15, 16, 17, 31, 32, 33, 63, 64, 65, 100, 1000, 4096]


@pytest.mark.parametrize("kind", ["ones", 2, 4, 256])
@pytest.mark.parametrize("n", EDGE_N)
def test_count_edges(torch, ctx, kind, n):
    r = np.random.default_rng(n)
    t = host_text(kind, n, n)
    for offset in (0, 3, 13):
        text = to_dev(torch, t, offset)
        for m in EDGE_M:
            if m > n + 1:
                continue
            for p in patterns_for(t, m, r, k=1):
                assert gpu_count(ctx, text, p) == oracle.naive_count(p, t), (kind, n, offset, m, p[:16])


@pytest.mark.parametrize("n", [TILE + 63, 2 * TILE + 64, 4 * TILE + 4096 + 3])
def test_count_tile_halo_boundaries(torch, ctx, n):
    # patterns planted across tile edges and in the last bytes
    t = host_text(4, n, 77)
    r = np.random.default_rng(5)
    text = to_dev(torch, t, 5)
    for m in (2, 7, 16, 63, 64, 65, 600, 4096):
        if m > n:
            continue
        for s in {0, TILE - 1, TILE - m // 2, TILE, 2 * TILE - 1, n - m, max(0, n - m - 1)}:
            if 0 <= s <= n - m:
                p = t[s:s + m].tobytes()
                assert gpu_count(ctx, text, p) == oracle.naive_count(p, t), (n, m, s)
        p = bytes(r.integers(0, 4, size=m).astype(np.uint8) + ord("A"))
        assert gpu_count(ctx, text, p) == oracle.naive_count(p, t)


def test_extreme_bytes(torch, ctx):
    r = np.random.default_rng(9)
    t = r.choice(np.array([0x00, 0xFF, 0x7F, 0x80], dtype=np.uint8), size=5 * TILE + 11)
    text = to_dev(torch, t, 1)
    for m in (1, 2, 3, 4, 9, 40):
        for p in patterns_for(t, m, r, k=3) + [b"\x00" * m, b"\xff" * m, (b"\x7f\x80" * m)[:m]]:
            assert gpu_count(ctx, text, p) == oracle.naive_count(p, t)


def test_degenerate_sizes(torch, ctx):
    empty = torch.zeros(0, dtype=torch.uint8, device="cuda")
    assert gpu_count(ctx, empty, b"a") == 0
    t = to_dev(torch, np.frombuffer(b"abc", np.uint8))
    assert gpu_count(ctx, t, b"abcd") == 0
    assert gpu_count(ctx, t, b"abc") == 1
    with pytest.raises(sm.SmError) as e:
        sm.sm_count(ctx, t, b"")
    assert e.value.status == sm.SM_EINVAL
    with pytest.raises(sm.SmError) as e:
        sm.sm_count(ctx, t, b"a" * (sm.SM_MAX_M + 1))
    assert e.value.status == sm.SM_EINVAL
    with pytest.raises(sm.SmError) as e:
        sm.sm_count(ctx, t, b"ab", pi=[0, 0])
    assert e.value.status == sm.SM_EINVAL


def test_paper_example(torch, ctx):
    # Fig. 1: t = "aabcd...", p = "abcd" -> one occurrence at position 1 (0-based)
    t = np.frombuffer(b"aabcd", np.uint8)
    pos, n, st = gpu_report(ctx, to_dev(torch, t), b"abcd", 4)
    assert st == sm.SM_OK and n == 1 and list(pos) == [1]


# ------------------------------------------------------------------ invariance

def test_invariance_order_peel_stages_grid(torch, ctx):
    n = 7 * TILE + 321
    for kind in (2, 4, "markov95", 256):
        t = host_text(kind, n, 11)
        text = to_dev(torch, t, 7)
        hist = oracle.histogram(t)
        r = np.random.default_rng(12)
        for m in (1, 3, 8, 33, 200):
            for p in patterns_for(t, m, r, k=2):
                want = oracle.naive_count(p, t)
                orders = [None, oracle.order_freq(p, hist), r.permutation(m).astype(np.uint32),
                          oracle.order_h(m), oracle.order_hs(p)]
                for pi in orders:
                    for peel in (0, 1, 2, 3, 5, m + 3):
                        assert gpu_count(ctx, text, p, pi=pi, peel=peel) == want
                    assert gpu_count(ctx, text, p, pi=pi, hist=hist) == want
                for stages in (2, 3, 8):
                    sm.sm_set_knob(ctx, sm.SM_KNOB_STAGES, stages)
                    for grid in (1, 3, 5, 1000):
                        sm.sm_set_knob(ctx, sm.SM_KNOB_GRID, grid)
                        assert gpu_count(ctx, text, p, hist=hist) == want
                sm.sm_set_knob(ctx, sm.SM_KNOB_STAGES, 4)
                sm.sm_set_knob(ctx, sm.SM_KNOB_GRID, 0)


def test_seven_bit_and_absent_symbol(torch, ctx):
    t = synth.markov95(6 * TILE + 99, seed=0, stream=3)
    hist = oracle.histogram(t)
    text = to_dev(torch, t, 2)
    r = np.random.default_rng(1)
    for m in (1, 2, 5, 16, 64, 300):
        for p in patterns_for(t, m, r, k=3):
            assert gpu_count(ctx, text, p, hist=hist) == oracle.naive_count(p, t)
    # symbols the text never holds (including bytes >= 0x80) give 0 without a scan
    for p in (b"\x80", b"ab\xffcd", b"\x01\x02"):
        assert gpu_count(ctx, text, p, hist=hist) == 0 == oracle.naive_count(p, t)


# ------------------------------------------------------------------ report

@pytest.fixture(params=["auto", "rescan", "bits"])
def report_mode(request, monkeypatch):
    """Both report designs: the library's choice, the rescan of the tiles with
    matches, and the passes over found bits (SM_REPORT forces one)."""
    if request.param != "auto":
        monkeypatch.setenv("SM_REPORT", request.param)
    return request.param


@pytest.mark.parametrize("kind", ["ones", 2, 4, 20, "markov95", 256])
def test_report_parity(torch, ctx, kind, report_mode):
    n = 9 * TILE + 1234
    t = host_text(kind, n, 21)
    text = to_dev(torch, t, 9)
    hist = oracle.histogram(t)
    r = np.random.default_rng(22)
    for m in (1, 2, 4, 8, 17, 64, 65, 1000):
        for p in patterns_for(t, m, r, k=2):
            want_pos, want = oracle.naive_report(p, t)
            for kw in ({}, {"hist": hist}, {"peel": 3, "pi": oracle.order_freq(p, hist)}):
                pos, c, st = gpu_report(ctx, text, p, want + 3, **kw)
                assert st == sm.SM_OK and c == want and np.array_equal(pos, want_pos), (kind, m)


def test_report_truncation(torch, ctx, report_mode):
    t = synth.uniform(5 * TILE + 17, 2, seed=0, stream=2)
    text = to_dev(torch, t, 0)
    p = b"01"
    want_pos, want = oracle.naive_report(p, t)
    assert want > 1000
    for cap in (0, 1, 999, want - 1):
        pos, c, st = gpu_report(ctx, text, p, cap)
        assert c == want and st == sm.SM_ETRUNC
        assert np.array_equal(pos, want_pos[:cap])
    pos, c, st = gpu_report(ctx, text, p, want)
    assert st == sm.SM_OK and np.array_equal(pos, want_pos)
    assert sm.sm_sync(ctx) == sm.SM_OK   # the status was cleared


@pytest.mark.parametrize("kind", [64, 4])
def test_report_clustered_matches(torch, ctx, kind, report_mode):
    """Warp-tiles whose matches are many or spread over many lanes next to
    warp-tiles with few: runs of one symbol and copies of the pattern every
    64 or 96 starts planted into a sparse background, so that the second
    pass meets slots in list form with few and with many entries and in
    bitmap form within one round of 32 warp-tiles, and rounds above and
    below its position-buffer size."""
    n = 40 * TILE + 999
    t = synth.text(kind, n, seed=0, stream=23).copy()
    sym = t[0]
    ws = 2048                                        # starts per warp-tile
    t[3 * ws + 100:3 * ws + 100 + 70] = sym          # one warp-tile, 69+ matches of sym sym
    for j in range(20):                              # 20 matches on 20 lanes of one warp-tile
        t[9 * ws + 96 * j:9 * ws + 96 * j + 2] = sym
    for j in range(32):                              # every lane of one warp-tile: bitmap form
        t[17 * ws + 64 * j + 5:17 * ws + 64 * j + 7] = sym
    t[200 * ws:200 * ws + 3000] = sym                # a round with more than the buffer holds
    p = bytes([sym, sym])
    hist = oracle.histogram(t)
    for off in (0, 7):
        text = to_dev(torch, t, off)
        want_pos, want = oracle.naive_report(p, t)
        for kw in ({}, {"hist": hist, "pi": oracle.order_freq(p, hist)}):
            pos, c, st = gpu_report(ctx, text, p, want, **kw)
            assert st == sm.SM_OK and c == want and np.array_equal(pos, want_pos), (kind, off)
        pos, c, st = gpu_report(ctx, text, p, want - 5, hist=hist)
        assert st == sm.SM_ETRUNC and c == want and np.array_equal(pos, want_pos[:want - 5])


def test_rescan_leaves_scratch_clear(torch, monkeypatch):
    """The rescanning report leaves its per-warp-tile counts and per-range
    sums zero for the next one (it clears what it read instead of zeroing
    them before every report). A sequence on a fresh context that could
    leave stale counts behind: back-to-back rescans, a larger text, a report
    over found bits (which writes every count word), a truncated report, an
    expired wait, and write-pass ranges that differ from the first pass's
    CTAs (a small grid: ranges of at most 288 tiles)."""
    c = sm.sm_create(0)
    big = synth.text(20, 41 * TILE + 77, seed=0, stream=31)
    small = synth.uniform(7 * TILE + 5, 2, seed=0, stream=32)
    wide = synth.text(64, 300 * TILE + 11, seed=0, stream=34).copy()
    r = np.random.default_rng(33)
    pa, pb = (big[s:s + 3].tobytes() for s in r.integers(0, big.size - 3, size=2))
    pw = wide[5:9].tobytes()
    for s in (0, 150 * TILE, 287 * TILE + 3, 288 * TILE - 2, 289 * TILE, wide.size - 4):
        wide[s:s + 4] = wide[5:9]                 # matches in the tiles around the range edges
    tb, ts, tw = to_dev(torch, big, 3), to_dev(torch, small, 0), to_dev(torch, wide, 0)

    def check(text, host, p, design, cap=None):
        monkeypatch.setenv("SM_REPORT", design)
        want_pos, want = oracle.naive_report(p, host)
        pos, n, st = gpu_report(c, text, p, want if cap is None else cap)
        k = want if cap is None else min(cap, want)
        assert n == want and np.array_equal(pos, want_pos[:k]), (design, p)
        assert st == (sm.SM_OK if k == want else sm.SM_ETRUNC)

    check(ts, small, b"0110", "rescan")
    check(tb, big, pa, "rescan")                  # the arrays grow
    check(tb, big, pb, "rescan")
    check(ts, small, b"01", "bits")               # every count word written
    check(tb, big, pa, "rescan")
    check(tb, big, big[:1].tobytes(), "rescan", cap=500)
    check(tb, big, pb, "rescan")
    sm.sm_set_knob(c, sm.SM_KNOB_SPIN_NS, 2_000_000)
    sm.sm_set_knob(c, sm.SM_KNOB_TEST_SKIP_COPY, 1)
    try:
        monkeypatch.setenv("SM_REPORT", "rescan")
        sm.sm_report(c, tb, pa, 1 << 16)
        assert sm.sm_sync(c) == sm.SM_ETIMEOUT
    finally:
        sm.sm_set_knob(c, sm.SM_KNOB_TEST_SKIP_COPY, 0)
        sm.sm_set_knob(c, sm.SM_KNOB_SPIN_NS, 1_000_000_000)
    check(tb, big, pa, "rescan")
    check(tb, big, pb, "rescan")
    for grid in (1, 3, 0):                        # 300 tiles: ranges of 288 + 12, of 100, default
        sm.sm_set_knob(c, sm.SM_KNOB_GRID, grid)
        check(tw, wide, pw, "rescan")
        check(tw, wide, pw, "rescan", cap=3)
    check(tw, wide, pw, "bits")
    check(tw, wide, pw, "rescan")


def test_bounded_wait_reports_timeout(torch, ctx):
    # The test hook leaves tile 0's copy unissued: its bounded wait must expire,
    # the kernel must return, and the context must stay usable.
    t = synth.uniform(4 * TILE, 4, seed=0, stream=8)
    text = to_dev(torch, t, 0)
    sm.sm_set_knob(ctx, sm.SM_KNOB_SPIN_NS, 2_000_000)
    sm.sm_set_knob(ctx, sm.SM_KNOB_TEST_SKIP_COPY, 1)
    try:
        sm.sm_count(ctx, text, b"ACGT")
        assert sm.sm_sync(ctx) == sm.SM_ETIMEOUT
    finally:
        sm.sm_set_knob(ctx, sm.SM_KNOB_TEST_SKIP_COPY, 0)
        sm.sm_set_knob(ctx, sm.SM_KNOB_SPIN_NS, 1_000_000_000)
    assert gpu_count(ctx, text, b"ACGT") == oracle.naive_count(b"ACGT", t)


# ------------------------------------------------------------------ workloads

def test_config_1mib_sigma4(torch, ctx):
    # n = 1 MiB of uniform {A,C,G,T}, seed 0; m = 8 copied from the text
    t = synth.uniform(1 << 20, 4, seed=0, stream=0)
    p = synth.sample_patterns(t, 8, 1, seed=0, stream=1)[0]
    text = to_dev(torch, t)
    hist = oracle.histogram(t)
    pi = sm.sm_order(p, hist)
    want_pos, want = oracle.naive_report(p, t)
    assert gpu_count(ctx, text, p, pi=pi, hist=hist) == want
    pos, c, st = gpu_report(ctx, text, p, want, pi=pi, hist=hist)
    assert st == sm.SM_OK and c == want and np.array_equal(pos, want_pos)


@pytest.mark.parametrize("kind", [2, 4, 20, 64, "markov95"])
def test_full_size_1gib(torch, ctx, kind):
    # n = 1 GiB, the sweep's text sizes; counts against the threaded oracle
    n = 1 << 30
    t = synth.text(kind, n, seed=0, stream=synth.stream_id("sweep", kind))
    text = torch.from_numpy(t).cuda()
    hist_gpu = sm.sm_histogram(ctx, text)
    hist = oracle.histogram(t)
    assert np.array_equal(hist_gpu.cpu().numpy().view(np.uint64), hist)
    for m in (2, 8, 64, 1024):
        for p in synth.sample_patterns(t, m, 2, seed=0, stream=synth.stream_id("pat", kind, m)):
            pi = sm.sm_order(p, hist)
            assert gpu_count(ctx, text, p, pi=pi, hist=hist) == oracle.count_threads(p, t)
    p = synth.sample_patterns(t, 16, 1, seed=0, stream=synth.stream_id("rep", kind))[0]
    want = oracle.count_threads(p, t)
    want_pos, _ = oracle.report_threads(p, t, want)
    pos, c, st = gpu_report(ctx, text, p, want, pi=sm.sm_order(p, hist), hist=hist)
    assert st == sm.SM_OK and c == want and np.array_equal(pos, want_pos)
    del text
    torch.cuda.empty_cache()


@pytest.mark.parametrize("kind", [2, 4, 20, "markov95"])
def test_full_size_dense_report(torch, ctx, kind):
    """Reports of short patterns at n = 1 GiB, where matches are densest
    (sigma = 2, m = 2: about n/4 positions), in the launch configuration the
    sweep uses (text histogram, rarest-first order). Every position is
    compared with the threaded oracle, streamed over 128 MiB windows of the
    text (each with its (m - 1)-byte halo)."""
    n = 1 << 30
    t = synth.text(kind, n, seed=0, stream=synth.stream_id("sweep", kind))
    text = torch.from_numpy(t).cuda()
    hist = oracle.histogram(t)
    for m in (2, 4):
        p = synth.sample_patterns(t, m, 1, seed=0, stream=synth.stream_id("pat", kind, m))[0]
        want = oracle.count_threads(p, t)
        pos, cnt = sm.sm_report(ctx, text, p, want, pi=sm.sm_order(p, hist), hist=hist)
        assert sm.sm_sync(ctx) == sm.SM_OK
        assert int(cnt.item()) == want
        win, off = 128 << 20, 0
        for a in range(0, n - m + 1, win):
            b = min(a + win, n - m + 1)            # starts [a, b)
            wp, wc = oracle.report_threads(p, t[a:b + m - 1], b - a)
            got = pos[off:off + wc].cpu().numpy().view(np.uint64)
            assert np.array_equal(got, wp + np.uint64(a)), (kind, m, a)
            off += wc
        assert off == want
        del pos
    del text
    torch.cuda.empty_cache()


def test_injected_alloc_failure(torch, monkeypatch):
    """Host-side fault injection: with SM_FAULT=alloc every workspace
    allocation fails, so the first call that must grow the workspace (a
    report's per-tile tables) returns SM_ENOMEM and enqueues nothing; without
    it the same context then gives the oracle's result."""
    import __graft_entry__
    __graft_entry__.build()
    fresh = sm.sm_create(0)
    t = synth.uniform(6 * TILE + 77, 20, seed=0, stream=61)
    text = to_dev(torch, t, 3)
    p = t[5000:5002].tobytes()
    want_pos, want = oracle.naive_report(p, t)
    monkeypatch.setenv("SM_FAULT", "alloc")
    with pytest.raises(sm.SmError) as e:
        sm.sm_report(fresh, text, p, want)
    assert e.value.status == sm.SM_ENOMEM
    with pytest.raises(sm.SmError) as e:
        sm.sm_create(0)
    assert e.value.status == sm.SM_ENOMEM
    monkeypatch.delenv("SM_FAULT")
    pos, c, st = gpu_report(fresh, text, p, want)
    assert st == sm.SM_OK and c == want and np.array_equal(pos, want_pos)
