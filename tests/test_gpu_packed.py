"""GPU parity of the coded compare paths (texts of at most four symbols).

With the text histogram, sm_count and sm_report compare 1-bit codes of the
symbols when the text holds at most two distinct bytes and 2-bit codes when
it holds at most four; SM_SEARCH_BYTES forces the byte compare on the same
input. Both must equal the CPU oracle bit for bit: counts and ordered
positions, across tile and halo edges, misaligned texts, forced peels, both
2-bit code layouts (adjacent bits, as for ACGT, and bits that are not
adjacent) and 1-bit codes from a low or the top bit.
"""
import numpy as np
import pytest

import oracle
from paper_1612_01506_gb300 import sm

pytestmark = pytest.mark.gpu

TILE = sm.SM_TILE_STARTS

# alphabets: ACGT (code bits 1, 2), bytes separable only by bits 0 and 2,
# two symbols, three symbols, one symbol
ALPHABETS = {
    "acgt": b"ACGT",
    "nonadjacent": b"\x00\x01\x04\x05",
    "binary": b"01",
    "binary_top_bit": b"\x10\x90",
    "three": b"xyz",
    "one": b"a",
}


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
    buf = torch.zeros(host.size + offset + 64, dtype=torch.uint8, device="cuda")
    if host.size:
        buf[offset:offset + host.size] = torch.from_numpy(host).cuda()
    return buf[offset:offset + host.size]


def text_over(alpha: bytes, n: int, seed: int) -> np.ndarray:
    r = np.random.default_rng(seed)
    return np.frombuffer(alpha, np.uint8)[r.integers(0, len(alpha), n)].copy()


def count(ctx, text, p, **kw):
    c = sm.sm_count(ctx, text, p, **kw)
    assert sm.sm_sync(ctx) == sm.SM_OK
    return int(c.item())


def report(ctx, text, p, cap, **kw):
    pos, c = sm.sm_report(ctx, text, p, cap, **kw)
    st = sm.sm_sync(ctx)
    n = int(c.item())
    return pos[: min(n, cap)].cpu().numpy().view(np.uint64), n, st


def patterns(t, alpha, m, r):
    out = []
    if t.size >= m:
        for _ in range(2):
            s = int(r.integers(0, t.size - m + 1))
            out.append(t[s:s + m].tobytes())
    a = np.frombuffer(alpha, np.uint8)
    out.append(a[r.integers(0, a.size, m)].tobytes())
    return out


@pytest.mark.parametrize("name", list(ALPHABETS))
@pytest.mark.parametrize("n", [1, 17, TILE - 1, TILE + 1, 3 * TILE + 777])
def test_packed_count_edges(torch, ctx, name, n):
    alpha = ALPHABETS[name]
    t = text_over(alpha, n, n)
    hist = oracle.histogram(t)
    r = np.random.default_rng(n + len(alpha))
    for offset in (0, 3, 13):
        text = to_dev(torch, t, offset)
        for m in (1, 2, 3, 5, 15, 16, 17, 31, 33, 63, 64, 65, 100, 600, 4096):
            if m > n:
                continue
            for p in patterns(t, alpha, m, r):
                want = oracle.naive_count(p, t)
                assert count(ctx, text, p, hist=hist) == want, (name, n, offset, m)
                assert count(ctx, text, p, hist=hist, bytes_only=True) == want, (name, n, offset, m)


@pytest.mark.parametrize("name", ["acgt", "nonadjacent", "binary", "binary_top_bit"])
def test_packed_peel_and_order(torch, ctx, name):
    alpha = ALPHABETS[name]
    n = 5 * TILE + 99
    t = text_over(alpha, n, 7)
    hist = oracle.histogram(t)
    text = to_dev(torch, t, 5)
    r = np.random.default_rng(8)
    for m in (1, 4, 9, 40, 130):
        for p in patterns(t, alpha, m, r):
            want = oracle.naive_count(p, t)
            for pi in (None, oracle.order_freq(p, hist), r.permutation(m).astype(np.uint32)):
                for peel in (0, 1, 2, 7, m):
                    assert count(ctx, text, p, pi=pi, peel=peel, hist=hist) == want, (m, peel)


@pytest.fixture(params=["auto", "rescan", "bits"])
def report_mode(request, monkeypatch):
    """Both report designs (SM_REPORT forces one; auto is the library's choice)."""
    if request.param != "auto":
        monkeypatch.setenv("SM_REPORT", request.param)
    return request.param


@pytest.mark.parametrize("name", list(ALPHABETS))
def test_packed_report(torch, ctx, name, report_mode):
    alpha = ALPHABETS[name]
    n = 4 * TILE + 1234
    t = text_over(alpha, n, 31)
    hist = oracle.histogram(t)
    text = to_dev(torch, t, 9)
    r = np.random.default_rng(32)
    for m in (1, 2, 6, 12, 20, 64, 65, 300):
        for p in patterns(t, alpha, m, r):
            want_pos, want = oracle.naive_report(p, t)
            for kw in ({"hist": hist}, {"hist": hist, "peel": 2}, {"hist": hist, "bytes_only": True}):
                pos, c, st = report(ctx, text, p, want + 2, **kw)
                assert st == sm.SM_OK and c == want and np.array_equal(pos, want_pos), (name, m, kw)


def test_packed_absent_symbol_and_truncation(torch, ctx, report_mode):
    t = text_over(b"ACGT", 3 * TILE + 5, 41)
    hist = oracle.histogram(t)
    text = to_dev(torch, t, 0)
    for p in (b"N", b"ACGN", b"acgt"):
        assert count(ctx, text, p, hist=hist) == 0 == oracle.naive_count(p, t)
    p = b"AC"
    want_pos, want = oracle.naive_report(p, t)
    for cap in (0, 1, want - 1):
        pos, c, st = report(ctx, text, p, cap, hist=hist)
        assert c == want and st == sm.SM_ETRUNC and np.array_equal(pos, want_pos[:cap])
    assert sm.sm_sync(ctx) == sm.SM_OK


def test_packed_tile_edges_planted(torch, ctx):
    n = 4 * TILE + 4096 + 3
    t = text_over(b"ACGT", n, 51)
    hist = oracle.histogram(t)
    text = to_dev(torch, t, 1)
    for m in (2, 7, 16, 63, 64, 65, 600, 4096):
        for s in {0, TILE - 1, TILE - m // 2, TILE, 2 * TILE - 1, n - m}:
            if 0 <= s <= n - m:
                p = t[s:s + m].tobytes()
                assert count(ctx, text, p, hist=hist) == oracle.naive_count(p, t), (m, s)
