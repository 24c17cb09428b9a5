"""Full-size parity for the batched and serving workloads.

* 256 MiB Markov-95 text with 4096 patterns (m log-uniform in [2, 1024],
  80 % from the text): every batched count equals the single-pattern scan's,
  and a sample equals the CPU oracle.
* 20,000 packed texts (lengths log-uniform 1 KiB - 16 MiB, alphabet per text
  from {4, 20, 95, 256}), 1-8 patterns of length 2-512 per text: counts and
  ordered positions in one call; sampled patterns against the oracle.
* Serving on a 4 GiB resident text (2 GiB ACGT + 2 GiB Markov-95): every
  query's result equals the query run alone and the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1612_01506_gb300 import sm, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    return sm.sm_create(0)


def test_batch_4096_patterns_256mib(torch, ctx):
    n, npat = 256 << 20, 4096
    t = synth.markov95(n, seed=0, stream=synth.stream_id("batch", "markov95"))
    r = np.random.default_rng(0)
    lens = np.exp(r.uniform(np.log(2), np.log(1024), npat)).astype(np.int64)
    alpha = np.frombuffer(synth.MARKOV95, np.uint8)
    pats = []
    for k in range(npat):
        m = int(lens[k])
        if r.random() < 0.8:
            o = int(r.integers(0, n - m + 1))
            pats.append(t[o:o + m].tobytes())
        else:
            pats.append(alpha[r.integers(0, alpha.size, m)].tobytes())
    d = torch.from_numpy(t).cuda()
    b = sm.sm_batch_create(ctx, d, np.array([0, n], np.int64), pats, np.zeros(npat, np.int32))
    got = sm.sm_batch_count(b).cpu().numpy()
    hist = sm.sm_histogram(ctx, d).cpu().numpy().view(np.uint64).copy()
    single = torch.zeros(npat, dtype=torch.int64, device="cuda")
    for k, p in enumerate(pats):
        sm.sm_count(ctx, d, p, pi=sm.sm_order(p, hist), hist=hist, out=single[k:k + 1])
    assert sm.sm_sync(ctx) == sm.SM_OK
    assert np.array_equal(got, single.cpu().numpy())
    for k in r.choice(npat, 24, replace=False):
        assert got[k] == oracle.count_threads(pats[k], t), k


def test_batch_20000_texts_with_positions(torch, ctx):
    r = np.random.default_rng(4)
    ntexts = 20_000
    lens = np.exp(r.uniform(np.log(1024), np.log(16 << 20), ntexts)).astype(np.int64)
    kinds = r.choice(np.array([4, 20, 95, 256]), ntexts)
    off = np.zeros(ntexts + 1, np.int64)
    off[1:] = np.cumsum(lens)
    flat = np.empty(int(off[-1]), np.uint8)
    for x in range(ntexts):
        k = int(kinds[x])
        synth.text("markov95" if k == 95 else k, int(lens[x]), seed=0, stream=synth.stream_id("c4", x),
                   out=flat[off[x]:off[x + 1]])
    pats, pat_text = [], []
    for x in range(ntexts):
        for _ in range(int(r.integers(1, 9))):
            m = int(np.exp(r.uniform(np.log(2), np.log(512))))
            m = min(m, int(lens[x]))
            s = int(r.integers(0, lens[x] - m + 1))
            pats.append(flat[off[x] + s: off[x] + s + m].tobytes())
            pat_text.append(x)
    npat = len(pats)
    pat_off = np.zeros(npat + 1, np.int64)
    pat_off[1:] = np.cumsum([len(p) for p in pats])
    pt = np.array(pat_text, np.int32)
    d = torch.from_numpy(flat).cuda()
    # counts first (sizes the position lists), then counts and positions in one call
    b = sm.sm_batch_create(ctx, d, off, pats, pt)
    counts = sm.sm_batch_count(b).cpu().numpy()
    pos_off = np.zeros(npat + 1, np.int64)
    pos_off[1:] = np.cumsum(counts)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_counts = torch.zeros(npat, dtype=torch.int64, device="cuda")
    d_pos = torch.zeros(max(int(pos_off[-1]), 1), dtype=torch.int64, device="cuda")
    sm.sm_count_batch(ctx, d, T(off), T(np.frombuffer(b"".join(pats), np.uint8).copy()), T(pat_off), T(pt),
                      d_counts, d_pos, T(pos_off))
    assert np.array_equal(d_counts.cpu().numpy(), counts)
    allpos = d_pos.cpu().numpy().view(np.uint64)
    for k in r.choice(npat, 300, replace=False):
        x = pt[k]
        text = flat[off[x]:off[x + 1]]
        want_pos, want = oracle.naive_report(pats[k], text)
        assert counts[k] == want, (k, x)
        assert np.array_equal(allpos[pos_off[k]:pos_off[k + 1]], want_pos), (k, x)


def test_serving_4gib(torch):
    from paper_1612_01506_gb300.serve import Query, Server
    half = 2 << 30
    t = np.empty(2 * half, np.uint8)
    synth.uniform(half, 4, seed=0, stream=synth.stream_id("serve", 4), out=t[:half])
    synth.markov95(half, seed=0, stream=synth.stream_id("serve", "markov95"), out=t[half:])
    text = torch.from_numpy(t).cuda()
    server = Server(text, chunk_bytes=256 << 20, max_m=2048, max_active=64, report_budget=4 << 30)
    r = np.random.default_rng(9)
    qs = []
    for i in range(48):
        m = int(np.exp(r.uniform(np.log(2), np.log(2048))))
        s = int(r.integers(0, t.size - m + 1))
        p = t[s:s + m].tobytes() if r.random() < 0.8 else bytes(r.choice(np.frombuffer(b"ACGT e", np.uint8), m))
        if r.random() < 0.2:
            p = p[: min(len(p), 12)] if len(p) > 12 else p   # keep report sizes moderate
        qs.append(Query(pattern=p, kind="report" if r.random() < 0.2 else "count", arrival=i * 0.0005))
    server.run(qs)
    ctx1 = sm.sm_create(0)
    for q in qs:
        alone = int(sm.sm_count(ctx1, text, q.pattern).item())
        assert q.count == alone == oracle.count_threads(q.pattern, t), q.pattern[:16]
        if q.kind == "report":
            pos, c = oracle.report_threads(q.pattern, t, q.count)
            assert np.array_equal(q.positions.cpu().numpy().view(np.uint64), pos)
