"""Serving: every query's result is the same alone and in the mix."""
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


def make_text(n_half):
    return np.concatenate([synth.uniform(n_half, 4, seed=0, stream=71), synth.markov95(n_half, seed=0, stream=72)])


def make_queries(t, k, seed, report_frac=0.2, mmax=2048):
    from paper_1612_01506_gb300.serve import Query
    r = np.random.default_rng(seed)
    qs = []
    for i in range(k):
        m = int(np.exp(r.uniform(np.log(2), np.log(mmax))))
        if r.random() < 0.8:
            s = int(r.integers(0, t.size - m + 1))
            p = t[s:s + m].tobytes()
        else:
            p = bytes(r.choice(np.frombuffer(b"ACGT e", np.uint8), m))
        qs.append(Query(pattern=p, kind="report" if r.random() < report_frac else "count", arrival=i * 0.0004))
    return qs


# report_batch_min 2: waiting report queries go through batched reports
@pytest.mark.parametrize("report_batch_min", [32, 2])
def test_serving_results_equal_alone(torch, report_batch_min):
    from paper_1612_01506_gb300.serve import Server
    t = make_text(3 << 20)
    text = torch.from_numpy(t).cuda()
    server = Server(text, chunk_bytes=1 << 20, max_m=2048, max_active=16, report_budget=1 << 26, burst_below=4,
                    report_batch_min=report_batch_min)
    assert server.nchunks == 6
    qs = make_queries(t, 60, seed=1)
    done = server.run(qs)
    assert len(server.done) == len(qs)
    ctx = sm.sm_create(0)
    for q in done:
        alone = int(sm.sm_count(ctx, text, q.pattern).item())
        assert q.count == alone == oracle.count_threads(q.pattern, t), q.pattern[:20]
        if q.kind == "report":
            pos, c = oracle.report_threads(q.pattern, t, q.count)
            assert np.array_equal(q.positions.cpu().numpy().view(np.uint64), pos)
    # the mix really overlapped: more queries than slots, several steps
    assert server.steps > server.nchunks


def test_stepper_joins_at_any_chunk(torch):
    # queries joining at different chunks and wrapping around give full counts
    from paper_1612_01506_gb300.serve import Server
    t = make_text(1 << 20)
    text = torch.from_numpy(t).cuda()
    server = Server(text, chunk_bytes=1 << 18, max_m=512, max_active=8, burst_below=0)   # one chunk per step
    qs = make_queries(t, 24, seed=2, report_frac=0.0, mmax=512)
    for k, q in enumerate(qs):
        q.arrival = 0.0
    # submit in waves between steps so that joins happen at many chunks
    pending = list(qs)
    while pending or server.busy:
        for _ in range(3):
            if pending:
                server.submit(pending.pop())
        server.step()
    torch.cuda.synchronize()
    for q in qs:
        assert q.count == oracle.count_threads(q.pattern, t)


def test_stepper_report_batch(torch):
    # one batched report of many patterns over the resident text: absent
    # symbols, m up to 4096, zero capacities, truncation
    import ctypes as C
    from paper_1612_01506_gb300.serve import Server
    t = make_text(1 << 20)
    text = torch.from_numpy(t).cuda()
    server = Server(text, chunk_bytes=1 << 18, max_m=4096, max_active=8)
    r = np.random.default_rng(5)
    pats = []
    for m in (1, 2, 3, 5, 8, 13, 40, 100, 700, 4096):
        for _ in range(3):
            s0 = int(r.integers(0, t.size - m + 1))
            pats.append(t[s0:s0 + m].tobytes())
    pats += [b"\x01ACGT", b"e" * 3, b"ACGT" * 7]
    want = [oracle.count_threads(p, t) for p in pats]
    for caps in (want, [min(c, 3) if k % 2 else c for k, c in enumerate(want)]):
        pos_off = np.zeros(len(pats) + 1, np.int64)
        pos_off[1:] = np.cumsum(caps)
        pat_off = np.zeros(len(pats) + 1, np.int64)
        pat_off[1:] = np.cumsum([len(p) for p in pats])
        flat = np.frombuffer(b"".join(pats), np.uint8)
        pos = torch.empty(max(int(pos_off[-1]), 1), dtype=torch.int64, device="cuda")
        cnt = torch.empty(len(pats), dtype=torch.int64, device="cuda")
        st = server.lib.sm_stepper_report(server.stepper, flat.ctypes.data_as(C.POINTER(C.c_uint8)),
                                          pat_off.ctypes.data_as(C.POINTER(C.c_int64)), len(pats),
                                          pos_off.ctypes.data_as(C.POINTER(C.c_int64)), pos.data_ptr(),
                                          cnt.data_ptr(), server.rstream.cuda_stream)
        assert st == sm.SM_OK
        server.rstream.synchronize()
        trunc = any(c < w for c, w in zip(caps, want))
        assert sm.sm_sync(server.ctx) == (sm.SM_ETRUNC if trunc else sm.SM_OK)
        assert np.array_equal(cnt.cpu().numpy(), np.array(want, np.int64))
        allpos = pos.cpu().numpy().view(np.uint64)
        for k, p in enumerate(pats):
            w, _ = oracle.report_threads(p, t, want[k])
            assert np.array_equal(allpos[pos_off[k]:pos_off[k + 1]], w[: caps[k]]), (k, len(p))


def test_stepper_patterns_across_chunk_classes(torch):
    # chunks of the ACGT half and of the Markov half have different symbol
    # sets; a pattern that starts in the last ACGT chunk and ends in the
    # Markov half holds symbols absent from that chunk, and must still count
    from paper_1612_01506_gb300.serve import Query, Server
    half = 1 << 20
    t = make_text(half)
    text = torch.from_numpy(t).cuda()
    server = Server(text, chunk_bytes=1 << 18, max_m=512, max_active=64, burst_below=0)
    qs = []
    for m in (2, 3, 8, 40, 300, 512):
        for back in (1, m // 2, m - 1):
            if 0 < back < m:
                s0 = half - back
                qs.append(Query(pattern=t[s0:s0 + m].tobytes(), kind="count", arrival=0.0))
    qs.append(Query(pattern=t[half - 5:half + 3].tobytes(), kind="report", arrival=0.0))
    server.run(qs)
    for q in qs:
        assert q.count == oracle.count_threads(q.pattern, t) >= 1, (len(q.pattern), q.pattern[:12])
    q = qs[-1]
    pos, _ = oracle.report_threads(q.pattern, t, q.count)
    assert np.array_equal(q.positions.cpu().numpy().view(np.uint64), pos)


def test_stepper_steps_chunk_ranges(torch):
    # sm_stepper_steps: each query scanned on its own number of chunks from a
    # start chunk, wrapping around the text, in one launch; the counts equal
    # the oracle's over exactly those chunks
    import ctypes as C
    from paper_1612_01506_gb300.serve import Server
    t = make_text(1 << 20)
    text = torch.from_numpy(t).cuda()
    chunk = 1 << 18
    server = Server(text, chunk_bytes=chunk, max_m=512, max_active=8)
    nch = server.nchunks
    r = np.random.default_rng(9)
    pats = []
    for m in (2, 5, 40, 512):
        s0 = int(r.integers(0, t.size - m + 1))
        pats.append(t[s0:s0 + m].tobytes())
    for first in (0, nch - 3):
        spans = [nch, 1, 3, nch - 1][: len(pats)]
        counters = torch.zeros(len(pats), dtype=torch.int64, device="cuda")
        for q, p in enumerate(pats):
            a = np.frombuffer(p, np.uint8)
            assert server.lib.sm_stepper_admit(server.stepper, q, a.ctypes.data_as(C.POINTER(C.c_uint8)), a.size) == 0
        qids = np.arange(len(pats), dtype=np.uint32)
        left = np.array(spans, dtype=np.uint32)
        assert server.lib.sm_stepper_steps(server.stepper, qids.ctypes.data_as(C.POINTER(C.c_uint32)),
                                           left.ctypes.data_as(C.POINTER(C.c_uint32)), len(pats), first,
                                           counters.data_ptr(), server.stream.cuda_stream) == 0
        server.stream.synchronize()
        got = counters.cpu().numpy()
        for q, p in enumerate(pats):
            want = 0
            for k in range(spans[q]):
                c = (first + k) % nch
                lo, hi = c * chunk, min((c + 1) * chunk, t.size)          # starts counted in chunk c
                seg = t[lo:min(hi + len(p) - 1, t.size)]
                want += oracle.count_threads(p, seg) if seg.size >= len(p) else 0
            assert got[q] == want, (q, first, spans[q])
        for q in range(len(pats)):
            server.lib.sm_stepper_retire(server.stepper, q)


def test_serving_report_admission(torch):
    """Report buffers are admitted by the budget and by the device's free
    memory: a report whose positions exceed the budget, or that cannot fit
    in free memory with nothing in flight to give memory back, is answered
    with an error; the other queries are unaffected."""
    from paper_1612_01506_gb300.serve import Query, Server
    t = make_text(1 << 20)
    text = torch.from_numpy(t).cuda()
    small_p = t[100:124].tobytes()
    want_small = oracle.naive_report(small_p, t)
    server = Server(text, chunk_bytes=1 << 20, max_m=64, max_active=8, report_budget=4096)
    big = Query(pattern=b"AC", kind="report")                 # ~n/32 matches: far above 4096 bytes
    small = Query(pattern=small_p, kind="report", arrival=0.001)
    cnt = Query(pattern=b"ACG", kind="count", arrival=0.002)
    server.run([big, small, cnt])
    assert big.error and big.positions is None and big.count == oracle.naive_count(b"AC", t)
    assert small.error is None and small.count == want_small[1]
    assert np.array_equal(small.positions.cpu().numpy().view(np.uint64), want_small[0])
    assert cnt.count == oracle.naive_count(b"ACG", t)
    # no free memory at all for positions: every report is refused, counts still run
    total = torch.cuda.mem_get_info()[1]
    starved = Server(text, chunk_bytes=1 << 20, max_m=64, max_active=8, memory_reserve=total)
    q1, q2 = Query(pattern=small_p, kind="report"), Query(pattern=b"GT", kind="count")
    starved.run([q1, q2])
    assert q1.error and "available" in q1.error and q1.count == want_small[1]
    assert q2.count == oracle.naive_count(b"GT", t)


def test_serving_idle_arrival_runs_alone(torch):
    """A query arriving at an idle server is one single search over the
    whole text; its count equals the oracle's, and a report follows it."""
    from paper_1612_01506_gb300.serve import Query, Server
    t = make_text(1 << 20)
    text = torch.from_numpy(t).cuda()
    server = Server(text, chunk_bytes=1 << 20, max_m=64, max_active=8)
    qs = [Query(pattern=t[i * 1000:i * 1000 + 9].tobytes(), kind=("report" if i % 2 else "count"),
                arrival=0.02 * i) for i in range(6)]
    server.run(qs)
    assert all(q.alone for q in qs)
    for q in qs:
        pos, c = oracle.naive_report(q.pattern, t)
        assert q.count == c
        if q.kind == "report":
            assert np.array_equal(q.positions.cpu().numpy().view(np.uint64), pos)
