"""GPU parity of batched counting against the oracle (bit-exact)."""
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
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    import __graft_entry__
    __graft_entry__.build()
    return sm.sm_create(0)


def make_batch(seed, sizes, kinds, pats_per_text, mmax):
    r = np.random.default_rng(seed)
    texts = [synth.text(k, n, seed=0, stream=synth.stream_id("bt", seed, i)) if n else np.zeros(0, np.uint8)
             for i, (k, n) in enumerate(zip(kinds, sizes))]
    off = np.zeros(len(texts) + 1, np.int64)
    off[1:] = np.cumsum([t.size for t in texts])
    pats, pat_text = [], []
    for x, t in enumerate(texts):
        for _ in range(pats_per_text):
            m = int(np.exp(r.uniform(0, np.log(mmax))))
            u = r.random()
            if t.size >= m and u < 0.7:
                s = int(r.integers(0, t.size - m + 1))
                pats.append(t[s:s + m].tobytes())
            elif u < 0.9:
                alpha = np.frombuffer(synth.alphabet_of(kinds[x]), np.uint8)
                pats.append(alpha[r.integers(0, alpha.size, m)].tobytes())
            else:
                pats.append(bytes(r.integers(0, 256, m, dtype=np.uint8)))
            pat_text.append(x)
    order = r.permutation(len(pats))      # patterns in any order
    pats = [pats[i] for i in order]
    pat_text = [pat_text[i] for i in order]
    flat = np.concatenate(texts) if texts else np.zeros(0, np.uint8)
    return texts, flat, off, pats, np.array(pat_text, np.int32)


def expected(texts, pats, pat_text):
    return np.array([oracle.naive_count(p, texts[x]) for p, x in zip(pats, pat_text)], np.int64)


def to_dev(torch, flat, offset=3):
    buf = torch.zeros(flat.size + offset + 64, dtype=torch.uint8, device="cuda")
    if flat.size:
        buf[offset:offset + flat.size] = torch.from_numpy(flat.copy()).cuda()
    return buf[offset:offset + flat.size]


# 8 patterns per text: every pattern runs the dense scan; 40: texts with at
# least 16 patterns whose rarest symbol is rare run the candidate path
@pytest.mark.parametrize("seed,per_text", [(1, 8), (2, 8), (3, 40), (4, 40)])
def test_batch_mixed(torch, ctx, seed, per_text):
    sizes = [0, 1, 17, 5000, 40_000, 3 * 16384 + 11, 200_000, 7]
    kinds = [4, 20, "markov95", 256, 4, 2, "markov95", 64]
    texts, flat, off, pats, pt = make_batch(seed, sizes, kinds, per_text, 600)
    d = to_dev(torch, flat)
    b = sm.sm_batch_create(ctx, d, off, pats, pt)
    got = sm.sm_batch_count(b).cpu().numpy()[: len(pats)]
    assert sm.sm_sync(ctx) == sm.SM_OK
    assert np.array_equal(got, expected(texts, pats, pt))
    # a second count from the same plan gives the same result
    assert np.array_equal(sm.sm_batch_count(b).cpu().numpy()[: len(pats)], got)


def test_batch_many_patterns_one_text(torch, ctx):
    # more patterns than one CTA counts (4096): the text is split into groups
    t = synth.markov95(600_000, seed=0, stream=11)
    r = np.random.default_rng(4)
    pats = []
    for _ in range(5000):
        m = int(np.exp(r.uniform(np.log(2), np.log(1024))))
        if r.random() < 0.8:
            s = int(r.integers(0, t.size - m + 1))
            pats.append(t[s:s + m].tobytes())
        else:
            pats.append(bytes(r.integers(0x20, 0x7F, m, dtype=np.uint8)))
    off = np.array([0, t.size], np.int64)
    d = to_dev(torch, t, 0)
    b = sm.sm_batch_create(ctx, d, off, pats, np.zeros(len(pats), np.int32))
    got = sm.sm_batch_count(b).cpu().numpy()
    want = np.array([oracle.naive_count(p, t) for p in pats], np.int64)
    assert np.array_equal(got, want)


def test_batch_graph_capture(torch, ctx):
    texts, flat, off, pats, pt = make_batch(9, [100_000, 70_000], [4, "markov95"], 16, 64)
    d = to_dev(torch, flat)
    b = sm.sm_batch_create(ctx, d, off, pats, pt)
    out = torch.zeros(len(pats), dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    sm.sm_batch_count(b, out=out, stream=s)   # warm up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sm.sm_batch_count(b, out=out, stream=s)
    out.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), expected(texts, pats, pt))


def test_count_batch_device_metadata_with_positions(torch, ctx):
    texts, flat, off, pats, pt = make_batch(5, [30_000, 0, 50_000, 9], [2, 4, 20, 4], 6, 40)
    want = expected(texts, pats, pt)
    d = to_dev(torch, flat, 1)
    poff = np.zeros(len(pats) + 1, np.int64)
    caps = np.minimum(want, 50)                # some reports truncate
    poff[1:] = np.cumsum(caps)
    pflat = np.frombuffer(b"".join(pats), np.uint8).copy()
    pat_off = np.zeros(len(pats) + 1, np.int64)
    pat_off[1:] = np.cumsum([len(p) for p in pats])
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    counts = torch.zeros(len(pats), dtype=torch.int64, device="cuda")
    dpos = torch.zeros(max(int(poff[-1]), 1), dtype=torch.int64, device="cuda")
    sm.sm_count_batch(ctx, d, T(off), T(pflat), T(pat_off), T(pt), counts, dpos, T(poff))
    assert sm.sm_sync(ctx) == (sm.SM_ETRUNC if (caps < want).any() else sm.SM_OK)
    assert np.array_equal(counts.cpu().numpy(), want)
    allpos = dpos.cpu().numpy().view(np.uint64)
    for k, (p, x) in enumerate(zip(pats, pt)):
        pos, c = oracle.naive_report(p, texts[x])
        assert np.array_equal(allpos[poff[k]:poff[k + 1]], pos[: caps[k]])


def oracle_positions(texts, pats, pt, caps):
    out = []
    for p, x, c in zip(pats, pt, caps):
        pos, _ = oracle.naive_report(p, texts[x])
        out.append(pos[:c])
    return out


@pytest.mark.parametrize("seed,per_text", [(21, 6), (22, 40)])
def test_batch_report_mixed(torch, ctx, seed, per_text):
    # ordered positions of every pattern in one batched report: dense and
    # candidate counting passes, empty and tiny texts, truncated capacities
    sizes = [0, 1, 17, 5000, 40_000, 3 * 16384 + 11, 200_000, 7]
    kinds = [4, 20, "markov95", 256, 4, 2, "markov95", 64]
    texts, flat, off, pats, pt = make_batch(seed, sizes, kinds, per_text, 600)
    want = expected(texts, pats, pt)
    d = to_dev(torch, flat)
    b = sm.sm_batch_create(ctx, d, off, pats, pt)
    sm.sm_sync(ctx)   # no status left from earlier calls
    for trunc in (False, True):
        caps = np.minimum(want, 7) if trunc else want
        poff = np.zeros(len(pats) + 1, np.int64)
        poff[1:] = np.cumsum(caps)
        d_off = torch.from_numpy(poff).cuda()
        counts, dpos = sm.sm_batch_report(b, d_off)
        st = sm.sm_sync(ctx)
        assert st == (sm.SM_ETRUNC if trunc and (caps < want).any() else sm.SM_OK)
        assert np.array_equal(counts.cpu().numpy()[: len(pats)], want)
        allpos = dpos.cpu().numpy().view(np.uint64)
        for k, pos in enumerate(oracle_positions(texts, pats, pt, caps)):
            assert np.array_equal(allpos[poff[k]:poff[k + 1]], pos), (k, len(pats[k]), pt[k])
    # counting with the same plan still works after a report
    assert np.array_equal(sm.sm_batch_count(b).cpu().numpy()[: len(pats)], want)


def test_batch_report_dense_matches(torch, ctx):
    # short patterns on small alphabets: matches in almost every tile, many
    # patterns per text (the candidate counting pass on the byte text)
    t2 = synth.uniform(5 * 16384 + 333, 2, seed=0, stream=31)
    t4 = synth.uniform(7 * 16384 + 5, 4, seed=0, stream=32)
    tm = synth.markov95(300_000, seed=0, stream=33)
    texts = [t2, t4, tm]
    r = np.random.default_rng(34)
    pats, pt = [], []
    for x, t in enumerate(texts):
        for _ in range(30):
            m = int(r.integers(1, 9))
            s0 = int(r.integers(0, t.size - m + 1))
            pats.append(t[s0:s0 + m].tobytes())
            pt.append(x)
    off = np.zeros(4, np.int64)
    off[1:] = np.cumsum([t.size for t in texts])
    flat = np.concatenate(texts)
    want = expected(texts, pats, pt)
    d = to_dev(torch, flat, 5)
    b = sm.sm_batch_create(ctx, d, off, pats, np.array(pt, np.int32))
    sm.sm_sync(ctx)
    poff = np.zeros(len(pats) + 1, np.int64)
    poff[1:] = np.cumsum(want)
    counts, dpos = sm.sm_batch_report(b, torch.from_numpy(poff).cuda())
    assert sm.sm_sync(ctx) == sm.SM_OK
    assert np.array_equal(counts.cpu().numpy(), want)
    allpos = dpos.cpu().numpy().view(np.uint64)
    for k, pos in enumerate(oracle_positions(texts, pats, pt, want)):
        assert np.array_equal(allpos[poff[k]:poff[k + 1]], pos), k


def test_batch_tune_keeps_results(torch, ctx):
    # the autotuner re-plans the batch; counts and positions stay exact
    texts, flat, off, pats, pt = make_batch(31, [70_000, 3 * 16384 + 5, 9000], ["markov95", 4, 20], 40, 300)
    want = expected(texts, pats, pt)
    d = to_dev(torch, flat)
    b = sm.sm_batch_create(ctx, d, off, pats, pt)
    best = sm.sm_batch_tune(b, reps=1)
    assert best["ms"] > 0 and best["cand_min"] in (4, 16, 64) and best["stages"] in (0, 2, 3, 4)
    assert np.array_equal(sm.sm_batch_count(b).cpu().numpy()[: len(pats)], want)
    poff = np.zeros(len(pats) + 1, np.int64)
    poff[1:] = np.cumsum(want)
    counts, dpos = sm.sm_batch_report(b, torch.from_numpy(poff).cuda())
    assert sm.sm_sync(ctx) == sm.SM_OK
    assert np.array_equal(counts.cpu().numpy()[: len(pats)], want)
    allpos = dpos.cpu().numpy().view(np.uint64)
    for k, pos in enumerate(oracle_positions(texts, pats, pt, want)):
        assert np.array_equal(allpos[poff[k]:poff[k + 1]], pos), k


def test_batch_coded_texts_long_patterns(torch, ctx):
    # texts of <= 4 symbols run on 2-bit codes in the batch kernel: long
    # patterns (up to the 4096 limit), tile and halo edges, a text with
    # three symbols and one with two, counts and ordered positions
    t4 = synth.uniform(6 * 16384 + 77, 4, seed=0, stream=41)
    t3 = np.frombuffer(b"xyz", np.uint8)[np.random.default_rng(42).integers(0, 3, 3 * 16384 + 5)].copy()
    t2 = synth.uniform(2 * 16384 + 9, 2, seed=0, stream=43)
    texts = [t4, t3, t2]
    r = np.random.default_rng(44)
    pats, pt = [], []
    for x, t in enumerate(texts):
        for m in (1, 3, 17, 64, 65, 300, 1500, 4096):
            for s0 in (0, 16384 - m // 2, t.size - m):
                if 0 <= s0 <= t.size - m:
                    pats.append(t[s0:s0 + m].tobytes())
                    pt.append(x)
        pats.append(b"ACGN")   # a symbol absent from every text
        pt.append(x)
    off = np.zeros(4, np.int64)
    off[1:] = np.cumsum([t.size for t in texts])
    want = expected(texts, pats, pt)
    d = to_dev(torch, np.concatenate(texts), 7)
    b = sm.sm_batch_create(ctx, d, off, pats, np.array(pt, np.int32))
    sm.sm_sync(ctx)
    assert np.array_equal(sm.sm_batch_count(b).cpu().numpy()[: len(pats)], want)
    poff = np.zeros(len(pats) + 1, np.int64)
    poff[1:] = np.cumsum(want)
    counts, dpos = sm.sm_batch_report(b, torch.from_numpy(poff).cuda())
    assert sm.sm_sync(ctx) == sm.SM_OK
    assert np.array_equal(counts.cpu().numpy()[: len(pats)], want)
    allpos = dpos.cpu().numpy().view(np.uint64)
    for k, pos in enumerate(oracle_positions(texts, pats, pt, want)):
        assert np.array_equal(allpos[poff[k]:poff[k + 1]], pos), (k, len(pats[k]), pt[k])
