"""A single search split over ranks (gloo, world size 2 and 3, CPU).

Each rank counts / reports its own start range of the text with its halo;
one all-reduce (counts) or all-gather (report offsets) combines them. The
local search here is the CPU oracle; the result must equal the oracle on the
whole text, for texts and patterns where matches straddle the split points.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _cases():
    r = np.random.default_rng(3)
    t = np.frombuffer(b"ab", np.uint8)[r.integers(0, 2, 5001)].copy()
    yield t, b"ab"
    yield t, t[2490:2510].tobytes()          # straddles the split of 2 and 3 ranks
    yield np.full(97, ord("a"), np.uint8), b"aaaa"   # overlaps everywhere
    yield t[:3].copy(), b"abab"             # m > n
    yield t[:7].copy(), t[:7].tobytes()     # m = n


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    from paper_1612_01506_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = []
    for t, p in _cases():
        n, m = t.size, len(p)
        c = shard.sharded_count(lambda b0, b1: oracle.naive_count(p, t[b0:b1]), n, m)
        first, pos, total = shard.sharded_report(lambda b0, b1: oracle.naive_report(p, t[b0:b1])[0].tolist(), n, m)
        out.append((c, first, pos, total))
    q.put((rank, out))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_search_gloo(world):
    import torch.multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for k, (t, pat) in enumerate(_cases()):
        want_pos, want = oracle.naive_report(pat, t)
        got_pos = []
        for r in range(world):
            c, first, pos, total = res[r][k]
            assert c == want and total == want
            assert first == len(got_pos)
            got_pos += pos
        assert np.array_equal(np.array(got_pos, np.uint64), want_pos), k


def test_ranges_cover_every_start_once():
    from paper_1612_01506_gb300 import shard
    for n in (0, 1, 5, 100, 1001):
        for m in (1, 2, 7, 100, 2000):
            for world in (1, 2, 3, 8):
                owned = []
                for r in range(world):
                    s0, s1 = shard.start_range(n, m, r, world)
                    b0, b1 = shard.text_range(n, m, r, world)
                    owned += list(range(s0, s1))
                    if s1 > s0:
                        assert b0 == s0 and b1 == s1 + m - 1 <= n   # every owned start's match fits
                assert owned == list(range(max(n - m + 1, 0)))


@pytest.mark.gpu
def test_sharded_slices_on_gpu():
    # the per-rank work of a sharded search run on one GPU, rank after rank:
    # sm_count / sm_report on each rank's text slice (start range + halo)
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    import oracle
    from paper_1612_01506_gb300 import shard, sm, synth
    __graft_entry__.build()
    ctx = sm.sm_create(0)
    t = synth.markov95(3 * 16384 * 8 + 1234, seed=0, stream=77)
    d = torch.from_numpy(t).cuda()
    r = np.random.default_rng(78)
    for m in (2, 9, 64, 700):
        for _ in range(3):
            s0 = int(r.integers(0, t.size - m + 1))
            p = t[s0:s0 + m].tobytes()
            want_pos, want = oracle.naive_report(p, t)
            for world in (2, 3, 8):
                total, allpos = 0, []
                for rank in range(world):
                    b0, b1 = shard.text_range(t.size, m, rank, world)
                    if b1 - b0 < m:
                        continue
                    hist = oracle.histogram(t[b0:b1])   # the slice's own symbol counts
                    total += int(sm.sm_count(ctx, d[b0:b1], p, hist=hist).item())
                    pos, c = sm.sm_report(ctx, d[b0:b1], p, want + 1, hist=hist)
                    allpos += (pos[: int(c.item())].cpu().numpy().view(np.uint64) + np.uint64(b0)).tolist()
                assert total == want, (m, world)
                assert np.array_equal(np.array(allpos, np.uint64), want_pos), (m, world)
