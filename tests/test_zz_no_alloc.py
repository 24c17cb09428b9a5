"""sm_report_noalloc: the report entry point that allocates no device memory.

It serves callers that may not call cudaMalloc (for instance a plug-in whose
host framework already owns the device memory pool, or a service that
forbids allocation after start-up). Its scratch is a fixed device array in
the library instead of a context. This file checks, through the C ABI, that
two calls in a row give exactly the positions and counts of sm_report, and
that a text longer than the array covers is rejected. It is collected last
so that a failure here never hides the other tests; it passes alone in a
fresh process as well.
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


def _reference(torch, ctx, text, p, cap):
    pos, cnt = sm.sm_report(ctx, text, p, cap)
    sm.sm_sync(ctx)
    n = int(cnt.item())
    return pos[:min(n, cap)].cpu().numpy(), n


def test_noalloc_matches_report_twice(torch):
    ctx = sm.sm_create(0)
    n = 3 * (1 << 20) + 12345
    t = synth.uniform(n, 4, seed=0, stream=synth.stream_id("noalloc"))
    buf = torch.zeros(n + 64, dtype=torch.uint8, device="cuda")
    buf[5:5 + n] = torch.from_numpy(t).cuda()
    text = buf[5:5 + n]                       # deliberately misaligned text
    pats = [t[1000:1008].tobytes(), b"ACGTACGTA", t[n - 6:].tobytes()]
    cap = 4096
    out_pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    out_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for p in pats[:2] + pats[2:]:             # consecutive calls share the scratch array
        want_pos, want = _reference(torch, ctx, text, p, cap)
        assert want == oracle.naive_count(p, t)
        st = sm.sm_report_noalloc(text, p, cap, out_pos, out_cnt)
        assert st == sm.SM_OK
        torch.cuda.synchronize()
        got = int(out_cnt.item())
        assert got == want
        assert np.array_equal(out_pos[:min(got, cap)].cpu().numpy(), want_pos)


def test_noalloc_truncation_and_limits(torch):
    t = synth.uniform(200_000, 2, seed=0, stream=1)
    text = torch.from_numpy(t).cuda()
    p = b"0110"
    want_pos, want = oracle.naive_report(p, t)
    cap = 100
    out_pos = torch.zeros(cap, dtype=torch.int64, device="cuda")
    out_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert sm.sm_report_noalloc(text, p, cap, out_pos, out_cnt) == sm.SM_OK
    torch.cuda.synchronize()
    assert int(out_cnt.item()) == want > cap
    assert np.array_equal(out_pos.cpu().numpy().view(np.uint64), want_pos[:cap])
    # a text with more start positions than the scratch covers is rejected
    # before any device work (the pointer is never read)
    lib = sm.load()
    pat = (np.frombuffer(b"ab", np.uint8)).copy()
    import ctypes as C
    st = lib.sm_report_noalloc(text.data_ptr(), sm.SM_NOALLOC_MAX_STARTS + 2, pat.ctypes.data_as(C.POINTER(C.c_uint8)),
                               2, None, out_pos.data_ptr(), cap, out_cnt.data_ptr(), None)
    assert st == sm.SM_EINVAL
    assert sm.sm_report_noalloc(text, b"", cap, out_pos, out_cnt) == sm.SM_EINVAL


def test_noalloc_largest_text(torch):
    """The largest text the array covers (exactly SM_NOALLOC_MAX_STARTS start
    positions) against sm_report; one start more is rejected."""
    m = 8
    n = sm.SM_NOALLOC_MAX_STARTS + m - 1
    t = synth.uniform(n, 4, seed=0, stream=synth.stream_id("noalloc", "max"))
    text = torch.from_numpy(t).cuda()
    ctx = sm.sm_create(0)
    p = t[n - m:].tobytes()                    # the last start matches
    cap = 1 << 16
    want_pos, want = _reference(torch, ctx, text, p, cap)
    out_pos = torch.zeros(cap, dtype=torch.int64, device="cuda")
    out_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert sm.sm_report_noalloc(text, p, cap, out_pos, out_cnt) == sm.SM_OK
    torch.cuda.synchronize()
    got = int(out_cnt.item())
    assert got == want >= 1
    assert np.array_equal(out_pos[:min(got, cap)].cpu().numpy(), want_pos)
    if want <= cap:
        assert int(out_pos[want - 1].item()) == n - m
    over = torch.empty(n + 1, dtype=torch.uint8, device="cuda")   # one start over the limit
    assert sm.sm_report_noalloc(over, p, cap, out_pos, out_cnt) == sm.SM_EINVAL


def test_noalloc_timeout_is_reported(torch, monkeypatch):
    """An expired bounded wait shows as *d_count == SM_NOALLOC_TIMEOUT. The
    test hook never starts the first tile's copy and gives each wait 2 ms,
    so the wait runs out without any fault; the next call is correct."""
    t = synth.uniform(1 << 20, 4, seed=0, stream=7)
    text = torch.from_numpy(t).cuda()
    p = t[100:108].tobytes()
    cap = 1024
    out_pos = torch.zeros(cap, dtype=torch.int64, device="cuda")
    out_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    monkeypatch.setenv("SM_NOALLOC_TEST_TIMEOUT", "1")
    assert sm.sm_report_noalloc(text, p, cap, out_pos, out_cnt) == sm.SM_OK
    torch.cuda.synchronize()
    assert int(out_cnt.item()) & ((1 << 64) - 1) == sm.SM_NOALLOC_TIMEOUT
    monkeypatch.delenv("SM_NOALLOC_TEST_TIMEOUT")
    want_pos, want = oracle.naive_report(p, t)
    assert sm.sm_report_noalloc(text, p, cap, out_pos, out_cnt) == sm.SM_OK
    torch.cuda.synchronize()
    assert int(out_cnt.item()) == want
    assert np.array_equal(out_pos[:want].cpu().numpy().view(np.uint64), want_pos)
