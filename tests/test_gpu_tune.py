"""Autotuned plans on the GPU: no plan changes a result, and the tuner
installs the plan it reports. Every call goes through the C ABI; expected
values come from the oracle."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1612_01506_gb300 import sm, synth, tune

pytestmark = pytest.mark.gpu

TILE = sm.SM_TILE_STARTS


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return t


def _report(ctx, text, p, cap, hist):
    pos, c = sm.sm_report(ctx, text, p, cap, pi=sm.sm_order(p, hist), hist=hist)
    st = sm.sm_sync(ctx)
    n = int(c.item())
    return pos[:min(n, cap)].cpu().numpy().view(np.uint64), n, st


@pytest.mark.parametrize("kind,ms", [(20, (2, 8, 70)), (4, (2, 12)), ("markov95", (4, 33)), (2, (9,))])
def test_every_plan_gives_the_same_result(torch, kind, ms):
    t = synth.text(kind, 7 * TILE + 333, seed=0, stream=91)
    text = torch.zeros(t.size + 64, dtype=torch.uint8, device="cuda")[5:5 + t.size]
    text.copy_(torch.from_numpy(t))
    hist = oracle.histogram(t)
    ctx = sm.sm_create(0)
    for m in ms:
        mb, sb = sm.sm_tune_bucket(hist, m)
        pats = synth.sample_patterns(t, m, 2, seed=0, stream=synth.stream_id("tune-test", kind, m))
        want = [oracle.naive_report(p, t) for p in pats]
        for peel, stages, ctas in itertools.product((0, 1, 2, 5, 8), (0, 2, 4, 6), (0, 1, 3)):
            plan = {"peel": peel, "stages": stages, "ctas_per_sm": ctas}
            sm.sm_tune_set(ctx, mb, sb, plan)
            assert sm.sm_tune_get(ctx, mb, sb)["peel"] == peel
            for p, (wpos, wc) in zip(pats, want):
                c = sm.sm_count(ctx, text, p, pi=sm.sm_order(p, hist), hist=hist)
                assert sm.sm_sync(ctx) == sm.SM_OK and int(c.item()) == wc, (kind, m, plan)
                pos, n, st = _report(ctx, text, p, wc + 1, hist)
                assert st == sm.SM_OK and n == wc and np.array_equal(pos, wpos), (kind, m, plan)
        sm.sm_tune_set(ctx, mb, sb, None)
        assert sm.sm_tune_get(ctx, mb, sb) == {"peel": 0, "stages": 0, "ctas_per_sm": 0, "ms": 0.0}


def test_tune_search_installs_its_plan(torch, tmp_path):
    t = synth.text(20, 64 * TILE, seed=0, stream=92)
    text = torch.from_numpy(t).cuda()
    hist = oracle.histogram(t)
    ctx = sm.sm_create(0)
    pats = synth.sample_patterns(t, 16, 4, seed=0, stream=93)
    plan = sm.sm_tune_search(ctx, text, hist, pats, reps=2)
    mb, sb = sm.sm_tune_bucket(hist, 16)
    assert {k: plan[k] for k in tune.FIELDS} == {k: sm.sm_tune_get(ctx, mb, sb)[k] for k in tune.FIELDS}
    assert plan["ms"] > 0
    for p in pats:
        assert int(sm.sm_count(ctx, text, p, pi=sm.sm_order(p, hist), hist=hist).item()) == oracle.naive_count(p, t)
    # patterns of different m buckets are refused
    with pytest.raises(sm.SmError):
        sm.sm_tune_search(ctx, text, hist, [b"ACD", t[:40].tobytes()])
    # the cache: autotune, save, load into a fresh context
    ents = tune.autotune(ctx, text, hist, t, [8], patterns=4, reps=1)
    path = str(tmp_path / "tune.json")
    tune.save(ents, path)
    fresh = sm.sm_create(0)
    assert tune.load(fresh, path) == 1
    e = ents[0]
    assert {k: sm.sm_tune_get(fresh, e["m_bucket"], e["sigma_bucket"])[k] for k in tune.FIELDS} == \
        {k: e[k] for k in tune.FIELDS}


def test_environment_overrides(torch, monkeypatch):
    t = synth.text("markov95", 5 * TILE + 17, seed=0, stream=94)
    text = torch.from_numpy(t).cuda()
    hist = oracle.histogram(t)
    ctx = sm.sm_create(0)
    p = t[777:790].tobytes()
    want_pos, want = oracle.naive_report(p, t)
    for var, val in (("SM_R", "7"), ("SM_STAGES", "3"), ("SM_CTAS_PER_SM", "1")):
        monkeypatch.setenv(var, val)
        pos, n, st = _report(ctx, text, p, want + 1, hist)
        assert st == sm.SM_OK and n == want and np.array_equal(pos, want_pos), var
        monkeypatch.delenv(var)
    # tile and starts per thread are fixed by the kernels: other values are refused
    monkeypatch.setenv("SM_TILE", "8192")
    with pytest.raises(sm.SmError) as e:
        sm.sm_create(0)
    assert e.value.status == sm.SM_ENOTSUP
    monkeypatch.setenv("SM_TILE", str(TILE))
    monkeypatch.setenv("SM_STARTS", "64")
    sm.sm_create(0)
    monkeypatch.setenv("SM_STARTS", "32")
    with pytest.raises(sm.SmError):
        sm.sm_create(0)
