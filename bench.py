#!/usr/bin/env python3
"""Benchmark: text GB/s per pattern of the SIMD-naive search on GB300.

Default workload (the paper-method sweep at n = 1 GiB): texts of 2^30 bytes,
i.i.d. uniform over sigma in {2, 4, 20, 64} plus English-like Markov text over
95 printable bytes; pattern lengths m in {2, 4, 8, ..., 1024}; 100 patterns per
(sigma, m) copied from the text at seeded offsets; count and report variants.

One step = the whole hot path over the sweep: the byte histogram of each
text, the rarest-first order of each pattern, and one count plus one report
per pattern. value = text bytes scanned per second over all searches
(n bytes per search). Inputs (1 GiB each) are larger than L2, so no flush is
needed between iterations.

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and
torch.cuda.synchronize(), CUDA events on the launching stream, max over ranks.
With --gpus N > 1 (torchrun) each rank searches its own patterns on its own
GPU with no collective on the data path (weak scaling).

--impl reference times the CPU oracle (plain Algorithm 1, threaded over the
host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KINDS_DEFAULT = "2,4,20,64,markov95"
MS_DEFAULT = "2,4,8,16,32,64,128,256,512,1024"
METRIC = "text GB/s per pattern (count+report sweep, n=1 GiB)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=1 << 30)
    ap.add_argument("--kinds", default=KINDS_DEFAULT)
    ap.add_argument("--ms", default=MS_DEFAULT)
    ap.add_argument("--patterns", type=int, default=100)
    ap.add_argument("--variants", default="count,report")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--json-detail", default="")
    ap.add_argument("--peel", type=int, default=0, help="peeling factor r (0 = automatic)")
    ap.add_argument("--stages", type=int, default=0, help="scan pipeline depth (0 = library default)")
    ap.add_argument("--ctas", type=int, default=0, help="scan CTAs (0 = one resident wave)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-counting leg (256 MiB Markov text, 4096 patterns; on by default)")
    ap.add_argument("--batch-only", action="store_true", help="measure only the batched counting")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the serving leg (4 GiB resident text, Poisson arrivals; on by default)")
    ap.add_argument("--serve-only", action="store_true", help="measure only the serving loop")
    ap.add_argument("--no-latency", action="store_true",
                    help="skip the single-search latency leg (1 MiB ACGT text, m = 8; on by default)")
    ap.add_argument("--latency-only", action="store_true", help="measure only the single-search latency")
    ap.add_argument("--no-multi", action="store_true",
                    help="skip the packed-texts leg (counts and positions over 20,000 texts, ~35 GB; on by default)")
    ap.add_argument("--multi-only", action="store_true", help="measure only the packed-texts batch")
    ap.add_argument("--multi-texts", type=int, default=20000)
    ap.add_argument("--tune-only", action="store_true",
                    help="autotune every (sigma, m) bucket of the sweep and compare tuned with untuned counts")
    ap.add_argument("--tune-save", default="", help="--tune-only: merge the plans into this JSON cache")
    ap.add_argument("--compare-stats", action="store_true",
                    help="early-exit counters: compares per 16-start chunk (builds and uses a profiling "
                         "library with -DSMK_COUNT_COMPARES=1)")
    ap.add_argument("--orders-only", action="store_true",
                    help="measure only the comparison orders of Sec. 2.2 / 2.4 (pi_freq, pi_h, pi_hs)")
    ap.add_argument("--orders-kinds", default="markov95,20,4")
    ap.add_argument("--orders-ms", default=",".join(str(m) for m in range(4, 65, 4)))
    ap.add_argument("--orders-peels", default="0,2,3,5")
    ap.add_argument("--serve-rates", default="100,200,500,1000,2000,4000")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-chunk-mib", type=int, default=256, help="serving: text chunk per step (MiB)")
    ap.add_argument("--serve-report-batch-min", type=int, default=32,
                    help="serving: waiting reports that trigger one batched report")
    ap.add_argument("--serve-burst-below", type=int, default=4,
                    help="serving: at most this many queries in flight and none waiting: all chunks in one launch")
    return ap.parse_args()


def kinds_of(s):
    return [k if k == "markov95" else int(k) for k in s.split(",") if k]


# ---------------------------------------------------------------- distributed

def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- workload

def make_workload(args, rank):
    from paper_1612_01506_gb300 import synth
    kinds, ms = kinds_of(args.kinds), [int(x) for x in args.ms.split(",") if x]
    texts, pats = {}, {}
    for kind in kinds:
        t = np.empty(args.n, dtype=np.uint8)
        synth.text(kind, args.n, seed=0, stream=synth.stream_id("sweep", kind), out=t)
        texts[kind] = t
        for m in ms:
            pats[(kind, m)] = synth.sample_patterns(t, m, args.patterns, seed=rank,
                                                    stream=synth.stream_id("pat", kind, m))
    return kinds, ms, texts, pats


def scan_traffic(n, record="scan_traffic.json"):
    """DRAM bytes per count launch at text size n from a committed ncu
    capture under profiles/, if the kernels' sources are unchanged since
    (else None)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", record)) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as g:
                h.update(g.read())
        if h.hexdigest() != rec["sources_sha256"]:
            return None
        per = sum(rec["dram_bytes_per_launch"]) / len(rec["dram_bytes_per_launch"])
        return round(per * n / rec["text_bytes"])
    except (OSError, KeyError, ValueError, ZeroDivisionError):
        return None


def report_traffic_ratio(record="report_traffic.json"):
    """DRAM bytes of a report's kernels over its algorithmic bytes n + 8 occ,
    summed over the reports of a committed ncu capture under profiles/ (one
    per (sigma, m) cell), if the sources it depends on are unchanged since
    (else None)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", record)) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as g:
                h.update(g.read())
        if h.hexdigest() != rec["sources_sha256"]:
            return None
        return sum(c["dram_bytes"] for c in rec["cells"]) / sum(c["alg_bytes"] for c in rec["cells"])
    except (OSError, KeyError, ValueError, ZeroDivisionError):
        return None


def peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------- GPU arm

def run_gpu(args, world, rank, local):
    import torch
    from paper_1612_01506_gb300 import sm

    kinds, ms, texts, pats = make_workload(args, rank)
    variants = [v for v in args.variants.split(",") if v]
    dev = torch.device("cuda", local)
    ctx = sm.sm_create(local)
    if args.stages:
        sm.sm_set_knob(ctx, sm.SM_KNOB_STAGES, args.stages)
    if args.ctas:
        sm.sm_set_knob(ctx, sm.SM_KNOB_GRID, args.ctas)
    stream = torch.cuda.current_stream()
    d_texts = {k: torch.from_numpy(texts[k]).to(dev) for k in kinds}
    counts = torch.zeros(len(ms) * args.patterns * 2 + 8, dtype=torch.int64, device=dev)
    max_cap = args.n  # any report fits: count <= n - m + 1
    d_pos = torch.empty(max_cap, dtype=torch.int64, device=dev) if "report" in variants else None
    hist_dev = torch.empty((len(kinds), 256), dtype=torch.int64, device=dev)

    # host-side order and histogram are computed once per text outside timing,
    # and again inside every step (a2 is part of the step)
    hists = {}
    for i, k in enumerate(kinds):
        sm.sm_histogram(ctx, d_texts[k], out=hist_dev[i])
    torch.cuda.synchronize()
    for i, k in enumerate(kinds):
        hists[k] = hist_dev[i].cpu().numpy().view(np.uint64).copy()

    # (start, end) events around each count and each report of the timed
    # steps, per (text, m): the per-(sigma, m) table, the gate and the two
    # rooflines come from them
    ev = {}
    launches = {"n": 0}
    P = args.patterns

    def step(timed: bool, text_map):
        for i, k in enumerate(kinds):
            sm.sm_histogram(ctx, text_map[k], out=hist_dev[i])
            launches["n"] += 1
            h = hists[k]
            for m in ms:
                pis = [sm.sm_order(p, h) for p in pats[(k, m)]]
                for var in variants:
                    lst = ev.setdefault((var, k, m), []) if timed else None
                    for j, p in enumerate(pats[(k, m)]):
                        if timed:
                            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                            a.record(stream)
                        if var == "count":
                            sm.sm_count(ctx, text_map[k], p, pi=pis[j], hist=h, peel=args.peel,
                                        out=counts[j:j + 1])
                            launches["n"] += 1
                        else:
                            sm.sm_report(ctx, text_map[k], p, max_cap, pi=pis[j], hist=h, peel=args.peel,
                                         out_pos=d_pos, out_count=counts[P + j:P + j + 1])
                            launches["n"] += 3
                        if timed:
                            b.record(stream)
                            lst.append((a, b))

    # matches per pattern (for the report's algorithmic bytes n + 8 occ)
    occ = {}
    for k in kinds:
        for m in ms:
            for j, p in enumerate(pats[(k, m)]):
                sm.sm_count(ctx, d_texts[k], p, out=counts[j:j + 1])
            occ[(k, m)] = [int(x) for x in counts[:P].cpu().numpy()]

    for _ in range(args.warmup):
        step(False, d_texts)
    if sm.sm_sync(ctx) != sm.SM_OK:
        raise RuntimeError("deferred device status after warm-up")
    launches["n"] = 0

    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step(True, d_texts)
        t1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    elapsed = t0.elapsed_time(t1) / 1e3
    elapsed = max_over_ranks(elapsed, world)
    st = sm.sm_sync(ctx)
    if st != sm.SM_OK:
        raise RuntimeError(f"deferred device status {st} in timed region")

    searches_per_step = len(kinds) * len(ms) * args.patterns * len(variants)
    bytes_per_step = searches_per_step * args.n
    value = world * bytes_per_step * args.steps / elapsed / 1e9

    # per-(sigma, m) mean launch times; count: n bytes, report: n + 8 occ
    peak, peak_kind = peak_gbs()
    durs = {key: [a.elapsed_time(b) / 1e3 for a, b in v] for key, v in ev.items()}
    detail, gate_cells = {}, {}
    for k in kinds:
        for m in ms:
            cell = {}
            if ("count", k, m) in durs:
                t = statistics.mean(durs[("count", k, m)])
                cell["count_gbs"] = round(args.n / t / 1e9, 1)
                cell["count_frac"] = round(args.n / t / 1e9 / peak, 3)
                if k != 2 and m <= 64:
                    gate_cells[f"{k}/m{m}"] = cell["count_frac"]
            if ("report", k, m) in durs:
                t = statistics.mean(durs[("report", k, m)])
                ab = args.n + 8 * statistics.mean(occ[(k, m)])
                cell["report_gbs"] = round(args.n / t / 1e9, 1)
                cell["report_frac"] = round(ab / t / 1e9 / peak, 3)
            detail[f"{k}/m{m}"] = cell
    gate = None
    if gate_cells:
        gate = {"rule": "count kernel >= 0.70 of measured HBM peak for m <= 64 on sigma >= 4",
                "pass": min(gate_cells.values()) >= 0.70, "min_frac": min(gate_cells.values()),
                "cells": gate_cells}

    def roofline(var, kernel, alg):
        tot_t = tot_b = 0.0
        nl = 0
        for (v, k, m), ds in durs.items():
            if v != var:
                continue
            for j, d in enumerate(ds):
                tot_t += d
                tot_b += alg(k, m, j % P)
                nl += 1
        if not nl:
            return None
        ach = tot_b / tot_t / 1e9
        return {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                "peak_source": peak_kind, "kernel": kernel, "launches": nl}

    roof = roofline("count", "scan_kernel<count>", lambda k, m, j: args.n)
    if roof:
        roof["traffic"] = scan_traffic(args.n)
    roof_rep = roofline("report", "report: scan_kernel<tile count> + range_sum_kernel + bitmap_write_kernel "
                        "(found bits) or scan_kernel<sparse> + scan_kernel<write> (rescan)",
                        lambda k, m, j: args.n + 8 * occ[(k, m)][j])
    if roof_rep:
        roof_rep["bytes"] = "n + 8 * matches per report"
        # DRAM bytes per report: the captured ratio of traffic to n + 8 occ
        # over one report per (sigma, m) cell, applied to this sweep's mean
        ratio = report_traffic_ratio()
        roof_rep["traffic"] = None
        if ratio:
            mean_alg = statistics.mean(args.n + 8 * statistics.mean(occ[(k, m)]) for k in kinds for m in ms)
            roof_rep["traffic"] = round(ratio * mean_alg)
            roof_rep["traffic_over_bytes"] = round(ratio, 4)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, ctx, kinds, ms, pats, hists, texts, dev, stream, d_texts, variants, world)

    return {"value": value, "elapsed": elapsed, "bytes_per_step": bytes_per_step, "detail": detail,
            "roofline": roof, "report_roofline": roof_rep, "gate": gate, "clocks": clk.summary(), "e2e": e2e,
            "launches": launches["n"], "searches_per_step": searches_per_step}


def run_e2e(args, ctx, kinds, ms, pats, hists, texts, dev, stream, d_texts, variants, world):
    """Same sweep through the public API from pinned host texts: every step
    copies each text host->device, searches, and reads the counts back."""
    import torch
    from paper_1612_01506_gb300 import sm
    pinned = {k: torch.from_numpy(texts[k]).pin_memory() for k in kinds}
    counts = torch.zeros(len(ms) * args.patterns * 2, dtype=torch.int64, device=dev)
    host_counts = torch.zeros_like(counts, device="cpu").pin_memory()
    d_pos = torch.empty(args.n, dtype=torch.int64, device=dev) if "report" in variants else None
    h2d = d2h = 0

    def one():
        nonlocal h2d, d2h
        for k in kinds:
            d_texts[k].copy_(pinned[k], non_blocking=True)
            h2d += args.n
            h = sm.sm_histogram(ctx, d_texts[k]).cpu().numpy().view(np.uint64)
            d2h += 256 * 8
            slot = 0
            for m in ms:
                for p in pats[(k, m)]:
                    pi = sm.sm_order(p, h)
                    if "count" in variants:
                        sm.sm_count(ctx, d_texts[k], p, pi=pi, hist=h, out=counts[slot:slot + 1])
                    slot += 1
                    if "report" in variants:
                        sm.sm_report(ctx, d_texts[k], p, args.n, pi=pi, hist=h, out_pos=d_pos,
                                     out_count=counts[slot:slot + 1])
                    slot += 1
                host_counts.copy_(counts, non_blocking=True)
                d2h += counts.numel() * 8
            torch.cuda.synchronize()

    one()   # warm-up
    h2d = d2h = 0
    steps = max(1, min(args.steps, 2))
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    el = max_over_ranks(time.perf_counter() - t0, world)
    bytes_scanned = len(kinds) * len(ms) * args.patterns * len(variants) * args.n * steps * world
    return {"value": round(bytes_scanned / el / 1e9, 1), "unit": "GB/s",
            "h2d_bytes_per_step": h2d // steps, "d2h_bytes_per_step": d2h // steps}


# ---------------------------------------------------------------- batched counting

def run_batch(args, local, steps=3, warmup=2):
    """Batched counting: one 256 MiB Markov-95 text, 4096 patterns with lengths
    log-uniform in [2, 1024], 80% copied from the text and 20% random over its
    alphabet; int64 counts. patterns*GB/s = patterns x text bytes / time, for
    the one persistent launch and for one sm_count launch per pattern."""
    import torch
    from paper_1612_01506_gb300 import sm, synth
    n, npat = 256 << 20, 4096
    t = synth.markov95(n, seed=0, stream=synth.stream_id("batch", "markov95"))
    r = np.random.default_rng(0)
    lens = np.exp(r.uniform(np.log(2), np.log(1024), npat)).astype(np.int64)
    offs = synth.below(npat, n, 0, synth.stream_id("batch", "offs"))
    alpha = np.frombuffer(synth.MARKOV95, np.uint8)
    pats = []
    for k in range(npat):
        m = int(lens[k])
        if r.random() < 0.8:
            o = min(int(offs[k]), n - m)
            pats.append(t[o:o + m].tobytes())
        else:
            pats.append(alpha[r.integers(0, alpha.size, m)].tobytes())
    dev = torch.device("cuda", local)
    ctx = sm.sm_create(local)
    d = torch.from_numpy(t).to(dev)
    off = np.array([0, n], np.int64)
    b = sm.sm_batch_create(ctx, d, off, pats, np.zeros(npat, np.int32))
    out = torch.zeros(npat, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        sm.sm_batch_count(b, out=out)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        sm.sm_batch_count(b, out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_batch = ev0.elapsed_time(ev1) / 1e3 / steps
    batch_counts = out.cpu().numpy().copy()
    # the autotuner (plan parameters by measurement), then the same timing
    tuning = sm.sm_batch_tune(b, reps=2)
    for _ in range(warmup):
        sm.sm_batch_count(b, out=out)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        sm.sm_batch_count(b, out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_tuned = ev0.elapsed_time(ev1) / 1e3 / steps
    tuned_agree = bool(np.array_equal(out.cpu().numpy(), batch_counts))
    # one launch per pattern, same orders (rarest first under the text histogram)
    hist = sm.sm_histogram(ctx, d).cpu().numpy().view(np.uint64).copy()
    single = torch.zeros(npat, dtype=torch.int64, device=dev)
    orders = [sm.sm_order(p, hist) for p in pats]
    for k in range(min(npat, 64)):
        sm.sm_count(ctx, d, pats[k], pi=orders[k], hist=hist, out=single[k:k + 1])
    torch.cuda.synchronize()
    ev0.record(stream)
    for k in range(npat):
        sm.sm_count(ctx, d, pats[k], pi=orders[k], hist=hist, out=single[k:k + 1])
    ev1.record(stream)
    torch.cuda.synchronize()
    t_single = ev0.elapsed_time(ev1) / 1e3
    agree = bool(np.array_equal(single.cpu().numpy(), batch_counts))
    pgb = npat * n / 1e9
    return {"workload": "batched counting: 256 MiB Markov-95 text, 4096 patterns, m log-uniform [2,1024], "
                        "80% from the text", "batch_ms": round(t_batch * 1e3, 3),
            "batch_patterns_gbs": round(pgb / t_batch, 1), "single_launch_ms": round(t_single * 1e3, 3),
            "single_launch_patterns_gbs": round(pgb / t_single, 1), "speedup": round(t_single / t_batch, 2),
            "counts_agree": agree, "tuned": tuning, "tuned_batch_ms": round(t_tuned * 1e3, 3),
            "tuned_patterns_gbs": round(pgb / t_tuned, 1), "tuned_counts_agree": tuned_agree}


def run_latency(args, local, reps=200):
    """Latency of one search on a small, L2-resident text: n = 1 MiB of
    uniform ACGT (seed 0), m = 8 copied from the text. Device time per call
    (CUDA events around back-to-back calls) and call latency (from the host
    call to the result on the host, each call synchronised), median over
    reps, for sm_count and sm_report."""
    import torch
    from paper_1612_01506_gb300 import sm, synth
    n, m = 1 << 20, 8
    t = synth.uniform(n, 4, seed=0, stream=0)
    p = t[1000:1000 + m].tobytes()
    dev = torch.device("cuda", local)
    ctx = sm.sm_create(local)
    d = torch.from_numpy(t).to(dev)
    hist = sm.sm_histogram(ctx, d).cpu().numpy().view(np.uint64).copy()
    out = torch.zeros(1, dtype=torch.int64, device=dev)
    cnt = int(sm.sm_count(ctx, d, p, hist=hist, out=out).item())
    pos = torch.empty(max(cnt, 1), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    res = {"workload": "1 MiB uniform ACGT (seed 0), m = 8 from the text, L2-resident", "count": cnt}
    for name, call in (("count", lambda: sm.sm_count(ctx, d, p, hist=hist, out=out)),
                       ("report", lambda: sm.sm_report(ctx, d, p, cnt, hist=hist, out_pos=pos, out_count=out))):
        for _ in range(20):
            call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            call()
        e1.record(stream)
        torch.cuda.synchronize()
        res[f"{name}_device_us"] = round(e0.elapsed_time(e1) * 1e3 / reps, 2)
        lat = []
        for _ in range(reps):
            t0 = time.perf_counter()
            call()
            int(out.item())
            lat.append(time.perf_counter() - t0)
        res[f"{name}_call_us_p50"] = round(float(np.percentile(lat, 50)) * 1e6, 1)
        res[f"{name}_call_us_p99"] = round(float(np.percentile(lat, 99)) * 1e6, 1)
    return res


def run_multi(args, local, steps=2, warmup=1):
    """Many packed texts: --multi-texts texts (20,000) with lengths log-uniform
    in [1 KiB, 16 MiB] (about 35 GB together), each over an alphabet drawn
    from {4, 20, Markov-95, 256}, each with 1-8 patterns of length
    log-uniform in [2, 512] (80% copied from the text, 20% random over its
    alphabet). One step = sm_batch_count (counts) and sm_batch_report
    (counts and every ascending position list, into exact-size slices).
    patterns*GB/s = sum over patterns of its text's bytes / time."""
    import concurrent.futures as cf
    import torch
    from paper_1612_01506_gb300 import sm, synth
    nt = args.multi_texts
    r = np.random.default_rng(4)
    lens = np.exp(r.uniform(np.log(1024), np.log(16 << 20), nt)).astype(np.int64)
    kinds = [(4, 20, "markov95", 256)[i] for i in r.integers(0, 4, nt)]
    npt = r.integers(1, 9, nt)
    off = np.zeros(nt + 1, np.int64)
    off[1:] = np.cumsum(lens)
    total = int(off[-1])
    dev = torch.device("cuda", local)
    d = torch.empty(total, dtype=torch.uint8, device=dev)
    # texts generated on the host cores in parallel, staged through 1 GiB
    stage = torch.empty(1 << 30, dtype=torch.uint8).pin_memory()
    sv = stage.numpy()
    pats, pat_text = [], []

    def gen(x):
        return synth.text(kinds[x], int(lens[x]), seed=0, stream=synth.stream_id("multi", x), threads=1)

    x0, used = 0, 0
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        for x, tx in enumerate(ex.map(gen, range(nt))):
            if used + tx.size > sv.size:
                d[off[x0]:off[x0] + used].copy_(stage[:used])
                x0, used = x, 0
            sv[used:used + tx.size] = tx
            used += tx.size
            for _ in range(int(npt[x])):
                m = min(int(np.exp(r.uniform(np.log(2), np.log(512)))), tx.size)
                if r.random() < 0.8:
                    o = int(r.integers(0, tx.size - m + 1))
                    pats.append(tx[o:o + m].tobytes())
                else:
                    a = np.frombuffer(synth.alphabet_of(kinds[x]), np.uint8)
                    pats.append(a[r.integers(0, a.size, m)].tobytes())
                pat_text.append(x)
    d[off[x0]:off[x0] + used].copy_(stage[:used])
    del stage, sv
    npat = len(pats)
    ctx = sm.sm_create(local)
    t0 = time.perf_counter()
    b = sm.sm_batch_create(ctx, d, off, pats, np.array(pat_text, np.int32))
    t_plan = time.perf_counter() - t0
    counts = sm.sm_batch_count(b)
    torch.cuda.synchronize()
    ch = counts.cpu().numpy()[:npat]
    pos_off = np.zeros(npat + 1, np.int64)
    pos_off[1:] = np.cumsum(ch)
    d_off = torch.from_numpy(pos_off).to(dev)
    d_pos = torch.empty(max(int(pos_off[-1]), 1), dtype=torch.int64, device=dev)
    rcounts = torch.empty(npat, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        sm.sm_batch_count(b, out=counts)
        sm.sm_batch_report(b, d_off, d_pos=d_pos, out=rcounts)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tc, tr = 0.0, 0.0
    for _ in range(steps):
        ev[0].record(stream)
        sm.sm_batch_count(b, out=counts)
        ev[1].record(stream)
        sm.sm_batch_report(b, d_off, d_pos=d_pos, out=rcounts)
        ev[2].record(stream)
        torch.cuda.synchronize()
        tc += ev[0].elapsed_time(ev[1]) / 1e3
        tr += ev[1].elapsed_time(ev[2]) / 1e3
    tc, tr = tc / steps, tr / steps
    # the autotuner on this batch, then the counting pass again
    tuning = sm.sm_batch_tune(b, reps=1)
    sm.sm_batch_count(b, out=counts)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(steps):
        sm.sm_batch_count(b, out=counts)
    ev[1].record(stream)
    torch.cuda.synchronize()
    t_tuned = ev[0].elapsed_time(ev[1]) / 1e3 / steps
    tuned_agree = bool(np.array_equal(counts.cpu().numpy()[:npat], ch))
    status = sm.sm_sync(ctx)
    # cross-check against single-pattern calls on a sample of patterns
    rs = np.random.default_rng(5)
    sample = rs.choice(npat, size=min(npat, 200), replace=False)
    agree = bool(np.array_equal(rcounts.cpu().numpy()[:npat], ch))
    allpos = None
    for k in sample:
        x = pat_text[k]
        tx = d[off[x]:off[x + 1]]
        c = int(ch[k])
        pos, cnt = sm.sm_report(ctx, tx, pats[k], max(c, 1))
        if int(cnt.item()) != c:
            agree = False
            break
        got = d_pos[pos_off[k]:pos_off[k + 1]]
        if not torch.equal(got, pos[:c]):
            agree = False
            break
    pgb = float(sum(int(lens[x]) for x in pat_text)) / 1e9
    return {"workload": f"{nt} packed texts ({total / 1e9:.1f} GB), lengths log-uniform [1 KiB, 16 MiB], "
                        f"sigma in {{4,20,markov95,256}}, {npat} patterns (1-8 per text, m log-uniform [2,512])",
            "texts_bytes": total, "patterns": npat, "positions": int(pos_off[-1]),
            "plan_s": round(t_plan, 3), "count_ms": round(tc * 1e3, 3), "report_ms": round(tr * 1e3, 3),
            "count_patterns_gbs": round(pgb / tc, 1), "report_patterns_gbs": round(pgb / tr, 1),
            "status": status, "sample_agrees_with_single_calls": agree, "sample": int(sample.size),
            "tuned": tuning, "tuned_count_ms": round(t_tuned * 1e3, 3),
            "tuned_count_patterns_gbs": round(pgb / t_tuned, 1), "tuned_counts_agree": tuned_agree}


def run_tune(args, local, reps=3):
    """Autotuner per (m, sigma) bucket on the sweep's texts: for each text and
    m, the count GB/s of --patterns patterns under the library's defaults,
    then sm_tune_search on 24 other patterns of the bucket (seed 1), then the
    same timed patterns under the tuned plan. The counts must not change."""
    import torch
    from paper_1612_01506_gb300 import sm, synth, tune
    kinds, ms = kinds_of(args.kinds), [int(x) for x in args.ms.split(",") if x]
    dev = torch.device("cuda", local)
    ctx = sm.sm_create(local)
    stream = torch.cuda.current_stream()
    counts = torch.zeros(args.patterns, dtype=torch.int64, device=dev)
    out = {"workload": f"tune: n={args.n}, sigma {args.kinds} x m {args.ms}, {args.patterns} timed patterns",
           "cells": {}, "counts_agree": True, "entries": []}

    def gbs(d, pats, pis, hist):
        def one():
            for j, p in enumerate(pats):
                sm.sm_count(ctx, d, p, pi=pis[j], hist=hist, out=counts[j:j + 1])
        one()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return round(len(pats) * args.n / min(ts) / 1e9, 1), counts.cpu().numpy().copy()

    for kind in kinds:
        t = np.empty(args.n, dtype=np.uint8)
        synth.text(kind, args.n, seed=0, stream=synth.stream_id("sweep", kind), out=t)
        d = torch.from_numpy(t).to(dev)
        hist = sm.sm_histogram(ctx, d).cpu().numpy().view(np.uint64).copy()
        for m in ms:
            pats = synth.sample_patterns(t, m, args.patterns, seed=0, stream=synth.stream_id("pat", kind, m))
            pis = [sm.sm_order(p, hist) for p in pats]
            mb, sb = sm.sm_tune_bucket(hist, m)
            sm.sm_tune_set(ctx, mb, sb, None)
            base, c0 = gbs(d, pats, pis, hist)
            ent = tune.autotune(ctx, d, hist, t, [m], patterns=24, reps=reps)[0]
            tuned, c1 = gbs(d, pats, pis, hist)
            if not np.array_equal(c0, c1):
                out["counts_agree"] = False
            out["entries"].append(ent)
            out["cells"][f"{kind}/m{m}"] = {"default_gbs": base, "tuned_gbs": tuned,
                                            "plan": {k: ent[k] for k in tune.FIELDS}}
        del d
    out["tuned_not_slower_cells"] = sum(1 for c in out["cells"].values() if c["tuned_gbs"] >= 0.99 * c["default_gbs"])
    out["cells_total"] = len(out["cells"])
    if args.tune_save:
        tune.write_entries(args.tune_save, tune.gpu_key(local), out["entries"])
    return out


def run_compare_stats(args, local):
    """Early-exit counters from a profiling build of the library (its scan
    kernels count, per 16-start chunk, the compares of the dense phase and,
    for chunks that survive it, of the sparse phase). Per (text, m): the
    --patterns count searches of the sweep (text histogram, rarest-first
    order). Texts sigma = 4 run on 2-bit codes (a chunk is one 16-start word)."""
    import ctypes as C
    import torch
    from paper_1612_01506_gb300 import build, sm, synth
    os.environ["SM_LIBRARY"] = build.build_lib(out=os.path.join(build.PKG, "_build", "cmpstats"),
                                               defines=("SMK_COUNT_COMPARES=1",))
    lib = sm.load()
    f = lib.sm_debug_compare_stats
    f.restype, f.argtypes = C.c_int, [C.POINTER(C.c_ulonglong), C.c_int]
    stats = (C.c_ulonglong * 4)()
    dev = torch.device("cuda", local)
    ctx = sm.sm_create(local)
    out = {"workload": f"early exit: n={args.n}, sigma {args.kinds} x m {args.ms}, {args.patterns} patterns "
                       "from the text, counts", "cells": {}}
    for kind in kinds_of(args.kinds):
        t = np.empty(args.n, dtype=np.uint8)
        synth.text(kind, args.n, seed=0, stream=synth.stream_id("sweep", kind), out=t)
        d = torch.from_numpy(t).to(dev)
        hist = sm.sm_histogram(ctx, d).cpu().numpy().view(np.uint64).copy()
        for m in [int(x) for x in args.ms.split(",") if x]:
            pats = synth.sample_patterns(t, m, args.patterns, seed=0, stream=synth.stream_id("pat", kind, m))
            f(stats, 1)
            for p in pats:
                sm.sm_count(ctx, d, p, pi=sm.sm_order(p, hist), hist=hist)
            if f(stats, 1) != 0:
                raise RuntimeError("reading the compare counters failed")
            ch, dense, alive, sparse = (int(x) for x in stats)
            out["cells"][f"{kind}/m{m}"] = {
                "compares_per_chunk": round((dense + sparse) / ch, 3), "dense_per_chunk": round(dense / ch, 3),
                "surviving_chunks": round(alive / ch, 5),
                "sparse_per_surviving_chunk": round(sparse / alive, 3) if alive else 0.0}
        del d
    return out


def run_orders(args, local, reps=2):
    """The comparison orders of Sec. 2.2 and 2.4 on the sweep's texts (n =
    --n): rarest first under the text's histogram (pi_freq), and the fixed
    orders pi_h and pi_hs, each with the peel r fixed (Algorithm 4) or chosen
    by the planner (0). Per (text, m): --patterns patterns copied from the
    text; GB/s = patterns x n / time of their count launches (median of reps
    timed passes over the patterns). The counts must not depend on the order."""
    import torch
    from paper_1612_01506_gb300 import sm, synth
    kinds = kinds_of(args.orders_kinds)
    ms = [int(x) for x in args.orders_ms.split(",") if x]
    peels = [int(x) for x in args.orders_peels.split(",") if x]
    dev = torch.device("cuda", local)
    ctx = sm.sm_create(local)
    stream = torch.cuda.current_stream()
    out = {"workload": f"orders: n={args.n}, texts {args.orders_kinds}, m {args.orders_ms}, "
                       f"{args.patterns} patterns from the text, peel {args.orders_peels} (0 = planner)",
           "gbs": {}, "counts_agree": True}
    counts = torch.zeros(args.patterns, dtype=torch.int64, device=dev)
    for kind in kinds:
        t = np.empty(args.n, dtype=np.uint8)
        synth.text(kind, args.n, seed=0, stream=synth.stream_id("sweep", kind), out=t)
        d = torch.from_numpy(t).to(dev)
        hist = sm.sm_histogram(ctx, d).cpu().numpy().view(np.uint64).copy()
        res = {}
        for m in ms:
            pats = synth.sample_patterns(t, m, args.patterns, seed=0, stream=synth.stream_id("orders", kind, m))
            orders = {"freq": [sm.sm_order(p, hist) for p in pats],
                      "h": [sm.sm_order_fixed(p, sm.SM_ORDER_H) for p in pats],
                      "hs": [sm.sm_order_fixed(p, sm.SM_ORDER_HS) for p in pats]}
            cell, ref = {}, None
            for name, pis in orders.items():
                for peel in peels:
                    def one():
                        for j, p in enumerate(pats):
                            sm.sm_count(ctx, d, p, pi=pis[j], hist=hist, peel=peel, out=counts[j:j + 1])
                    one()
                    got = counts.cpu().numpy().copy()
                    if ref is None:
                        ref = got
                    elif not np.array_equal(ref, got):
                        out["counts_agree"] = False
                    ts = []
                    for _ in range(reps):
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        one()
                        e1.record(stream)
                        torch.cuda.synchronize()
                        ts.append(e0.elapsed_time(e1) / 1e3)
                    cell[f"{name}/r{peel}"] = round(len(pats) * args.n / statistics.median(ts) / 1e9, 1)
            res[str(m)] = cell
        out["gbs"][str(kind)] = res
        del d
    return out


# ---------------------------------------------------------------- serving

def run_serve(args, local):
    """Serving loop on a 4 GiB resident text (2 GiB uniform ACGT + 2 GiB
    Markov-95). Poisson arrivals at each rate for --serve-seconds; m
    log-uniform in [2, 2048]; 80% counts, 20% reports; 80% of patterns copied
    from the text. p50/p99 latency and queries/s of the continuous-batching
    server and of one query at a time on the same arrival trace."""
    import torch
    from paper_1612_01506_gb300 import synth
    from paper_1612_01506_gb300.serve import Query, Server, latency_stats, one_at_a_time
    half = 2 << 30
    t = np.empty(2 * half, dtype=np.uint8)
    synth.uniform(half, 4, seed=0, stream=synth.stream_id("serve", 4), out=t[:half])
    synth.markov95(half, seed=0, stream=synth.stream_id("serve", "markov95"), out=t[half:])
    text = torch.from_numpy(t).to(torch.device("cuda", local))
    out = {"workload": "serving: 4 GiB resident text (2 GiB ACGT + 2 GiB Markov-95), Poisson arrivals, "
                       "m log-uniform [2,2048], 80/20 count/report", "chunk_bytes": args.serve_chunk_mib << 20,
           "report_batch_min": args.serve_report_batch_min, "burst_below": args.serve_burst_below, "rates": {}}
    server = Server(text, chunk_bytes=args.serve_chunk_mib << 20, max_m=2048, max_active=4096,
                    report_budget=24 << 30, report_batch_min=args.serve_report_batch_min,
                    burst_below=args.serve_burst_below)
    server.warm_up([t[1000:1000 + m].tobytes() for m in (3, 40, 700, 2048)])
    one_at_a_time(text, [Query(pattern=t[5:12].tobytes(), kind="report"), Query(pattern=t[9:30].tobytes())],
                  hist=server.hist)
    for rate in [float(x) for x in args.serve_rates.split(",") if x]:
        r = np.random.default_rng(int(rate))
        k = max(1, int(rate * args.serve_seconds))
        arr = np.cumsum(r.exponential(1.0 / rate, k))
        def trace():
            qs = []
            rr = np.random.default_rng(int(rate) + 1)
            for i in range(k):
                m = int(np.exp(rr.uniform(np.log(2), np.log(2048))))
                if rr.random() < 0.8:
                    s = int(rr.integers(0, t.size - m + 1))
                    p = t[s:s + m].tobytes()
                else:
                    p = bytes(rr.choice(np.frombuffer(b"ACGT etaoin", np.uint8), m))
                qs.append(Query(pattern=p, kind="report" if rr.random() < 0.2 else "count", arrival=float(arr[i])))
            return qs
        qs = trace()
        server.done = []
        t0 = time.perf_counter()
        server.run(qs)
        wall = time.perf_counter() - t0
        srv = latency_stats(qs)
        base = latency_stats(one_at_a_time(text, trace(), hist=server.hist))
        out["rates"][str(int(rate))] = {"server": srv, "one_at_a_time": base, "server_wall_s": round(wall, 2)}
    return out


# ---------------------------------------------------------------- CPU oracle

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def run_cpu_baseline(args, budget_s: float):
    """The oracle on a bounded sample of the sweep, on the host cores.

    Threaded leg (three quarters of the budget): Algorithm 1 split over all
    cores, on 64 MiB prefixes of the sweep texts, cycling over (sigma, m,
    variant) in the sweep's mix (count and report of every pattern) with
    fresh patterns until the budget is spent. Single-thread leg (the rest):
    plain Algorithm 1 on one core, counts on 8 MiB prefixes, same cycle."""
    import oracle
    from paper_1612_01506_gb300 import synth
    kinds, ms = kinds_of(args.kinds), [int(x) for x in args.ms.split(",") if x]
    variants = [v for v in args.variants.split(",") if v]
    cores = os.cpu_count() or 1
    sample_n = min(args.n, 64 << 20)
    single_n = min(args.n, 8 << 20)
    texts = {k: synth.text(k, sample_n, seed=0, stream=synth.stream_id("sweep", k)) for k in kinds}
    order = [(k, m) for m in ms for k in kinds]

    def leg(budget, n, threaded):
        scanned, spent, searches = {v: 0 for v in variants}, {v: 0.0 for v in variants}, 0
        rep = 0
        while sum(spent.values()) < budget and rep < 100:
            for k, m in order:
                if sum(spent.values()) >= budget:
                    break
                t = texts[k][:n]
                p = synth.sample_patterns(t, m, rep + 1, seed=0, stream=synth.stream_id("pat", k, m))[rep]
                for v in (variants if threaded else ["count"]):
                    t0 = time.perf_counter()
                    if not threaded:
                        oracle.naive_count(p, t)
                    elif v == "count":
                        oracle.count_threads(p, t, cores)
                    else:
                        oracle.report_threads(p, t, n - m + 1, cores)
                    spent[v] += time.perf_counter() - t0
                    scanned[v] += n
                    searches += 1
            rep += 1
        tot = sum(spent.values())
        per = {f"{v}_gbs": round(scanned[v] / spent[v] / 1e9, 3) for v in spent if spent[v] > 0}
        return round(sum(scanned.values()) / tot / 1e9, 3), searches, tot, per

    v_thr, n_thr, s_thr, per = leg(0.75 * budget_s, sample_n, True)
    v_one, n_one, s_one, _ = leg(0.25 * budget_s, single_n, False)
    out = {"value": v_thr, "unit": "GB/s", "cores": cores, "kind": "oracle",
           "sample": f"{n_thr} searches ({'+'.join(variants)} of each pattern) over {sample_n >> 20} MiB prefixes "
                     f"of the sweep texts (sigma {args.kinds}; m {args.ms}), {s_thr:.1f} s, threaded over {cores} cores",
           "cpu_model": cpu_model(),
           "single_thread": {"value": v_one, "unit": "GB/s", "cores": 1,
                             "sample": f"{n_one} counts (plain Algorithm 1) over {single_n >> 20} MiB prefixes, "
                                       f"{s_one:.1f} s"}}
    out.update(per)
    return out


# ---------------------------------------------------------------- main

def config_block(args, world):
    return {"workload": f"sweep n={args.n} bytes: sigma {args.kinds} x m {args.ms} x {args.patterns} "
                        f"patterns from the text, {args.variants}",
            "n": args.n, "kinds": args.kinds, "ms": args.ms, "patterns": args.patterns,
            "variants": args.variants,
            "l2": (f"inputs larger than L2 ({args.n >> 20} MiB texts against 129 MB), no flush"
                   if args.n > 129_000_000 else f"{args.n >> 20} MiB texts fit in L2: no flush, timings are warm"),
            "parallelism": f"weak: {world} rank(s), independent patterns per rank"}


def main():
    args = parse()
    world, rank, local = dist_setup(args)

    if args.impl == "reference":
        if rank != 0:
            return
        budget = max(5.0, min(60.0, args.cpu_seconds))
        vals = []
        for _ in range(max(args.warmup, 0)):
            run_cpu_baseline(args, 1.0)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            vals.append(run_cpu_baseline(args, budget / max(args.steps, 1)))
        el = time.perf_counter() - t0
        v = statistics.median([x["value"] for x in vals])
        line = {"metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": 0, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(el / max(args.steps, 1) * 1e3, 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
                "data": "synthetic", "config": config_block(args, 1), "impl": "reference",
                "cpu_baseline": vals[-1], "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0,
                                                  "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    if args.batch_only:
        if rank == 0:
            print(json.dumps({"batch": run_batch(args, local)}), flush=True)
        return
    if args.serve_only:
        if rank == 0:
            print(json.dumps({"serving": run_serve(args, local)}), flush=True)
        return
    if args.multi_only:
        if rank == 0:
            print(json.dumps({"multi": run_multi(args, local)}), flush=True)
        return
    if args.compare_stats:
        if rank == 0:
            print(json.dumps({"compare_stats": run_compare_stats(args, local)}), flush=True)
        return
    if args.tune_only:
        if rank == 0:
            print(json.dumps({"tune": run_tune(args, local)}), flush=True)
        return
    if args.orders_only:
        if rank == 0:
            print(json.dumps({"orders": run_orders(args, local)}), flush=True)
        return
    if args.latency_only:
        if rank == 0:
            print(json.dumps({"latency": run_latency(args, local)}), flush=True)
        return
    res = run_gpu(args, world, rank, local)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = run_cpu_baseline(args, args.cpu_seconds)
    if rank == 0:
        line = {"metric": METRIC, "value": round(res["value"], 1), "unit": "GB/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(res["elapsed"] / args.steps * 1e3, 2), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
                "config": config_block(args, world), "roofline": res["roofline"],
                "report_roofline": res["report_roofline"], "gate": res["gate"], "cpu_baseline": cpu,
                "e2e": res["e2e"], "gpu_launches": res["launches"], "clocks": res["clocks"],
                "sweep": res["detail"]}
        if not args.no_batch and world == 1:
            line["batch"] = run_batch(args, local)
        if not args.no_serve and world == 1:
            line["serving"] = run_serve(args, local)
        if not args.no_multi and world == 1:
            line["multi"] = run_multi(args, local)
        if not args.no_latency and world == 1:
            line["latency"] = run_latency(args, local)
        print(json.dumps(line), flush=True)
        if args.json_detail:
            with open(args.json_detail, "w") as f:
                json.dump({"line": line, "detail_gbs": res["detail"]}, f, indent=1)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
