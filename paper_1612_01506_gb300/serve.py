"""Serving loop: count and report queries against one device-resident text.

Continuous batching: the text stays in HBM, cut into chunks. Every step scans
the next chunk for all active queries in one batched launch
(``sm_stepper_step``), so queries in flight share each pass over the text.
A query is admitted whenever a counter slot is free -- it joins at whatever
chunk comes next -- and its count is complete after one step on every chunk.
A report query then needs a position buffer of exactly count x 8 bytes and is
admitted when both the report budget and the device's free memory (what the
driver reports free plus what torch's allocator holds unused, minus a reserve)
have room; one that can never fit is answered with an error instead. Its
positions are written on
a second stream while the next steps run: by ``sm_report`` alone, or, when at
least ``report_batch_min`` report queries wait, together with them in one
batched report over the text (``sm_stepper_report``).

A query that arrives while the server is idle runs at once as one
single-pattern search over the whole text (``sm_count``), as it would alone;
so do arrivals while no batched query and at most ``burst_below`` single
searches are in flight, one launch each (a batched pass pays off once
several patterns share it).

Every query's result is the same as when it runs alone (the tests check
this against single calls and the CPU oracle).
"""
from __future__ import annotations

import collections
import ctypes as C
import time
from dataclasses import dataclass, field

import numpy as np

from . import sm


@dataclass
class Query:
    pattern: bytes
    kind: str = "count"            # "count" or "report"
    arrival: float = 0.0           # seconds on the server's clock
    count: int | None = None
    positions: object = None       # device tensor (int64) for reports
    done: float | None = None
    qid: int = -1
    error: str | None = None       # a report that could not be admitted
    alone: bool = False            # counted by a single search at an idle server

    @property
    def latency(self) -> float:
        return (self.done or 0.0) - self.arrival


def _bind_stepper():
    lib = sm.load()
    if getattr(lib, "_stepper_bound", False):
        return lib
    vp, u8p, u32p = C.c_void_p, C.POINTER(C.c_uint8), C.POINTER(C.c_uint32)
    st = C.c_int
    lib.sm_stepper_create.argtypes = [vp, vp, C.c_uint64, C.c_uint64, C.c_uint32, C.POINTER(C.c_uint64),
                                      C.POINTER(vp)]
    lib.sm_stepper_create.restype = st
    lib.sm_stepper_chunks.argtypes = [vp]
    lib.sm_stepper_chunks.restype = C.c_uint32
    lib.sm_stepper_admit.argtypes = [vp, C.c_uint32, u8p, C.c_uint32]
    lib.sm_stepper_admit.restype = st
    lib.sm_stepper_step.argtypes = [vp, u32p, C.c_uint32, C.c_uint32, vp, vp]
    lib.sm_stepper_step.restype = st
    lib.sm_stepper_steps.argtypes = [vp, u32p, u32p, C.c_uint32, C.c_uint32, vp, vp]
    lib.sm_stepper_steps.restype = st
    lib.sm_stepper_retire.argtypes = [vp, C.c_uint32]
    lib.sm_stepper_retire.restype = st
    i64p = C.POINTER(C.c_int64)
    lib.sm_stepper_report.argtypes = [vp, u8p, i64p, C.c_uint32, i64p, vp, vp, vp]
    lib.sm_stepper_report.restype = st
    lib.sm_stepper_destroy.argtypes = [vp]
    lib.sm_stepper_destroy.restype = None
    lib._stepper_bound = True
    return lib


class Server:
    """Continuous-batching server over the resident uint8 CUDA tensor `text`."""

    def __init__(self, text, chunk_bytes: int = 256 << 20, max_m: int = 2048, max_active: int = 1024,
                 report_budget: int = 8 << 30, burst_below: int = 4, report_batch_min: int = 32,
                 memory_reserve: int = 1 << 30):
        import torch
        self.torch = torch
        self.text = text
        self.dev = text.device
        self.lib = _bind_stepper()
        self.ctx = sm.sm_create(self.dev.index or 0)           # steps, on self.stream (and batched reports)
        self.rctx = sm.sm_create(self.dev.index or 0)          # single reports, on self.rstream
        self.stream = torch.cuda.Stream(device=self.dev)
        self.rstream = torch.cuda.Stream(device=self.dev)
        self.hist = sm.sm_histogram(self.ctx, text, stream=self.stream)
        self.stream.synchronize()
        self.hist = self.hist.cpu().numpy().view(np.uint64).copy()
        self.max_m = max_m
        chunk = max(sm.SM_TILE_STARTS, (chunk_bytes // sm.SM_TILE_STARTS) * sm.SM_TILE_STARTS)
        h = C.c_void_p()
        sm._check(self.lib.sm_stepper_create(self.ctx.handle, text.data_ptr(), text.numel(), chunk, max_m,
                                              self.hist.ctypes.data_as(C.POINTER(C.c_uint64)), C.byref(h)))
        self.stepper = h.value
        self.nchunks = int(self.lib.sm_stepper_chunks(self.stepper))
        self.max_active = max_active
        # with at most this many queries in flight and none waiting, a step
        # scans every chunk back to back; otherwise one chunk per step, so that
        # arrivals join at the next chunk
        self.burst_below = burst_below
        self.counters = torch.zeros(max_active, dtype=torch.int64, device=self.dev)
        self.host_counters = torch.zeros(max_active, dtype=torch.int64).pin_memory()
        self.free_slots = list(range(max_active - 1, -1, -1))
        self.pending: collections.deque[Query] = collections.deque()
        self.active: dict[int, list] = {}         # slot -> [query, chunks left]
        self.finishing: list = []                 # (event, [queries]) whose counts are final
        self.report_wait: collections.deque[Query] = collections.deque()
        self.reporting: list = []                 # (event, query, bytes)
        self.report_budget = report_budget
        # device memory kept free of report buffers (workspace growth, other users)
        self.memory_reserve = memory_reserve
        # with at least this many report queries waiting they are reported in
        # one batched pass; fewer run one report each (a batched pass holds
        # every SM for its whole length, which delays the count steps)
        self.report_batch_min = report_batch_min
        self.report_reserved = 0
        self.next_chunk = 0
        self.done: list[Query] = []
        self.steps = 0
        self.t0 = time.perf_counter()

    def __del__(self):
        h, self.stepper = getattr(self, "stepper", None), None
        if h:
            self.lib.sm_stepper_destroy(h)

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, q: Query):
        if len(q.pattern) < 1 or len(q.pattern) > self.max_m:
            raise ValueError("pattern length out of range")
        self.pending.append(q)

    @property
    def busy(self) -> bool:
        return bool(self.pending or self.active or self.finishing or self.report_wait or self.reporting)

    # ------------------------------------------------------------ one step
    def step(self):
        torch = self.torch
        if (len(self.pending) == 1 and not self.active and not self.finishing and self.free_slots
                and not self.reporting and not self.report_wait):
            self._run_alone(self.pending.popleft())
            self._poll()
            return
        singles = sum(1 for _, qs, _ in self.finishing for q in qs if q.alone)
        if (not self.active and 0 < len(self.pending) and singles + len(self.pending) <= self.burst_below
                and len(self.free_slots) >= len(self.pending)):
            # a few arrivals, no batched query in flight and at most
            # burst_below single searches: one search each, back to back (one
            # launch per pattern beats a batched pass over the text until
            # several patterns share it; beyond that the arrivals are batched)
            single = []
            while self.pending:
                single.append(self._run_single(self.pending.popleft()))
            self._finish(single)
            self._poll()
            return
        # admission: a free counter slot per query
        while self.pending and self.free_slots:
            q = self.pending.popleft()
            slot = self.free_slots.pop()
            q.qid = slot
            p = np.frombuffer(q.pattern, np.uint8)
            sm._check(self.lib.sm_stepper_admit(self.stepper, slot, p.ctypes.data_as(C.POINTER(C.c_uint8)),
                                                p.size))
            with torch.cuda.stream(self.stream):
                self.counters[slot].zero_()
            self.active[slot] = [q, self.nchunks]
        if self.active and len(self.active) <= self.burst_below and not self.pending:
            self._step_chunk(burst=True)   # every active query to its end, one launch
        elif self.active:
            self._step_chunk()
        self._poll()

    def _step_chunk(self, burst: bool = False):
        """One step on the next chunk for every active query; with burst, each
        active query over all the chunks it still needs, in one launch."""
        torch = self.torch
        slots = np.fromiter(self.active.keys(), dtype=np.uint32, count=len(self.active))
        if burst:
            left = np.array([self.active[int(q)][1] for q in slots], dtype=np.uint32)
            sm._check(self.lib.sm_stepper_steps(self.stepper, slots.ctypes.data_as(C.POINTER(C.c_uint32)),
                                                left.ctypes.data_as(C.POINTER(C.c_uint32)), slots.size,
                                                self.next_chunk, self.counters.data_ptr(), self.stream.cuda_stream))
            done_chunks = int(left.max())
        else:
            sm._check(self.lib.sm_stepper_step(self.stepper, slots.ctypes.data_as(C.POINTER(C.c_uint32)),
                                               slots.size, self.next_chunk, self.counters.data_ptr(),
                                               self.stream.cuda_stream))
            done_chunks = 1
        finished = []
        for slot in list(self.active):
            ent = self.active[slot]
            ent[1] -= min(ent[1], done_chunks)
            if ent[1] == 0:
                finished.append(ent[0])
                del self.active[slot]
        if finished:
            self._finish(finished)
        self.next_chunk = (self.next_chunk + done_chunks) % self.nchunks
        self.steps += 1

    def _finish(self, finished: list):
        """Read the final counts of `finished` back to the host: one copy of
        the whole counter array into the pinned mirror allocated at start-up
        (on the step stream, after the work enqueued so far). Nothing is
        allocated here: a pinned allocation in the loop took seconds on first
        use. A later copy rewrites the mirror, but a finished query's counter
        does not change until its slot is freed, after it has been read."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            self.host_counters.copy_(self.counters, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(self.stream)
        self.finishing.append((ev, finished, None))

    def _run_single(self, q: Query) -> Query:
        """Enqueue one single-pattern count of q over the whole text into a
        counter slot (read back by _finish; a report query then goes through
        the report queue)."""
        slot = self.free_slots.pop()
        q.qid = slot
        sm.sm_count(self.ctx, self.text, q.pattern, pi=sm.sm_order(q.pattern, self.hist), hist=self.hist,
                    out=self.counters[slot:slot + 1], stream=self.stream)
        q.alone = True
        self.steps += 1
        return q

    def _run_alone(self, q: Query):
        """An arrival at an idle server: one single-pattern count over the
        whole text, planned under the text's own frequencies, as the query
        would run alone. A report query then waits for its count and, when
        its position buffer is admitted, has its report enqueued right after
        it on the same stream (the loop holds no other work); otherwise it
        goes through the report queue."""
        slot = self.free_slots.pop()
        q.qid = slot
        pi = sm.sm_order(q.pattern, self.hist)
        sm.sm_count(self.ctx, self.text, q.pattern, pi=pi, hist=self.hist, out=self.counters[slot:slot + 1],
                    stream=self.stream)
        q.alone = True
        self.steps += 1
        if q.kind != "report":
            self._finish([q])
            return
        torch = self.torch
        with torch.cuda.stream(self.stream):
            self.host_counters[slot].copy_(self.counters[slot], non_blocking=True)
        self.stream.synchronize()
        q.count = int(self.host_counters[slot])
        self.free_slots.append(slot)
        need = max(q.count, 1) * 8
        if self.report_wait or (need > self._room() and need > self._room(full=True)):
            self.report_wait.append(q)
            return
        self.report_reserved += need
        with torch.cuda.stream(self.stream):
            pos = torch.empty(max(q.count, 1), dtype=torch.int64, device=self.dev)
            cnt = torch.empty(1, dtype=torch.int64, device=self.dev)
        sm.sm_report(self.ctx, self.text, q.pattern, q.count, pi=pi, out_pos=pos, out_count=cnt, stream=self.stream,
                     hist=self.hist)
        ev = torch.cuda.Event()
        ev.record(self.stream)
        q.positions = pos[: q.count]
        self.reporting.append((ev, [q], need, False))

    def warm_up(self, patterns: list[bytes]):
        """Run a few queries through every path once (loads kernels, sizes buffers)."""
        qs = [Query(pattern=p, kind=("report" if i % 2 else "count")) for i, p in enumerate(patterns)]
        for q in qs:
            self.submit(q)
        while self.busy:
            self.step()
        self.torch.cuda.synchronize()
        self.done = []

    def _poll(self):
        torch = self.torch
        keep = []
        for ev, qs, host in self.finishing:
            if not ev.query():
                keep.append((ev, qs, host))
                continue
            now = self.now()
            hc = self.host_counters.numpy()
            for q in qs:
                c = hc[q.qid]
                q.count = int(c)
                if not getattr(q, "alone", False):
                    self.lib.sm_stepper_retire(self.stepper, q.qid)
                self.free_slots.append(q.qid)
                if q.kind == "report":
                    self.report_wait.append(q)
                else:
                    q.done = now
                    self.done.append(q)
        self.finishing = keep
        # finished reports (single or batched): their queries are done
        keep = []
        for ev, qs, need, bt in self.reporting:
            if ev.query():
                now = self.now()
                for q in qs:
                    q.done = now
                    self.done.append(q)
                self.report_reserved -= need
            else:
                keep.append((ev, qs, need, bt))
        self.reporting = keep
        if len(self.report_wait) >= self.report_batch_min and not any(bt for _, _, _, bt in self.reporting):
            self._report_batch()
        # single reports: admitted by the memory their position buffers need
        while self.report_wait and len(self.report_wait) < self.report_batch_min:
            q = self.report_wait[0]
            need = max(q.count, 1) * 8
            if not self._admit(q, need, self._room()):
                break
            if q.error:
                continue
            self.report_wait.popleft()
            self.report_reserved += need
            with torch.cuda.stream(self.rstream):
                pos = torch.empty(max(q.count, 1), dtype=torch.int64, device=self.dev)
                cnt = torch.empty(1, dtype=torch.int64, device=self.dev)
            sm.sm_report(self.rctx, self.text, q.pattern, q.count, pi=sm.sm_order(q.pattern, self.hist),
                         out_pos=pos, out_count=cnt, stream=self.rstream, hist=self.hist)
            ev = torch.cuda.Event()
            ev.record(self.rstream)
            q.positions = pos[: q.count]
            self.reporting.append((ev, [q], need, False))

    def _room(self, full: bool = False) -> int:
        """Bytes a new report buffer may take now: what is left of the report
        budget, and the device memory free for it minus the reserve. The
        quick figure counts only what the driver reports free (~10 us); the
        full one adds what torch's caching allocator holds unused, whose
        statistics cost ~0.1 ms a read -- a large part of a lone report's
        latency -- so it is read only when the quick figure is too small
        (the quick figure never exceeds the full one)."""
        torch = self.torch
        free, _ = torch.cuda.mem_get_info(self.dev)
        if full:
            free += torch.cuda.memory_reserved(self.dev) - torch.cuda.memory_allocated(self.dev)
        return min(self.report_budget - self.report_reserved, free - self.memory_reserve)

    def _admit(self, q: Query, need: int, room: int) -> bool:
        """Whether the report at the head of the wait queue may go on: True
        when it fits `room` (or the room read afresh); a report that never
        can (above the budget, or above the free memory with no report in
        flight to give any back) is answered with an error and taken off the
        queue (also True); False when it has to wait for reports in flight."""
        if need <= room:
            return True
        room = self._room(full=True)
        if need <= room:
            return True
        if need > self.report_budget or not self.report_reserved:
            self.report_wait.popleft()
            q.error = (f"report needs {need} bytes of positions; budget {self.report_budget}, "
                       f"{max(room, 0)} bytes available")
            q.done = self.now()
            self.done.append(q)
            return True
        return False

    def _report_batch(self):
        """The waiting report queries whose position buffers (count x 8 bytes)
        fit the memory budget and the free device memory, reported together
        in one batched pass."""
        torch = self.torch
        batch, need = [], 0
        room = self._room()
        while self.report_wait:
            q = self.report_wait[0]
            b = max(q.count, 1) * 8
            if batch and need + b > room:
                break
            if not batch:
                if not self._admit(q, b, room):
                    break
                if q.error:
                    continue
            self.report_wait.popleft()
            batch.append(q)
            need += b
        if not batch:
            return
        pos_off = np.zeros(len(batch) + 1, np.int64)
        pos_off[1:] = np.cumsum([q.count for q in batch])
        pat_off = np.zeros(len(batch) + 1, np.int64)
        pat_off[1:] = np.cumsum([len(q.pattern) for q in batch])
        flat = np.frombuffer(b"".join(q.pattern for q in batch), np.uint8)
        with torch.cuda.stream(self.rstream):
            pos = torch.empty(max(int(pos_off[-1]), 1), dtype=torch.int64, device=self.dev)
            cnt = torch.empty(len(batch), dtype=torch.int64, device=self.dev)
        sm._check(self.lib.sm_stepper_report(
            self.stepper, flat.ctypes.data_as(C.POINTER(C.c_uint8)), pat_off.ctypes.data_as(C.POINTER(C.c_int64)),
            len(batch), pos_off.ctypes.data_as(C.POINTER(C.c_int64)), pos.data_ptr(), cnt.data_ptr(),
            self.rstream.cuda_stream))
        ev = torch.cuda.Event()
        ev.record(self.rstream)
        for k, q in enumerate(batch):
            q.positions = pos[pos_off[k]:pos_off[k + 1]]
        self.report_reserved += need
        self.reporting.append((ev, batch, need, True))

    # ------------------------------------------------------------ drivers
    def run(self, queries: list[Query], time_scale: float = 1.0, max_steps: int | None = None) -> list[Query]:
        """Submit queries at their arrival times (seconds x time_scale) and
        step until every one is done."""
        order = sorted(queries, key=lambda q: q.arrival)
        i = 0
        self.t0 = time.perf_counter()
        for q in order:
            q.arrival *= time_scale
        while i < len(order) or self.busy:
            now = self.now()
            while i < len(order) and order[i].arrival <= now:
                self.submit(order[i])
                i += 1
            if not self.busy and i < len(order):
                wait = order[i].arrival - now
                if wait > 0.0005:   # sleep most of the gap, spin the rest (sleep overshoots)
                    time.sleep(wait - 0.0003)
                continue
            if not self.pending and not self.active and not self.report_wait and (self.finishing or self.reporting):
                # only results in flight and nothing to step: poll their events
                # until one is done or the next arrival is due (blocking on the
                # oldest count would hold back a report that ends first)
                evs = [e[0] for e in self.finishing] + [e[0] for e in self.reporting]
                due = order[i].arrival if i < len(order) else float("inf")
                while not any(e.query() for e in evs) and self.now() < due:
                    pass
            self.step()
            if max_steps is not None and self.steps >= max_steps:
                break
        self.torch.cuda.synchronize()
        return order


def _wait_until(t0: float, t: float) -> None:
    """Return at time t0 + t (perf_counter seconds): sleep most of the gap,
    spin the rest (a sleep overshoots by tens of microseconds)."""
    while True:
        left = t0 + t - time.perf_counter()
        if left <= 0:
            return
        if left > 0.0005:
            time.sleep(left - 0.0003)


def one_at_a_time(text, queries: list[Query], hist=None) -> list[Query]:
    """Baseline: each query alone, in arrival order, waiting for the previous."""
    import torch
    ctx = sm.sm_create(text.device.index or 0)
    if hist is None:
        hist = sm.sm_histogram(ctx, text).cpu().numpy().view(np.uint64).copy()
    order = sorted(queries, key=lambda q: q.arrival)
    t0 = time.perf_counter()
    for q in order:
        _wait_until(t0, q.arrival)
        pi = sm.sm_order(q.pattern, hist)
        c = sm.sm_count(ctx, text, q.pattern, pi=pi, hist=hist)
        q.count = int(c.item())
        if q.kind == "report":
            pos, _ = sm.sm_report(ctx, text, q.pattern, max(q.count, 1), pi=pi, hist=hist)
            q.positions = pos[: q.count]
            torch.cuda.synchronize()
        q.done = time.perf_counter() - t0
    return order


def latency_stats(qs: list[Query]) -> dict:
    """p50 / p99 latency (ms) and throughput of answered queries, also per kind."""
    def pct(sel):
        lat = np.array([q.latency for q in sel]) * 1e3
        return {"queries": len(sel), "p50_ms": round(float(np.percentile(lat, 50)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3)}
    span = max(q.done for q in qs) - min(q.arrival for q in qs)
    out = {**pct(qs), "qps": round(len(qs) / span, 1)}
    for kind in ("count", "report"):
        sel = [q for q in qs if q.kind == kind]
        if sel:
            out[kind] = pct(sel)
    return out
