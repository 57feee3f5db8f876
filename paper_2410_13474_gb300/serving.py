"""Serving loop: continuous batching of view requests over resident holograms.

Holograms stay resident as plans (their oversampled spectra and FP64 tables
cached on the device).  Requests (hologram id, view) arrive over time; the
scheduler admits them into batches as GPU slots (streams) and HBM budget free
up, so requests that arrive while others run are batched and their work
overlaps on the device.  Each batch is one nufds_reconstruct_batch call on
its slot's stream; per-request latency runs from arrival to the completion
event of its batch.

The scheduling logic is device-independent: an executor runs batches.
``GpuExecutor`` drives the library on CUDA streams; tests use a simulated
executor to check admission, ordering and accounting on the CPU.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field


@dataclass
class Request:
    rid: int
    holo: int
    view: object                   # paper_2410_13474_gb300.View
    t_arrival: float               # seconds from the start of the run
    ws_bytes: int = 0              # device workspace the view needs
    t_admit: float | None = None
    t_done: float | None = None
    status: int | None = None
    out: object = None


@dataclass
class Stats:
    n: int
    completed: int                 # finished with status 0
    failed: int                    # finished with an error status (not in throughput or latency)
    rejected: int
    wall_s: float
    throughput: float              # completed views per second of wall time
    p50_ms: float
    p99_ms: float
    mean_batch: float
    batches: int
    max_inflight_bytes: int

    def as_dict(self):
        return {k: (round(v, 4) if isinstance(v, float) else v) for k, v in self.__dict__.items()}


def percentile(xs, q):
    if not xs:
        return float("nan")
    s = sorted(xs)
    k = (len(s) - 1) * q
    f, c = math.floor(k), math.ceil(k)
    return s[f] + (s[c] - s[f]) * (k - f)


class Scheduler:
    """Continuous batching under an HBM budget.

    budget_bytes: device memory available for the batches' working memory
    (the resident plans are accounted for by the caller).  The library keeps
    each stream's batch workspace at its high-water mark, so a slot holds
    max(its largest batch so far, its current batch); a batch is admitted only
    if the sum over slots stays within the budget.  A request whose workspace
    alone exceeds the budget is rejected (status ENOMEM).
    slots: concurrent batches (one stream each); max_batch: views per batch.
    batch_queue: adaptive batching.  A batch takes every queued request (up to
    max_batch) only while at least batch_queue requests wait; with fewer it
    takes the oldest one alone.  A batch's requests all complete when the
    batch does, so batching a short queue delays its first requests without
    a throughput gain; a long queue (a backlog) is where batching pays.
    overlap_bytes: latency guard for concurrent batches, with workspace bytes
    as the measure of a batch's work.  While a batch above overlap_bytes runs,
    another slot starts only a batch of at most overlap_bytes (small views
    pass a large one instead of queueing behind it, but two large ones never
    share the GPU, which would stretch both); None lets any batches overlap.
    """

    def __init__(self, executor, budget_bytes: int, slots: int = 2, max_batch: int = 16,
                 clock=time.perf_counter, idle_sleep: float = 2e-4,
                 overlap_bytes: int | None = None, batch_queue: int = 1):
        self.ex = executor
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.max_batch = int(max_batch)
        self.clock = clock
        self.idle_sleep = idle_sleep
        self.overlap_bytes = None if overlap_bytes is None else int(overlap_bytes)
        self.batch_queue = max(1, int(batch_queue))

    def run(self, requests) -> Stats:
        reqs = sorted(requests, key=lambda r: r.t_arrival)
        pending = collections.deque()
        inflight = {}                      # slot -> (batch, handle, bytes)
        reserved = [0] * self.slots        # retained workspace per slot (high-water mark)
        inflight_bytes = max_inflight = 0
        nxt = done = rejected = failed = 0
        n = len(reqs)
        batch_sizes = []
        t0 = self.clock()
        while done + rejected < n:
            now = self.clock() - t0
            while nxt < n and reqs[nxt].t_arrival <= now:
                r = reqs[nxt]
                nxt += 1
                if r.ws_bytes > self.budget:
                    r.status = -2
                    rejected += 1
                else:
                    pending.append(r)
            progressed = False
            for s in list(inflight):
                batch, handle, nbytes = inflight[s]
                if self.ex.done(handle):
                    t = self.clock() - t0
                    statuses = self.ex.statuses(handle)
                    for r, st in zip(batch, statuses):
                        r.t_done = t
                        r.status = st
                        failed += st != 0
                    done += len(batch)
                    inflight_bytes -= nbytes
                    del inflight[s]
                    progressed = True
            for s in range(self.slots):
                if s in inflight or not pending:
                    continue
                room = self.budget - sum(reserved[k] for k in range(self.slots) if k != s)
                if (self.overlap_bytes is not None and inflight
                        and max(b[2] for b in inflight.values()) > self.overlap_bytes):
                    room = min(room, self.overlap_bytes)
                batch, nbytes = [], 0
                limit = self.max_batch if len(pending) >= self.batch_queue else 1
                while pending and len(batch) < limit:
                    r = pending[0]
                    if nbytes + r.ws_bytes > room:
                        break
                    batch.append(pending.popleft())
                    nbytes += r.ws_bytes
                if not batch:
                    continue
                t = self.clock() - t0
                for r in batch:
                    r.t_admit = t
                inflight[s] = (batch, self.ex.launch(s, batch), nbytes)
                reserved[s] = max(reserved[s], nbytes)
                inflight_bytes += nbytes
                max_inflight = max(max_inflight, sum(reserved))
                batch_sizes.append(len(batch))
                progressed = True
            if not progressed:
                # nothing to do until an arrival or a completion: with every
                # slot busy the executor may block on a running batch (one
                # slot: no arrival can start before it ends); with none busy,
                # sleep to the next arrival
                handles = [b[1] for b in inflight.values()]
                self.ex.idle(t0 + reqs[nxt].t_arrival if nxt < n else None, self.idle_sleep,
                             wait=handles[0] if self.slots == 1 and handles else None,
                             busy=bool(handles))
        wall = self.clock() - t0
        lat = [1e3 * (r.t_done - r.t_arrival) for r in reqs
               if r.t_done is not None and r.status == 0]
        ok = done - failed
        return Stats(n=n, completed=ok, failed=failed, rejected=rejected, wall_s=wall,
                     throughput=ok / wall if wall > 0 else float("nan"),
                     p50_ms=percentile(lat, 0.50), p99_ms=percentile(lat, 0.99),
                     mean_batch=(sum(batch_sizes) / len(batch_sizes)) if batch_sizes else 0.0,
                     batches=len(batch_sizes), max_inflight_bytes=max_inflight)


class GpuExecutor:
    """Runs batches with nufds_reconstruct_batch, one CUDA stream per slot;
    a batch of one view runs as nufds_reconstruct (the same arithmetic without
    the batch's descriptor upload and graph launch).

    plans: list of Plan (resident holograms).  single=True runs each view with
    nufds_reconstruct (the one-at-a-time reference, slots=1, max_batch=1).
    keep_outputs stores each request's output tensor on it.
    """

    def __init__(self, plans, slots: int, single: bool = False, keep_outputs: bool = False):
        import torch
        import paper_2410_13474_gb300 as nf
        self.torch, self.nf = torch, nf
        self.plans = plans
        self.single = single
        self.keep = keep_outputs
        self.streams = [torch.cuda.Stream() for _ in range(slots)]

    def workspace_bytes(self, holo, view) -> int:
        return int(self.plans[holo].view_plan(view)["workspace_bytes"])

    def launch(self, slot, batch):
        torch, nf = self.torch, self.nf
        st = self.streams[slot]
        outs = []
        with torch.cuda.stream(st):
            for r in batch:
                outs.append(self.plans[r.holo].output_like(r.view))
            if self.single or len(batch) == 1:
                statuses = []
                for r, o in zip(batch, outs):
                    try:
                        self.plans[r.holo].reconstruct(r.view, o, stream=st)
                        statuses.append(0)
                    except nf.NufdsError as e:
                        statuses.append(e.code)
            else:
                statuses = nf.reconstruct_batch([self.plans[r.holo] for r in batch],
                                                [r.view for r in batch], outs, stream=st)
            ev = torch.cuda.Event()
            ev.record(st)
        if self.keep:
            for r, o in zip(batch, outs):
                r.out = o
        return (ev, statuses, outs)

    def done(self, handle) -> bool:
        return handle[0].query()

    def statuses(self, handle):
        return handle[1]

    def idle(self, next_arrival, sleep, wait=None, busy=True):
        """Pass the time until something can happen: block on `wait` (a
        running batch) when given; with nothing running, sleep until the next
        arrival (the last 0.2 ms by polling the clock, since a sleep can
        overrun by tens of microseconds); otherwise sleep `sleep` seconds."""
        if wait is not None:
            wait[0].synchronize()
            return
        if not busy and next_arrival is not None:
            while True:
                left = next_arrival - time.perf_counter()
                if left <= 0:
                    return
                if left > 2e-4:
                    time.sleep(left - 2e-4)
        else:
            time.sleep(sleep)


class SimExecutor:
    """Simulated device for scheduler tests: a batch on a slot takes
    fixed + per_byte * (its workspace bytes) seconds; time only moves when the
    scheduler is idle (to the next completion or arrival)."""

    def __init__(self, fixed: float = 1e-3, per_byte: float = 1e-12):
        self.t = 0.0
        self.fixed, self.per_byte = fixed, per_byte
        self.ends = []
        self.launched = []

    def clock(self):
        return self.t

    def launch(self, slot, batch):
        end = self.t + self.fixed + self.per_byte * sum(r.ws_bytes for r in batch)
        self.ends.append(end)
        self.launched.append((slot, [r.rid for r in batch], self.t))
        return (end, [0] * len(batch))

    def done(self, handle):
        return self.t >= handle[0]

    def statuses(self, handle):
        return handle[1]

    def idle(self, next_arrival, sleep, wait=None, busy=True):
        cands = [e for e in self.ends if e > self.t]
        if next_arrival is not None and next_arrival > self.t:
            cands.append(next_arrival)
        self.t = min(cands) if cands else self.t + sleep


def poisson_arrivals(n: int, rate: float, seed: int):
    """n arrival times (seconds) of a Poisson process of the given rate."""
    import numpy as np
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
