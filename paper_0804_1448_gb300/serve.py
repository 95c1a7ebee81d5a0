"""Serving loop: one resident reference set, query batches arriving over time,
continuous batching across slots, memory-based admission, p50/p99 latency.

The paper searches one query set against one reference set (Sec. 2.1); a
service answers many such searches against the same reference set.  Here the
reference set is uploaded once (knn_set_reference) and every slot is a handle
created with knn_create_shared on it: its own CUDA stream and workspace, the
reference data shared.  A request (a batch of n queries with its own k) is
admitted, first come first served, as soon as a slot is free and the
workspace it needs (knn_workspace_size) fits in the memory budget beside the
requests already running; requests that arrive while others are on the GPU
join them there.  Each slot's workspace is reserved up front (knn_reserve) for
the largest request it may take, so no allocation happens while serving.

Latency of a request = (time its results are complete on the GPU) - (its
arrival time), both on one clock: arrivals are host times from the start of
the run, completions are CUDA-event times from an event recorded at that
start.

The scheduler (admission, bookkeeping, statistics) is plain host code, driven
through an executor with three calls -- start(slot, request), poll(slot) and
completion time -- so it runs on the CPU with a simulated executor in tests.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float            # seconds from the start of the run
    n: int                    # queries in the batch
    k: int
    ws_bytes: int = 0         # workspace the search needs (filled by the server)
    queries: object = None    # device tensor n x d (GPU executor)
    start: float = math.nan   # admission time (host clock, seconds)
    done: float = math.nan    # completion time (device clock, seconds)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class Scheduler:
    """First-come-first-served admission into `slots` slots under a memory
    budget (bytes of workspace held by running requests)."""

    def __init__(self, slots: int, mem_budget: int):
        if slots < 1:
            raise ValueError("need at least one slot")
        self.slots = slots
        self.mem_budget = int(mem_budget)
        self.free = list(range(slots))[::-1]
        self.running = {}           # slot -> Request
        self.mem_in_use = 0
        self.peak_running = 0
        self.peak_mem = 0

    def can_admit(self, req: Request) -> bool:
        if not self.free:
            return False
        if req.ws_bytes > self.mem_budget:
            raise ValueError(f"request {req.rid} needs {req.ws_bytes} bytes, "
                             f"more than the whole budget {self.mem_budget}")
        return self.mem_in_use + req.ws_bytes <= self.mem_budget

    def admit(self, req: Request) -> int:
        slot = self.free.pop()
        self.running[slot] = req
        self.mem_in_use += req.ws_bytes
        self.peak_running = max(self.peak_running, len(self.running))
        self.peak_mem = max(self.peak_mem, self.mem_in_use)
        return slot

    def release(self, slot: int) -> Request:
        req = self.running.pop(slot)
        self.mem_in_use -= req.ws_bytes
        self.free.append(slot)
        return req


def run(requests, executor, slots: int, mem_budget: int, clock=time.perf_counter,
        idle=lambda: None):
    """Serve `requests` (sorted by arrival) through `executor`.  Returns the
    requests with start/done filled and the scheduler (for its peaks)."""
    reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
    sched = Scheduler(slots, mem_budget)
    pending = collections.deque()
    nxt = 0
    finished = 0
    t0 = clock()
    executor.begin()
    while finished < len(reqs):
        now = clock() - t0
        while nxt < len(reqs) and reqs[nxt].arrival <= now:
            pending.append(reqs[nxt])
            nxt += 1
        progressed = False
        while pending and sched.can_admit(pending[0]):
            req = pending.popleft()
            req.start = now
            executor.start(sched.admit(req), req)
            progressed = True
        for slot in list(sched.running):
            if executor.poll(slot):
                req = sched.release(slot)
                req.done = executor.completion(slot)
                finished += 1
                progressed = True
        if not progressed:
            idle()
    executor.end()
    return reqs, sched


def summary(reqs, makespan: float | None = None) -> dict:
    lat = np.array([r.latency for r in reqs], dtype=np.float64)
    queries = int(sum(r.n for r in reqs))
    if makespan is None:
        makespan = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {
        "requests": len(reqs),
        "queries": queries,
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_ms": float(lat.mean() * 1e3),
        "queries_per_s": queries / makespan if makespan > 0 else float("nan"),
        "makespan_s": makespan,
    }


def workload(count: int, seed: int, rate: float | None, n_max: int = 8192, k_max: int = 256,
             k_cap: int | None = None):
    """Requests with batch sizes log-uniform in [1, n_max], k uniform in
    [1, k_max], Poisson arrivals at `rate` batches/s (rate None: all at 0)."""
    g = np.random.Generator(np.random.Philox(int(seed)))
    n = np.exp(g.uniform(0.0, math.log(n_max), size=count)).astype(np.int64)
    n = np.clip(n, 1, n_max)
    k = g.integers(1, k_max + 1, size=count)
    if k_cap is not None:
        k = np.minimum(k, k_cap)
    if rate is None:
        t = np.zeros(count)
    else:
        t = np.cumsum(g.exponential(1.0 / rate, size=count))
    return [Request(rid=i, arrival=float(t[i]), n=int(n[i]), k=int(k[i])) for i in range(count)]


class GpuExecutor:
    """Slots = handles sharing one reference set, each with a torch stream."""

    def __init__(self, primary, slots: int, precision: str, reserve_bytes: int, device: int = 0):
        import torch
        from . import knn
        self.torch = torch
        self.device = device
        self.handles = [knn.Index.shared(primary) for _ in range(slots)]
        for h in self.handles:
            h.reserve(reserve_bytes)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.events = [None] * slots
        self.outputs = {}
        self.t0 = None

    def begin(self):
        torch = self.torch
        self.t0 = torch.cuda.Event(enable_timing=True)
        self.t0.record(torch.cuda.current_stream(self.device))

    def allocate(self, reqs):
        """Output buffers of every request, before the run (no allocation
        while serving)."""
        torch = self.torch
        self.outputs = {}
        for r in reqs:
            self.outputs[r.rid] = (
                torch.empty((r.n, r.k), dtype=torch.float32, device=f"cuda:{self.device}"),
                torch.empty((r.n, r.k), dtype=torch.int32, device=f"cuda:{self.device}"))
        torch.cuda.synchronize(self.device)

    def start(self, slot, req):
        torch = self.torch
        st = self.streams[slot]
        dist, idx = self.outputs[req.rid]
        # the queries and outputs were produced on the default stream before the run
        st.wait_event(self.t0)
        self.handles[slot].search_into(req.queries, req.k, dist, idx, "l2", st)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(st)
        self.events[slot] = ev

    def poll(self, slot) -> bool:
        return self.events[slot].query()

    def completion(self, slot) -> float:
        return self.t0.elapsed_time(self.events[slot]) / 1e3

    def end(self):
        self.torch.cuda.synchronize(self.device)

    def close(self):
        for h in self.handles:
            h.close()


class Server:
    """Resident reference set + slots; serves request lists."""

    def __init__(self, R, precision: str = "bf16", slots: int = 4, mem_budget: int | None = None,
                 n_max: int = 8192, k_max: int = 256, device: int = 0):
        from . import knn
        self.primary = knn.Index(device, precision)
        self.primary.set_reference(R)
        self.reserve = self.primary.workspace_size(n_max, k_max)
        self.slots = slots
        self.mem_budget = mem_budget if mem_budget is not None else slots * self.reserve
        self.executor = GpuExecutor(self.primary, slots, precision, self.reserve, device)

    def sized(self, reqs):
        for r in reqs:
            r.ws_bytes = self.primary.workspace_size(r.n, r.k)
        return reqs

    def serve(self, reqs):
        self.sized(reqs)
        self.executor.allocate(reqs)
        done, sched = run(reqs, self.executor, self.slots, self.mem_budget)
        return done, sched, self.executor.outputs

    def alone(self, req):
        """One request by itself on slot 0 (nothing else running)."""
        self.sized([req])
        req2 = dataclasses.replace(req, arrival=0.0)
        self.executor.allocate([req2])
        run([req2], self.executor, 1, max(self.mem_budget, req2.ws_bytes))
        return self.executor.outputs[req.rid]

    def close(self):
        self.executor.close()
        self.primary.close()
