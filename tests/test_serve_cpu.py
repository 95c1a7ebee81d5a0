"""Host logic of the serving loop (paper_0804_1448_gb300/serve.py) on a
simulated executor and clock: first-come-first-served admission, the slot
and memory limits, latency bookkeeping, request generation.  No GPU."""
import math

import numpy as np
import pytest

from paper_0804_1448_gb300 import serve


class SimClock:
    def __init__(self, dt=1e-4):
        self.t = 0.0
        self.dt = dt

    def now(self):
        return self.t

    def advance(self):
        self.t += self.dt


class SimExecutor:
    """Service time a + b*n per request, independent per slot."""

    def __init__(self, clock, a=2e-3, b=1e-6):
        self.clock, self.a, self.b = clock, a, b
        self.finish = {}
        self.log = []

    def begin(self):
        pass

    def start(self, slot, req):
        assert slot not in self.finish, "slot started twice"
        self.finish[slot] = self.clock.now() + self.a + self.b * req.n
        self.log.append(("start", req.rid, slot, self.clock.now()))

    def poll(self, slot):
        return self.clock.now() >= self.finish[slot]

    def completion(self, slot):
        return self.finish.pop(slot)

    def end(self):
        pass


def _run(reqs, slots, budget):
    clock = SimClock()
    ex = SimExecutor(clock)
    done, sched = serve.run(reqs, ex, slots, budget, clock=clock.now, idle=clock.advance)
    return done, sched, ex


def test_every_request_served_once_with_consistent_times():
    reqs = serve.workload(60, seed=3, rate=200.0, n_max=4096, k_max=64)
    for r in reqs:
        r.ws_bytes = 1000 + 10 * r.n
    done, sched, ex = _run(reqs, slots=3, budget=10 ** 9)
    assert sorted(r.rid for r in done) == list(range(60))
    for r in done:
        assert r.start >= r.arrival - 1e-12
        assert r.done >= r.start
        assert math.isclose(r.latency, r.done - r.arrival)
    assert sched.peak_running <= 3
    assert sched.mem_in_use == 0 and not sched.running


def test_admission_is_first_come_first_served():
    reqs = serve.workload(40, seed=5, rate=1000.0, n_max=2048, k_max=16)
    for r in reqs:
        r.ws_bytes = 1
    done, sched, ex = _run(reqs, slots=2, budget=10)
    starts = [rid for (what, rid, slot, t) in ex.log if what == "start"]
    assert starts == sorted(starts), "admission reordered requests"


def test_memory_budget_is_never_exceeded_and_limits_concurrency():
    reqs = [serve.Request(rid=i, arrival=0.0, n=100, k=5, ws_bytes=400) for i in range(12)]
    done, sched, ex = _run(reqs, slots=8, budget=1000)
    assert sched.peak_mem <= 1000
    assert sched.peak_running == 2          # 3 x 400 > 1000
    # with a larger budget the slots are the limit
    reqs = [serve.Request(rid=i, arrival=0.0, n=100, k=5, ws_bytes=400) for i in range(12)]
    done, sched, ex = _run(reqs, slots=8, budget=10 ** 6)
    assert sched.peak_running == 8


def test_request_larger_than_budget_is_refused():
    reqs = [serve.Request(rid=0, arrival=0.0, n=10, k=1, ws_bytes=2000)]
    with pytest.raises(ValueError):
        _run(reqs, slots=1, budget=1000)


def test_overlapping_requests_shorten_latency():
    reqs = [serve.Request(rid=i, arrival=0.0, n=1000, k=5, ws_bytes=1) for i in range(8)]
    d1, _, _ = _run([serve.Request(**{**vars(r)}) for r in reqs], slots=1, budget=100)
    d4, _, _ = _run([serve.Request(**{**vars(r)}) for r in reqs], slots=4, budget=100)
    s1, s4 = serve.summary(d1), serve.summary(d4)
    assert s4["p99_ms"] < s1["p99_ms"]
    assert s4["queries_per_s"] > s1["queries_per_s"]


def test_workload_distribution():
    reqs = serve.workload(4000, seed=9, rate=50.0, n_max=8192, k_max=256)
    n = np.array([r.n for r in reqs])
    k = np.array([r.k for r in reqs])
    t = np.array([r.arrival for r in reqs])
    assert n.min() >= 1 and n.max() <= 8192
    assert k.min() >= 1 and k.max() <= 256
    # log-uniform: the median of log n is near log(8192)/2
    assert abs(np.median(np.log(n)) - math.log(8192) / 2) < 0.2
    # Poisson arrivals: mean gap 1/rate, gaps ~ exponential (cv ~ 1)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 50.0) < 0.002
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    assert np.all(gaps >= 0)


def test_summary_percentiles():
    reqs = [serve.Request(rid=i, arrival=0.0, n=1, k=1) for i in range(100)]
    for i, r in enumerate(reqs):
        r.done = (i + 1) * 1e-3
    s = serve.summary(reqs)
    assert s["requests"] == 100 and s["queries"] == 100
    assert abs(s["p50_ms"] - 50.5) < 1e-9
    assert abs(s["p99_ms"] - 99.01) < 1e-6
