"""The serving scheduler's host logic on CPU, with a fake backend: every
request is served exactly once with its own result, a graph is never used
by two calls at once, resident bytes stay within the budget (least-recently
used idle graphs are evicted), and requests overlap."""
import threading
import time

import pytest

from paper_1708_06866_gb300 import serve


class FakeBackend:
    def __init__(self, sizes, delay=0.002):
        self.sizes = sizes
        self.delay = delay
        self.lock = threading.Lock()
        self.in_use = set()
        self.resident_bytes = 0
        self.peak_bytes = 0
        self.violations = []

    def new_stream(self):
        return object()

    def estimate_bytes(self, gid):
        return self.sizes[gid]

    def build(self, gid, stream):
        with self.lock:
            self.resident_bytes += self.sizes[gid]
            self.peak_bytes = max(self.peak_bytes, self.resident_bytes)
        time.sleep(self.delay)
        return {"gid": gid}

    def free(self, handle):
        with self.lock:
            self.resident_bytes -= self.sizes[handle["gid"]]

    def query(self, handle, req, stream):
        g = handle["gid"]
        with self.lock:
            if g in self.in_use:
                self.violations.append(g)
            self.in_use.add(g)
        time.sleep(self.delay)
        with self.lock:
            self.in_use.discard(g)
        return g * 1000 + (req.k if req.kind == "ktruss" else 1)


def expected(req):
    return req.graph * 1000 + (req.k if req.kind == "ktruss" else 1)


def test_all_served_once_with_overlap_and_exclusivity():
    be = FakeBackend({g: 10 for g in range(6)})
    srv = serve.Server(be, slots=4, budget_bytes=1000)
    trace = serve.poisson_trace(300, rate=0, graph_ids=range(6), seed=1)
    wall = serve.replay(srv, trace)
    srv.shutdown()
    reqs = [r for _, r in trace]
    assert len(srv.completed) == 300
    assert sorted(r.rid for r in srv.completed) == list(range(300))
    assert all(r.result == expected(r) and r.error is None for r in reqs)
    assert not be.violations
    assert srv.max_concurrent >= 2
    s = serve.summarize(reqs, wall)
    assert s["requests"] == 300 and s["p99_ms"] >= s["p50_ms"]


def test_budget_evicts_least_recently_used():
    sizes = {g: 40 for g in range(5)}
    be = FakeBackend(sizes)
    srv = serve.Server(be, slots=2, budget_bytes=100)     # two graphs fit at a time
    trace = serve.poisson_trace(120, rate=0, graph_ids=range(5), seed=2)
    serve.replay(srv, trace)
    srv.shutdown()
    assert all(r.result == expected(r) for _, r in trace)
    assert be.peak_bytes <= 100
    assert srv.evictions > 0 and srv.builds > 5


def test_backend_errors_are_reported_per_request():
    class Failing(FakeBackend):
        def query(self, handle, req, stream):
            if req.rid % 7 == 0:
                raise RuntimeError("boom")
            return super().query(handle, req, stream)
    be = Failing({g: 1 for g in range(3)})
    srv = serve.Server(be, slots=3, budget_bytes=100)
    trace = serve.poisson_trace(50, rate=0, graph_ids=range(3), seed=3)
    serve.replay(srv, trace)
    srv.shutdown()
    for _, r in trace:
        if r.rid % 7 == 0:
            assert r.error and r.result is None
        else:
            assert r.result == expected(r)


def test_poisson_trace_shape():
    tr = serve.poisson_trace(2000, rate=100.0, graph_ids=[1, 2, 3], seed=4)
    times = [t for t, _ in tr]
    assert times == sorted(times) and times[0] == 0.0
    assert 15 < times[-1] < 25           # ~2000 / 100 s
    kinds = [r.kind for _, r in tr]
    assert 0.4 < kinds.count("count") / 2000 < 0.6
    assert {r.k for _, r in tr if r.kind == "ktruss"} <= {3, 4, 5, 6, 7, 8}
