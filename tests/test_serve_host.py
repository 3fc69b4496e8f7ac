"""The native server's host logic on CPU (its test hook runs the scheduler
with sleeps in place of device work, no CUDA calls): every request is
served exactly once with its own result, a graph is never used by two calls
at once, reserved bytes stay within the budget (least-recently-used idle
graphs are evicted), requests overlap, none starts before it arrives, and
malformed requests are refused."""
import numpy as np
import pytest

import paper_1708_06866_gb300 as tc
from paper_1708_06866_gb300 import serve


@pytest.fixture
def fake():
    prev = tc.tc_debug_server_fake(True)
    yield
    tc.tc_debug_server_fake(prev)


def pool_of(sizes):
    return {g: (np.zeros(m, np.int32), np.ones(m, np.int32), 2) for g, m in enumerate(sizes)}


def expected(r):
    return r.graph * 1000 + (0 if r.kind == "count" else r.k)


def test_every_request_served_once_with_its_result(fake):
    srv = serve.NativeServer(pool_of([1000] * 12), slots=6, budget_bytes=1 << 40)
    trace = serve.poisson_trace(400, 0, list(range(12)), seed=3)
    srv.run(trace, open_loop=False)
    st = srv.stats()
    for _, r in trace:
        assert r.error is None and r.result == expected(r)
        assert 0 <= r.slot < 6 and r.done >= r.start
    assert st["violations"] == 0
    assert st["max_concurrent"] >= 2
    assert st["builds"] == 12 and st["evictions"] == 0
    srv.close()


def test_budget_evicts_least_recently_used_idle_graphs(fake):
    sizes = [200_000] * 10   # each ~29 MB reserved: 140 B per pair + 1 MiB
    per = 140 * 200_000 + (1 << 20)
    budget = 3 * per + 1000
    srv = serve.NativeServer(pool_of(sizes), slots=4, budget_bytes=budget)
    trace = serve.poisson_trace(300, 0, list(range(10)), seed=5)
    srv.run(trace, open_loop=False)
    st = srv.stats()
    assert all(r.error is None and r.result == expected(r) for _, r in trace)
    assert st["peak_reserved_bytes"] <= budget
    assert st["evictions"] > 0 and st["builds"] == st["evictions"] + st["resident_graphs"]
    assert st["resident_graphs"] <= 3 and st["violations"] == 0
    srv.close()


def test_open_loop_respects_arrivals_and_keeps_graphs_between_runs(fake):
    srv = serve.NativeServer(pool_of([500] * 4), slots=3, budget_bytes=1 << 40)
    trace = serve.poisson_trace(60, 2000.0, [0, 1, 2, 3], seed=9)
    wall = srv.run(trace)
    assert wall >= trace[-1][0]
    for at, r in trace:
        assert r.error is None and r.result == expected(r)
        assert r.start >= at - 1e-6 and r.latency >= 0
    builds = srv.stats()["builds"]
    srv.run(serve.fresh(trace))
    assert srv.stats()["builds"] == builds      # still resident
    summ = serve.summarize([r for _, r in trace], wall)
    assert summ["errors"] == 0 and summ["p99_ms"] >= summ["p50_ms"]
    srv.close()


def test_bad_requests_and_arguments_are_refused(fake):
    srv = serve.NativeServer(pool_of([10, 10]), slots=2, budget_bytes=1 << 30)
    with pytest.raises(KeyError):
        srv.run([(0.0, serve.Request(0, 5, "count"))])
    with pytest.raises(tc.TCError) as ei:
        srv.run([(0.0, serve.Request(0, 1, "ktruss", 1))])
    assert ei.value.code == tc.TC_EINVAL
    with pytest.raises(tc.TCError):
        srv.run([(0.5, serve.Request(0, 0, "count")), (0.1, serve.Request(1, 1, "count"))])
    srv.close()
    with pytest.raises(tc.TCError):
        serve.NativeServer(pool_of([10]), slots=0)
    with pytest.raises(tc.TCError):
        serve.NativeServer(pool_of([10]), budget_bytes=0)


def test_waiting_requests_for_one_graph_are_answered_together(fake):
    """With several slots, a slot that takes a request also takes the
    requests for the same graph that have arrived and wait: they share one
    call (same slot, same start), each with its own result.  One slot is the
    plain loop: every request its own call."""
    srv = serve.NativeServer(pool_of([100] * 3), slots=2, budget_bytes=1 << 40)
    trace = [(0.0, serve.Request(i, i % 3, "ktruss" if i % 2 else "count", 3 + i % 5))
             for i in range(30)]
    for _, r in trace:
        if r.kind == "count":
            r.k = 0
    srv.run(trace, open_loop=False)
    calls = {(r.slot, r.start) for _, r in trace}
    assert len(calls) < len(trace)            # some calls answered several requests
    for _, r in trace:
        assert r.error is None and r.result == expected(r)
    for (slot, start) in calls:               # a call serves one graph
        assert len({r.graph for _, r in trace if (r.slot, r.start) == (slot, start)}) == 1
    one = serve.fresh(trace)
    srv.run(one, open_loop=False, slots=1)
    assert len({(r.slot, r.start) for _, r in one}) == len(one)
    assert all(r.error is None and r.result == expected(r) for _, r in one)
    srv.close()
