"""Serving on the GPU through the native server: results of requests served
concurrently (several slots, overlapping streams, resident graphs, kept
truss decompositions) equal the results of the same queries made one at a
time, and the oracle's; a small budget forces evictions and rebuilds with
the same results."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1708_06866_gb300 as tc  # noqa: E402
from paper_1708_06866_gb300 import serve  # noqa: E402


def alone_results(pool):
    """Every query answered alone: one graph, one call at a time, default stream."""
    out = {}
    for gid, (s, d, n) in pool.items():
        g = tc.tc_build_csr(s, d, n)
        out[(gid, "count", 0)] = tc.tc_count(g)
        for k in range(3, 9):
            out[(gid, "ktruss", k)] = tc.ktruss(g, k)[1]
        g.free()
    return out


def test_results_alone_equal_results_in_the_mix():
    pool = graphgen.rmat_pool(8, seed=11, n_min=1 << 8, n_max=1 << 13)
    srv = serve.NativeServer(pool, slots=6, budget_bytes=8 << 30)
    trace = serve.poisson_trace(200, rate=0, graph_ids=list(pool), seed=12)
    srv.run(trace, open_loop=False)
    # and again open loop, on resident graphs with kept decompositions
    trace2 = serve.poisson_trace(200, rate=5000.0, graph_ids=list(pool), seed=13)
    srv.run(trace2)
    st = srv.stats()
    srv.close()
    reqs = [r for _, r in trace + trace2]
    assert all(r.error is None for r in reqs), [r.error for r in reqs if r.error]
    assert st["max_concurrent"] >= 2 and st["errors"] == 0
    alone = alone_results(pool)
    for r in reqs:
        assert r.result == alone[(r.graph, r.kind, r.k)], r
    for gid in list(pool)[:3]:
        s, d, n = pool[gid]
        og = oracle.OracleGraph.from_edges(s, d, n)
        assert alone[(gid, "count", 0)] == og.count()
        for k in (3, 5, 8):
            assert alone[(gid, "ktruss", k)] == og.ktruss(k)[2]


def test_budget_forces_eviction_and_rebuild_on_gpu():
    pool = graphgen.rmat_pool(6, seed=13, n_min=1 << 9, n_max=1 << 11)
    est = sorted(140 * len(pool[g][0]) + (1 << 20) for g in pool)
    srv = serve.NativeServer(pool, slots=2, budget_bytes=sum(est[-2:]))
    trace = serve.poisson_trace(80, rate=0, graph_ids=list(pool), seed=14)
    srv.run(trace, open_loop=False)
    st = srv.stats()
    srv.close()
    assert st["evictions"] > 0 and st["errors"] == 0
    alone = alone_results(pool)
    for _, r in trace:
        assert r.error is None and r.result == alone[(r.graph, r.kind, r.k)], r


def test_failed_allocation_fails_one_request_and_the_server_goes_on():
    """An injected device-allocation failure during a run (on the host: the
    library's allocation hook) fails the call that hit it with TC_ENOMEM —
    the requests that call answered (several, when same-graph requests were
    coalesced) report the error; every other request in the run still gets
    its exact result, and the next run on the same server succeeds
    throughout."""
    pool = graphgen.rmat_pool(6, seed=21, n_min=1 << 8, n_max=1 << 11)
    alone = alone_results(pool)
    srv = serve.NativeServer(pool, slots=3, budget_bytes=4 << 30)
    trace = serve.poisson_trace(60, rate=0, graph_ids=list(pool), seed=22)
    tc.tc_debug_fail_alloc(25)          # the 25th device allocation from now fails
    try:
        srv.run(trace, open_loop=False)
    finally:
        tc.tc_debug_fail_alloc(0)
    failed = [r for _, r in trace if r.error is not None]
    assert len(failed) >= 1, [r.error for r in failed]
    assert all("code -3" in r.error for r in failed)
    assert len({(r.slot, r.start) for r in failed}) <= 2   # at most two calls failed
    for _, r in trace:
        if r.error is None:
            assert r.result == alone[(r.graph, r.kind, r.k)], r
    again = serve.fresh(trace)
    srv.run(again, open_loop=False)
    assert all(r.error is None and r.result == alone[(r.graph, r.kind, r.k)] for _, r in again)
    assert srv.stats()["errors"] == len(failed)
    srv.close()


def test_server_degenerate_graphs_and_k2():
    """Graphs with no edges, a single vertex, only loops and repeats, and a
    clique, served together; k = 2 (every edge) and k above kmax."""
    empty = (np.zeros(0, np.int32), np.zeros(0, np.int32), 5)
    single = (np.zeros(0, np.int32), np.zeros(0, np.int32), 1)
    loops = (np.array([0, 1, 1, 2], np.int32), np.array([0, 1, 1, 2], np.int32), 3)
    clique = graphgen.complete(7)
    pool = {0: empty, 1: single, 2: loops, 3: clique}
    want = {(0, "count", 0): 0, (1, "count", 0): 0, (2, "count", 0): 0, (3, "count", 0): 35}
    for g in (0, 1, 2):
        for k in (2, 3, 9):
            want[(g, "ktruss", k)] = 0
    for k in (2, 3, 7, 8, 9):
        want[(3, "ktruss", k)] = 21 if k <= 7 else 0
    trace = []
    for i, (key, _) in enumerate(sorted(want.items()) * 3):
        g, kind, k = key
        trace.append((0.0, serve.Request(i, g, kind, k)))
    srv = serve.NativeServer(pool, slots=4, budget_bytes=1 << 30)
    srv.run(trace, open_loop=False)
    srv.close()
    for _, r in trace:
        assert r.error is None and r.result == want[(r.graph, r.kind, r.k)], r


def _stored_pool_answers():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "serve_pool_oracle.txt")
    want = {}
    with open(path) as f:
        for ln in f:
            p = ln.split("#", 1)[0].split()
            if p and p[0] == "g":
                gid, m, T = int(p[1]), int(p[3]), int(p[4])
                want[(gid, "count", 0)] = T
                for k, c in zip(range(3, 9), p[5:]):
                    want[(gid, "ktruss", k)] = int(c)
    return want


def test_served_pool_matches_stored_oracle_with_results_not_kept():
    """The bench's pool (64 R-MAT graphs, n log-uniform in [2^10, 2^22], seed
    4) served concurrently with no results kept between requests (every
    k-truss request peels): every graph's triangle count and k-truss sizes for
    k = 3..8, in shuffled order, equal the oracle's stored answers."""
    want = _stored_pool_answers()
    pool = graphgen.rmat_pool(64, seed=4)
    keys = sorted(want)
    rng = np.random.default_rng(31)
    order = rng.permutation(len(keys))
    trace = [(0.0, serve.Request(i, *keys[j])) for i, j in enumerate(order)]
    srv = serve.NativeServer(pool, slots=8, budget_bytes=120 << 30, keep_results=False)
    srv.run(trace, open_loop=False)
    st = srv.stats()
    srv.close()
    assert st["errors"] == 0 and st["max_concurrent"] >= 2
    for _, r in trace:
        assert r.error is None and r.result == want[(r.graph, r.kind, r.k)], r


def test_results_alone_equal_results_in_the_mix_without_kept_results():
    """With no results kept, concurrent requests (each k-truss request a
    peel on the device, several at once on different streams) give what the
    same queries give alone."""
    pool = graphgen.rmat_pool(10, seed=17, n_min=1 << 8, n_max=1 << 14)
    srv = serve.NativeServer(pool, slots=8, budget_bytes=8 << 30, keep_results=False)
    trace = serve.poisson_trace(300, rate=0, graph_ids=list(pool), seed=18)
    srv.run(trace, open_loop=False)
    st = srv.stats()
    srv.close()
    assert st["errors"] == 0 and st["max_concurrent"] >= 2
    alone = alone_results(pool)
    for _, r in trace:
        assert r.error is None and r.result == alone[(r.graph, r.kind, r.k)], r
