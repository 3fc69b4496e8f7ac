"""Serving on the GPU: results of requests served concurrently (several
slots, overlapping streams, resident graphs) equal the results of the same
queries made one at a time, and the oracle's."""
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


def test_results_alone_equal_results_in_the_mix():
    pool = graphgen.rmat_pool(8, seed=11, n_min=1 << 8, n_max=1 << 13)
    backend = serve.GpuBackend(pool)
    srv = serve.Server(backend, slots=6, budget_bytes=8 << 30)
    trace = serve.poisson_trace(160, rate=0, graph_ids=list(pool), seed=12)
    serve.replay(srv, trace)
    srv.shutdown()
    reqs = [r for _, r in trace]
    assert all(r.error is None for r in reqs), [r.error for r in reqs if r.error]
    assert srv.max_concurrent >= 2
    # alone: one graph, one call at a time, default stream
    alone = {}
    for gid, (s, d, n) in pool.items():
        g = tc.tc_build_csr(s, d, n)
        alone[(gid, "count", 0)] = tc.tc_count(g)
        for k in range(3, 9):
            alone[(gid, "ktruss", k)] = tc.ktruss(g, k)[1]
        g.free()
    for r in reqs:
        assert r.result == alone[(r.graph, r.kind, r.k)], r
    # and the oracle, on a few graphs
    for gid in list(pool)[:3]:
        s, d, n = pool[gid]
        og = oracle.OracleGraph.from_edges(s, d, n)
        assert alone[(gid, "count", 0)] == og.count()
        for k in (3, 5, 8):
            assert alone[(gid, "ktruss", k)] == og.ktruss(k)[2]


def test_budget_forces_eviction_and_rebuild_on_gpu():
    pool = graphgen.rmat_pool(6, seed=13, n_min=1 << 9, n_max=1 << 11)
    backend = serve.GpuBackend(pool)
    two = sorted(backend.estimate_bytes(g) for g in pool)[-2:]
    srv = serve.Server(backend, slots=2, budget_bytes=sum(two))
    trace = serve.poisson_trace(60, rate=0, graph_ids=list(pool), seed=14)
    serve.replay(srv, trace)
    srv.shutdown()
    assert srv.evictions > 0
    for _, r in trace:
        s, d, n = pool[r.graph]
        g = tc.tc_build_csr(s, d, n)
        want = tc.tc_count(g) if r.kind == "count" else tc.ktruss(g, r.k)[1]
        g.free()
        assert r.result == want
