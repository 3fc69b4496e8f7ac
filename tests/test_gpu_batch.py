"""Batches (tc_batch_run) against the oracle and against per-graph calls.

Every graph's triangle count, edge count and k-truss size must be the same
alone (separate ABI calls, and the oracle) and inside the batch, with the
query phase captured into a CUDA graph or not, and whichever kernel forms the
autotuner picked.
"""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1708_06866_gb300 as tc  # noqa: E402


def mixed_batch(seed=0):
    """Varied members: R-MAT, Erdős–Rényi, complete graphs, an image graph,
    a single vertex, self-loops only, repeats and reversals, a star."""
    rng = np.random.default_rng(seed)
    graphs = []
    for i in range(24):
        kind = i % 6
        if kind == 0:
            s, d, n = graphgen.rmat(int(rng.integers(5, 11)), seed=100 + i)
        elif kind == 1:
            n = int(rng.integers(20, 3000))
            s, d, n = graphgen.er(n, int(n * rng.uniform(2, 10)), seed=200 + i)
        elif kind == 2:
            s, d, n = graphgen.complete(int(rng.integers(3, 40)))
        elif kind == 3:
            s, d, n = graphgen.king(int(rng.integers(2, 30)))
        elif kind == 4:
            s, d, n = graphgen.rmat_n(int(rng.integers(50, 2000)), 8, seed=300 + i)
            s, d = graphgen.messy(s, d, seed=i, loops=20, dup_frac=0.3, flip_frac=0.3)
        else:
            s, d, n = graphgen.star(int(rng.integers(2, 500)))
        graphs.append((np.asarray(s, np.int32), np.asarray(d, np.int32), int(n)))
    graphs.append((np.zeros(0, np.int32), np.zeros(0, np.int32), 1))      # one vertex
    graphs.append((np.array([3, 3, 5], np.int32), np.array([3, 3, 5], np.int32), 7))  # loops only
    graphs.insert(5, (np.zeros(0, np.int32), np.zeros(0, np.int32), 12))  # isolated vertices
    return graphs


def pack(graphs):
    n = np.array([g[2] for g in graphs], np.int32)
    off = np.zeros(len(graphs) + 1, np.int64)
    off[1:] = np.cumsum([len(g[0]) for g in graphs])
    src = np.concatenate([g[0] for g in graphs]) if off[-1] else np.zeros(0, np.int32)
    dst = np.concatenate([g[1] for g in graphs]) if off[-1] else np.zeros(0, np.int32)
    return n, off, src, dst


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_matches_oracle_per_graph(use_graph):
    graphs = mixed_batch()
    n, off, src, dst = pack(graphs)
    out = tc.tc_batch_run(n, off, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(),
                          k=4, use_graph=use_graph)
    assert out["stats"]["captured"] == int(use_graph)
    for i, (s, d, nv) in enumerate(graphs):
        og = oracle.OracleGraph.from_edges(s, d, nv)
        assert out["edges"][i] == og.m, i
        assert out["triangles"][i] == og.count(), i
        assert out["truss_edges"][i] == og.ktruss(4)[2], i
    assert out["stats"]["triangles"] == out["triangles"].sum()
    assert out["stats"]["m"] == out["edges"].sum()


def test_batch_equals_separate_calls_and_tuner_cache():
    n, off, src, dst, kind = graphgen.batch(60, seed=7, n_max=4096)
    first = tc.tc_batch_run(n, off, src, dst, k=4)       # host inputs
    second = tc.tc_batch_run(n, off, torch.from_numpy(src).cuda(),
                             torch.from_numpy(dst).cuda(), k=4)
    assert second["stats"]["tuned_from_cache"] == 1
    for key in ("triangles", "edges", "truss_edges"):
        assert np.array_equal(first[key], second[key])
    for i in range(len(n)):
        s = src[off[i]:off[i + 1]]
        d = dst[off[i]:off[i + 1]]
        g = tc.tc_build_csr(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), int(n[i]))
        assert g.m == first["edges"][i]
        assert tc.tc_count(g) == first["triangles"][i]
        assert tc.ktruss(g, 4)[1] == first["truss_edges"][i]
        g.free()


def test_batch_count_only_and_errors():
    graphs = mixed_batch(1)[:10]
    n, off, src, dst = pack(graphs)
    out = tc.tc_batch_run(n, off, src, dst, k=0)
    assert out["stats"]["peel_form"] == 0
    assert np.array_equal(out["truss_edges"], out["edges"])
    bad = src.copy()
    bad[0] = n[0] + 5            # outside graph 0
    with pytest.raises(tc.TCError) as ei:
        tc.tc_batch_run(n, off, bad, dst, k=0)
    assert ei.value.code == tc.TC_ERANGE
    with pytest.raises(tc.TCError) as ei:
        tc.tc_batch_run(n, off, src, dst, k=1)
    assert ei.value.code == tc.TC_EINVAL


def test_batch10k_sample_against_stored_oracle():
    """The bench's batch (10,000 graphs, n log-uniform in [64, 65536], half
    Erdős–Rényi and half R-MAT, seed 3) in one captured launch: a seeded
    sample of 200 graphs covering every size class has the oracle's stored
    edge count, triangle count and 4-truss size."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "batch10k_sample_oracle.txt")
    rows = []
    with open(path) as f:
        for ln in f:
            p = ln.split("#", 1)[0].split()
            if p and p[0] == "g":
                rows.append([int(x) for x in p[1:]])
    assert len(rows) >= 200
    n, off, src, dst, kind = graphgen.batch(10_000, seed=3)
    out = tc.tc_batch_run(n, off, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(),
                          k=4, use_graph=True)
    del src, dst
    for i, nv, m, T, t4 in rows:
        assert n[i] == nv
        assert (out["edges"][i], out["triangles"][i], out["truss_edges"][i]) == (m, T, t4), i
