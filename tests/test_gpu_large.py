"""Full-size workloads in the bench's launch configuration.

The 8192 x 8192 image graph (268M edges) is checked in full against the
closed forms of Section IV-C.  R-MAT scale 24 (268M generated pairs) is
checked against the oracle on sampled outputs and on properties that hold
at any size.

The oracle's full truss peel at this size takes hours, so:
  * the canonical edge list is compared in full (the oracle's cleaning is a
    sort and a repeat removal);
  * per-edge supports are compared on a seeded sample of edges, each counted
    by the oracle one by one; sum of supports = 3 * triangles;
  * for each k of 3, 4, 6, 8: survivors of the k-truss have support >= k - 2
    within it and removed edges close < k - 2 triangles with it (maximality),
    on seeded samples; the trusses nest; the reported size is the mask's.
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


def test_rmat24_full_size_sampled_against_oracle():
    w = graphgen.WORKLOADS["rmat24"]
    s, d, n = w.generate()
    g = tc.tc_build_csr(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
    m = g.m
    lo, hi = tc.tc_edges(g)
    lo = lo.cpu().numpy()
    hi = hi.cpu().numpy()
    T = tc.tc_count(g)
    sup, T2 = tc.tc_edge_support(g)
    sup = sup.cpu().numpy()
    masks = {}
    for k in w.truss_ks:
        mk, left = tc.ktruss(g, k)
        mk = mk.cpu().numpy()
        assert int(mk.sum()) == left
        masks[k] = mk
    g.free()
    del s, d

    s, d, n = w.generate()
    olo, ohi = oracle.canonical_edges(s, d, n)
    del s, d
    assert len(olo) == m
    assert np.array_equal(lo, olo) and np.array_equal(hi, ohi)
    del lo, hi
    assert T == T2 and int(sup.sum(dtype=np.int64)) == 3 * T
    og = oracle.OracleGraph(n, olo, ohi)
    rng = np.random.default_rng(24)
    sample = rng.integers(0, m, 3000)
    assert np.array_equal(og.support_of(sample), sup[sample])
    prev = None
    for k in w.truss_ks:
        mk = masks[k]
        if prev is not None:
            assert not (mk.astype(bool) & ~prev.astype(bool)).any()
        prev = mk
        inside = np.flatnonzero(mk)
        outside = np.flatnonzero(mk == 0)
        if len(inside):
            si = rng.choice(inside, min(1500, len(inside)), replace=False)
            assert (og.support_within_of(mk, si) >= k - 2).all(), k
        if len(outside):
            so = rng.choice(outside, min(1500, len(outside)), replace=False)
            assert (og.support_within_of(mk, so) < k - 2).all(), k


def king_expected_support(lo, hi, M):
    """Closed-form support of every edge of the M x M image graph (Section
    IV-C): a diagonal edge closes 2 triangles; a horizontal edge 4, or 2 on
    the top and bottom rows; a vertical edge 4, or 2 on the side columns."""
    lo = lo.astype(np.int64)
    d = hi.astype(np.int64) - lo
    r, c = lo // M, lo % M
    out = np.full(len(lo), -1, dtype=np.int32)
    diag = (d == M + 1) | (d == M - 1)
    out[diag] = 2
    horiz = d == 1
    out[horiz] = np.where((r[horiz] == 0) | (r[horiz] == M - 1), 2, 4)
    vert = d == M
    out[vert] = np.where((c[vert] == 0) | (c[vert] == M - 1), 2, 4)
    return out


def test_king_graph_8192_closed_forms():
    """The bench's image-graph workload at full size (268M edges) against
    what Section IV-C fixes: m = (M-1)(4M-2), T = 4(M-1)^2, the support of
    every edge by its position, the 4-truss is the whole graph, the 5-truss
    is empty, so kmax = 4 and every truss number is 4."""
    M = 8192
    s, d, n = graphgen.WORKLOADS["king8192"].generate()
    g = tc.tc_build_csr(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
    del s, d
    m = (M - 1) * (4 * M - 2)
    assert g.m == m
    T = tc.tc_count(g)
    assert T == 4 * (M - 1) ** 2
    lo, hi = tc.tc_edges(g)
    lo = lo.cpu().numpy()
    hi = hi.cpu().numpy()
    # m distinct pairs, lexicographic, each an image-graph edge: the edge set
    key = lo.astype(np.int64) * n + hi
    assert (np.diff(key) > 0).all() and (lo < hi).all()
    sup_want = king_expected_support(lo, hi, M)
    assert (sup_want > 0).all()
    dr = hi // M - lo // M
    dc = hi % M - lo % M
    assert (((dr == 0) & (dc == 1)) | ((dr == 1) & (np.abs(dc) <= 1))).all()
    del key, dr, dc
    sup, T2 = tc.tc_edge_support(g)
    assert T2 == T
    assert np.array_equal(sup.cpu().numpy(), sup_want)
    del sup, sup_want, lo, hi
    for k, left in ((3, m), (4, m), (5, 0)):
        mk, c = tc.ktruss(g, k)
        assert c == left and int(mk.sum()) == left, k
    kmax, truss = tc.ktruss_max(g)
    assert kmax == 4
    assert (truss == 4).all().item()
    g.free()
