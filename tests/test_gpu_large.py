"""Full-size R-MAT scale 24 (268M generated pairs), in the bench's launch
configuration, against the oracle on sampled outputs and on properties that
hold at any size.

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
