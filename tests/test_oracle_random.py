"""Randomised pins for the oracle (CPU): on many small random graphs the
oracle's count, supports, k-truss masks and truss numbers equal brute force
over all vertex triples and the bulk-peel model of tests/test_peel_rules.py
(itself checked against the definition there)."""
import itertools

import numpy as np
import pytest

import oracle
from test_peel_rules import bulk_peel, triangles_of_edges

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


def brute(n, lo, hi):
    A = np.zeros((n, n), dtype=bool)
    A[lo, hi] = A[hi, lo] = True
    idx = {(int(a), int(b)): e for e, (a, b) in enumerate(zip(lo, hi))}
    s = np.zeros(len(lo), dtype=np.int64)
    T = 0
    for a, b, c in itertools.combinations(range(n), 3):
        if A[a, b] and A[a, c] and A[b, c]:
            T += 1
            s[idx[(a, b)]] += 1
            s[idx[(a, c)]] += 1
            s[idx[(b, c)]] += 1
    return T, s


def exhaustive_ktruss(m, tri, k):
    """Largest edge subset in which every edge closes >= k - 2 triangles
    (by removing, one at a time, edges that close too few: the unique
    maximal such subset)."""
    keep = [True] * m
    changed = True
    while changed:
        changed = False
        for e in range(m):
            if keep[e] and sum(1 for f, g in tri[e] if keep[f] and keep[g]) < k - 2:
                keep[e] = False
                changed = True
    return np.array(keep, dtype=np.uint8)


@settings(max_examples=120, deadline=None)
@given(n=st.integers(2, 13), pairs=st.lists(st.tuples(st.integers(0, 12), st.integers(0, 12)),
                                             max_size=60))
def test_oracle_on_random_small_graphs(n, pairs):
    pairs = [(a % n, b % n) for a, b in pairs]
    src = np.array([a for a, _ in pairs], dtype=np.int32)
    dst = np.array([b for _, b in pairs], dtype=np.int32)
    og = oracle.OracleGraph.from_edges(src, dst, n)
    lo, hi = oracle.canonical_edges(src, dst, n)
    T, s = brute(n, lo, hi)
    assert og.count() == T
    assert np.array_equal(og.support(), s)
    tri = triangles_of_edges(n, lo, hi)
    for k in (2, 3, 4, 5):
        mask, _, left = og.ktruss(k)
        assert np.array_equal(mask, exhaustive_ktruss(len(lo), tri, k)), k
        assert left == int(mask.sum())
    kmax, truss = og.truss_decomposition()
    _, mkmax, mtruss = bulk_peel(tri, 3, single=False)
    assert kmax == mkmax
    assert np.array_equal(truss, mtruss)
