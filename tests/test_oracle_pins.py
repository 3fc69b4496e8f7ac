"""Pins for the CPU oracle: checks against what the paper and the mathematics fix.

Every oracle function is checked here against something other than itself:
  * brute force over all vertex triples on small graphs (count, support);
  * closed forms: K_n, trees/stars/paths/4-grids, the 8-neighbour image graphs
    of Section IV-C (vertices, edges and triangles; Table II's printed values);
  * the paper's Fig. 1 and Fig. 2 examples (tests/golden);
  * a float64 dense trace(A^3) / 6 and (A^2)_uv on the 4096-vertex
    Erdős–Rényi workload (Algorithm 2 of Section III-A; exact, all values < 2^53);
  * a literal dense statement of Algorithm 4 (incidence matrix, R = E A,
    incremental update) on small graphs (k-truss masks and supports);
  * a bulk-removal fixed point and an exhaustive search over edge subsets for
    the k-truss definition of Section III-B.
"""
import itertools
import math
import os

import numpy as np
import pytest

import graphgen
import oracle
from conftest import ROOT, read_fixture


# ----------------------------------------------------------------- helpers

def dense_adj(n, lo, hi):
    A = np.zeros((n, n), dtype=np.int64)
    A[lo, hi] = 1
    A[hi, lo] = 1
    return A


def brute_triangles(n, A):
    """All triples a < b < c with the three edges present."""
    tri = []
    for a in range(n):
        for b in range(a + 1, n):
            if not A[a, b]:
                continue
            for c in range(b + 1, n):
                if A[a, c] and A[b, c]:
                    tri.append((a, b, c))
    return tri


def brute_support(lo, hi, tris):
    idx = {(int(a), int(b)): e for e, (a, b) in enumerate(zip(lo, hi))}
    s = np.zeros(len(lo), dtype=np.int64)
    for a, b, c in tris:
        s[idx[(a, b)]] += 1
        s[idx[(a, c)]] += 1
        s[idx[(b, c)]] += 1
    return s


def bulk_fixed_point_truss(n, lo, hi, k):
    """k-truss by repeated simultaneous removal, supports recounted by brute force."""
    alive = np.ones(len(lo), dtype=bool)
    while True:
        A = np.zeros((n, n), dtype=np.int64)
        A[lo[alive], hi[alive]] = 1
        A[hi[alive], lo[alive]] = 1
        s = np.array([int((A[a] & A[b]).sum()) if alive[e] else 0
                      for e, (a, b) in enumerate(zip(lo, hi))])
        drop = alive & (s < k - 2)
        if not drop.any():
            return alive
        alive &= ~drop


def exhaustive_truss(lo, hi, k):
    """Union of all edge subsets in which every edge lies in >= k-2 triangles of the subset."""
    m = len(lo)
    best = np.zeros(m, dtype=bool)
    for bits in range(1 << m):
        sel = [(bits >> e) & 1 for e in range(m)]
        es = {(int(lo[e]), int(hi[e])) for e in range(m) if sel[e]}
        ok = True
        for (a, b) in es:
            cnt = 0
            for w in range(int(max(hi)) + 1 if m else 0):
                if w in (a, b):
                    continue
                if (min(a, w), max(a, w)) in es and (min(b, w), max(b, w)) in es:
                    cnt += 1
            if cnt < k - 2:
                ok = False
                break
        if ok:
            for e in range(m):
                if sel[e]:
                    best[e] = True
    return best


def literal_algorithm4(n, lo, hi, k):
    """Algorithm 4 of Section III-B, stated with dense integer matrices.

    E is the unoriented incidence matrix (one row per edge, a 1 in each of its
    two vertex columns); the rows removed keep their original edge ids so the
    surviving set can be compared.  Returns (mask, support within the truss).
    """
    m = len(lo)
    E = np.zeros((m, n), dtype=np.int64)
    E[np.arange(m), lo] = 1
    E[np.arange(m), hi] = 1
    ids = np.arange(m)
    d = E.sum(axis=0)
    A = E.T @ E - np.diag(d)
    R = E @ A
    s = (R == 2).sum(axis=1)
    x = np.flatnonzero(s < k - 2)
    while len(x):
        keep = np.ones(len(ids), dtype=bool)
        keep[x] = False
        Ex = E[x]
        E = E[keep]
        ids = ids[keep]
        dx = Ex.sum(axis=0)
        R = R[keep]
        R = R - E @ (Ex.T @ Ex - np.diag(dx))
        s = (R == 2).sum(axis=1)
        x = np.flatnonzero(s < k - 2)
    mask = np.zeros(m, dtype=np.uint8)
    mask[ids] = 1
    sup = np.zeros(m, dtype=np.int64)
    sup[ids] = s
    return mask, sup


def small_random_graphs(count, nmax, seed):
    rng = np.random.default_rng(seed)
    for i in range(count):
        n = int(rng.integers(1, nmax + 1))
        p = float(rng.uniform(0.05, 0.9))
        A = rng.random((n, n)) < p
        A = np.triu(A, 1)
        lo, hi = np.nonzero(A)
        yield n, lo.astype(np.int32), hi.astype(np.int32)


# ----------------------------------------------------------------- cleaning

def test_canonical_edges_cleaning_rules():
    # Section II: self-loops removed, reversed and repeated pairs collapse to one edge
    src = np.array([3, 1, 2, 2, 0, 1, 3, 0], dtype=np.int32)
    dst = np.array([1, 3, 2, 0, 2, 3, 3, 1], dtype=np.int32)
    lo, hi = oracle.canonical_edges(src, dst, 4)
    assert list(zip(lo.tolist(), hi.tolist())) == [(0, 1), (0, 2), (1, 3)]


def test_canonical_edges_messy_equals_clean():
    s, d, n = graphgen.er(300, 2000, seed=5)
    ms, md = graphgen.messy(s, d, seed=1, loops=50, dup_frac=0.5, flip_frac=0.5)
    a = oracle.canonical_edges(s, d, n)
    b = oracle.canonical_edges(ms, md, n)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert len(a[0]) == 2000


def test_canonical_edges_rejects_bad_ids():
    with pytest.raises(ValueError):
        oracle.canonical_edges([0, 5], [1, 2], 5)
    with pytest.raises(ValueError):
        oracle.canonical_edges([-1], [1], 5)


def test_oracle_open_rejects_non_canonical():
    with pytest.raises(ValueError):
        oracle.OracleGraph(3, np.array([1, 0]), np.array([2, 1]))  # not sorted
    with pytest.raises(ValueError):
        oracle.OracleGraph(3, np.array([0, 0]), np.array([1, 1]))  # repeated


def test_empty_and_tiny_graphs():
    g = oracle.OracleGraph(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert g.count() == 0 and len(g.support()) == 0
    assert g.truss_decomposition()[0] == 0
    g = oracle.OracleGraph(2, np.array([0]), np.array([1]))
    assert g.count() == 0 and g.support().tolist() == [0]
    kmax, t = g.truss_decomposition()
    assert kmax == 2 and t.tolist() == [2]
    mask, _, left = g.ktruss(2)
    assert left == 1 and mask.tolist() == [1]
    mask, _, left = g.ktruss(3)
    assert left == 0
    with pytest.raises(ValueError):
        g.ktruss(1)


# ----------------------------------------------------------------- brute force

def test_count_and_support_match_brute_force():
    for n, lo, hi in small_random_graphs(60, 40, seed=11):
        g = oracle.OracleGraph(n, lo, hi)
        tris = brute_triangles(n, dense_adj(n, lo, hi))
        assert g.count() == len(tris)
        assert np.array_equal(g.support(), brute_support(lo, hi, tris))
        assert g.support().sum() == 3 * len(tris)
        sel = np.arange(0, len(lo), 3)
        assert np.array_equal(g.support_of(sel), brute_support(lo, hi, tris)[sel])


# ----------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [3, 4, 5, 7, 12, 30])
def test_complete_graph(n):
    s, d, _ = graphgen.complete(n)
    g = oracle.OracleGraph.from_edges(s, d, n)
    assert g.count() == math.comb(n, 3)
    assert (g.support() == n - 2).all()
    kmax, t = g.truss_decomposition()
    assert kmax == n and (t == n).all()
    assert g.ktruss(n)[2] == g.m
    assert g.ktruss(n + 1)[2] == 0


@pytest.mark.parametrize("maker", [
    lambda: graphgen.star(50), lambda: graphgen.path(64), lambda: graphgen.random_tree(200, 3),
    lambda: graphgen.grid4(12)])
def test_triangle_free_families(maker):
    s, d, n = maker()
    g = oracle.OracleGraph.from_edges(s, d, n)
    assert g.count() == 0
    assert (g.support() == 0).all()
    kmax, t = g.truss_decomposition()
    assert kmax == 2 and (t == 2).all()


def king_support(M, lo, hi):
    """Closed-form supports of the image graph: diagonal edges 2; axis edges 4
    inside, 2 on the border rows/columns they run along."""
    r0, c0, r1, c1 = lo // M, lo % M, hi // M, hi % M
    diag = (r0 != r1) & (c0 != c1)
    horiz = r0 == r1
    border = np.where(horiz, (r0 == 0) | (r0 == M - 1), (c0 == 0) | (c0 == M - 1))
    return np.where(diag, 2, np.where(border, 2, 4))


@pytest.mark.parametrize("M", [2, 3, 4, 8, 17, 64])
def test_image_graph_closed_forms(M):
    s, d, n = graphgen.king(M)
    assert n == M * M
    g = oracle.OracleGraph.from_edges(s, d, n)
    assert g.m == (M - 1) * (4 * M - 2)
    assert g.count() == 4 * (M - 1) ** 2
    assert np.array_equal(g.support(), king_support(M, g.lo, g.hi))
    kmax, t = g.truss_decomposition()
    assert kmax == 4 and (t == 4).all()


def test_table2_image_graphs():
    """Table II: vertex and edge columns match the generator; the printed
    triangle column is 2x the true count, which the oracle gives."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "table2_image_graphs.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([int(v) for v in line.split()])
    assert len(rows) == 6
    for p, nodes, edges, printed in rows:
        M = 2 ** p
        assert nodes == M * M
        assert edges == (M - 1) * (4 * M - 2)
        assert printed == 8 * (M - 1) ** 2
    for p, nodes, edges, printed in rows[:2]:   # n = 8, 9 run through the oracle
        s, d, n = graphgen.king(2 ** p)
        g = oracle.OracleGraph.from_edges(s, d, n)
        assert g.n == nodes and g.m == edges
        assert g.count() == printed // 2


def test_fig1_diamond():
    fx = read_fixture("fig1_diamond.txt")
    e = np.array(fx["edge"], dtype=np.int32)
    g = oracle.OracleGraph.from_edges(e[:, 0], e[:, 1], 4)
    assert g.count() == fx["triangles"][0][0]
    assert g.support().tolist() == fx["support"][0]


def test_fig2_pendant_3truss():
    fx = read_fixture("fig2_pendant.txt")
    e = np.array(fx["edge"], dtype=np.int32)
    g = oracle.OracleGraph.from_edges(e[:, 0], e[:, 1], 4)
    mask, _, left = g.ktruss(3)
    assert mask.tolist() == fx["truss3"][0] and left == 3


# ----------------------------------------------------------------- Algorithm 2 in float64

def test_er4096_trace_of_A_cubed():
    """Algorithm 2: n_T = sum(A^2 ∘ A) / 6; per-edge support = (A^2)_uv.

    Dense float64 on the 4096-vertex workload; every entry of A^2 is at most
    4095 and every sum below 2^53, so the float64 products are exact."""
    w = graphgen.WORKLOADS["er4096"]
    s, d, n = w.generate()
    g = oracle.OracleGraph.from_edges(s, d, n)
    A = np.zeros((n, n), dtype=np.float64)
    A[g.lo, g.hi] = 1.0
    A[g.hi, g.lo] = 1.0
    A2 = A @ A
    T = int(round((A2 * A).sum() / 6.0))
    assert g.count() == T
    assert np.array_equal(g.support(), A2[g.lo, g.hi].astype(np.int64))
    assert g.support().sum() == 3 * T


# ----------------------------------------------------------------- k-truss

def test_ktruss_matches_literal_algorithm4():
    for n, lo, hi in small_random_graphs(40, 24, seed=7):
        if len(lo) == 0:
            continue
        g = oracle.OracleGraph(n, lo, hi)
        for k in (2, 3, 4, 5, 6):
            mask_ref, sup_ref = literal_algorithm4(n, lo, hi, k)
            mask, sup, left = g.ktruss(k)
            assert np.array_equal(mask, mask_ref), (n, k)
            assert np.array_equal(sup, sup_ref), (n, k)
            assert left == int(mask_ref.sum())


def test_ktruss_matches_bulk_fixed_point():
    for n, lo, hi in small_random_graphs(40, 12, seed=3):
        g = oracle.OracleGraph(n, lo, hi)
        for k in (3, 4, 5):
            assert np.array_equal(g.ktruss(k)[0].astype(bool),
                                  bulk_fixed_point_truss(n, lo, hi, k)), (n, k)


def test_ktruss_matches_exhaustive_definition():
    rng = np.random.default_rng(4)
    done = 0
    while done < 12:
        n = int(rng.integers(3, 7))
        A = np.triu(rng.random((n, n)) < 0.7, 1)
        lo, hi = np.nonzero(A)
        if len(lo) == 0 or len(lo) > 12:
            continue
        g = oracle.OracleGraph(n, lo.astype(np.int32), hi.astype(np.int32))
        for k in (3, 4, 5):
            assert np.array_equal(g.ktruss(k)[0].astype(bool), exhaustive_truss(lo, hi, k))
        done += 1


def test_truss_decomposition_consistent_with_ktruss():
    s, d, n = graphgen.rmat(10, seed=9)
    g = oracle.OracleGraph.from_edges(s, d, n)
    kmax, t = g.truss_decomposition()
    assert kmax >= 3
    prev = None
    for k in range(2, kmax + 2):
        mask, sup, left = g.ktruss(k)
        assert np.array_equal(mask.astype(bool), t >= k), k
        # every survivor lies in >= k-2 triangles of the truss
        within = g.support_within(mask)
        assert np.array_equal(within, sup)
        assert (sup[mask == 1] >= k - 2).all()
        if prev is not None:
            assert not (mask.astype(bool) & ~prev).any()   # nesting
        prev = mask.astype(bool)
    assert g.ktruss(kmax + 1)[2] == 0 and g.ktruss(kmax)[2] > 0


def test_truss_levels_equal_the_bulk_fixed_point_at_each_k():
    """The decomposition's first levels (one support pass, then k = 3, 4, ...
    each continuing from the previous survivors) give, at every k, the size
    of the k-truss found by an independent bulk fixed point on the whole
    graph (the k-trusses nest, Section III-B); K_n: every edge up to k = n,
    nothing above."""
    for n, lo, hi in small_random_graphs(30, 14, seed=6):
        g = oracle.OracleGraph(n, lo, hi)
        sizes = g.truss_levels(7)
        want = [int(bulk_fixed_point_truss(n, lo, hi, k).sum()) for k in range(3, 8)]
        assert sizes == want, (n, sizes, want)
    s, d, n = graphgen.complete(9)
    g = oracle.OracleGraph.from_edges(s, d, n)
    assert g.truss_levels(11) == [36] * 7 + [0, 0]
    with pytest.raises(ValueError):
        g.truss_levels(2)


def test_support_invariant_on_rmat():
    s, d, n = graphgen.rmat(12, seed=1)
    g = oracle.OracleGraph.from_edges(s, d, n)
    assert g.support().sum() == 3 * g.count()


def test_support_within_of_matches_full_version():
    s, d, n = graphgen.rmat(10, seed=3)
    g = oracle.OracleGraph.from_edges(s, d, n)
    mask, sup, _ = g.ktruss(5)
    sel = np.flatnonzero(mask)[::7]
    assert np.array_equal(g.support_within_of(mask, sel), g.support_within(mask)[sel])
    assert np.array_equal(g.support_within_of(mask, sel), sup[sel])


def test_edges_outside_a_truss_close_too_few_triangles_with_it():
    """Maximality of the k-truss (Section III-B): an edge outside it closes
    fewer than k - 2 triangles with truss edges."""
    s, d, n = graphgen.rmat(11, seed=4)
    g = oracle.OracleGraph.from_edges(s, d, n)
    for k in (3, 4, 6, 8):
        mask, _, _ = g.ktruss(k)
        out = np.flatnonzero(mask == 0)
        if len(out):
            assert (g.support_within_of(mask, out) < k - 2).all()


# ------------------------------------------------------- truss components

def closure_components(n, lo, hi, mask):
    """Connected components of the masked edges by boolean reachability
    (squaring I + A until it is stable), independent of the oracle's search:
    label = smallest vertex reachable, -1 for vertices without a masked edge."""
    sel = np.asarray(mask).astype(bool)
    R = np.eye(n, dtype=bool)
    R[lo[sel], hi[sel]] = True
    R[hi[sel], lo[sel]] = True
    while True:
        R2 = (R.astype(np.int64) @ R.astype(np.int64)) > 0
        if (R2 == R).all():
            break
        R = R2
    touched = np.zeros(n, dtype=bool)
    touched[lo[sel]] = True
    touched[hi[sel]] = True
    vl = np.where(touched, R.argmax(axis=1), -1).astype(np.int32)
    el = np.where(sel, vl[lo] if len(lo) else np.zeros(0, np.int32), -1).astype(np.int32)
    return el, vl, len(set(vl[touched].tolist()))


def test_components_match_reachability():
    rng = np.random.default_rng(8)
    for n, lo, hi in small_random_graphs(40, 30, seed=7):
        g = oracle.OracleGraph(n, lo, hi)
        masks = [rng.random(len(lo)) < 0.3, np.ones(len(lo), bool)]
        masks += [g.ktruss(k)[0] for k in (3, 4)]
        for mk in masks:
            el, vl, c = g.components(mk)
            wel, wvl, wc = closure_components(n, lo, hi, mk)
            assert c == wc and np.array_equal(el, wel) and np.array_equal(vl, wvl)


def two_cliques_and_a_bridge():
    """K5 on 0..4, K5 on 10..14, a path 4-5-6-...-10 between them (n = 15)."""
    pairs = [(a, b) for a in range(5) for b in range(a + 1, 5)]
    pairs += [(a, b) for a in range(10, 15) for b in range(a + 1, 15)]
    pairs += [(i, i + 1) for i in range(4, 10)]
    s, d = np.array(pairs, dtype=np.int32).T
    return s, d, 15


def test_components_closed_forms():
    s, d, n = two_cliques_and_a_bridge()
    g = oracle.OracleGraph.from_edges(s, d, n)
    el, vl, c = g.ktruss_components(5)     # each K5: every edge in 3 triangles
    assert c == 2
    assert sorted(set(el[el >= 0].tolist())) == [0, 10] and (el >= 0).sum() == 20
    assert vl.tolist() == [0] * 5 + [-1] * 5 + [10] * 5
    el, vl, c = g.ktruss_components(2)     # the 2-truss: one component
    assert c == 1 and (el == 0).all()
    assert g.ktruss_components(6)[2] == 0
    for M in (3, 6):
        s, d, n = graphgen.king(M)
        g = oracle.OracleGraph.from_edges(s, d, n)
        el, vl, c = g.ktruss_components(4)
        assert c == 1 and (el == 0).all() and (vl == 0).all()
        el, vl, c = g.ktruss_components(5)
        assert c == 0 and (el == -1).all() and (vl == -1).all()
