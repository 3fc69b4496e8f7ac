"""The bulk peel's rules, run in plain Python and checked against the oracle.

The device peel (Section III-B's iteration, Algorithm 4's bulk removal)
removes a whole frontier per round and keeps per-edge supports up to date by
decrements.  It relies on rules that the oracle's one-edge-at-a-time peel
never needs:

  * ownership: a triangle destroyed in a round is handled by the smallest
    removed edge of that round among its edges, which lowers the support of
    each of its other edges that survives the round;
  * the next frontier is exactly the surviving edges whose support fell
    below k - 2 during the round;
  * level skipping: when a level's scan finds no edge below k - 2, the levels
    up to (smallest surviving support) + 2 remove nothing, so the next level
    to peel is that support + 3;
  * the truss number of an edge removed while peeling level k is k - 1;
  * windowed scans: a full scan (of the alive edges) also collects the
    "window" of alive edges with support below thr + WINDOW; the next levels
    scan only the window, which gains every edge whose support falls to just
    below the window bound during a round, and the level-skipping minimum of
    a windowed scan is capped at the bound.

This file states those rules as a slow model (no code shared with the CUDA
path or the oracle) and checks, on small graphs, that after every round each
surviving edge's support equals its number of live triangles, and that the
k-truss masks, kmax and truss numbers equal the oracle's.
"""
import numpy as np
import pytest

import graphgen
import oracle


def triangles_of_edges(n, lo, hi):
    """For every canonical edge, the pairs (f, g) of other edges that close a
    triangle with it."""
    idx = {(int(a), int(b)): e for e, (a, b) in enumerate(zip(lo, hi))}
    nbr = [set() for _ in range(n)]
    for a, b in zip(lo, hi):
        nbr[int(a)].add(int(b))
        nbr[int(b)].add(int(a))
    tri = [[] for _ in range(len(lo))]
    for e, (a, b) in enumerate(zip(lo, hi)):
        a, b = int(a), int(b)
        for w in nbr[a] & nbr[b]:
            f = idx[(min(a, w), max(a, w))]
            g = idx[(min(b, w), max(b, w))]
            tri[e].append((f, g))
    return tri


def bulk_peel(tri, k_first, single, owner_rule=True):
    """The device peel's rules.  Returns (alive mask, kmax, truss numbers);
    kmax is the largest truss number (0 without edges).  owner_rule=False
    drops the ownership rule (a plausible mistake: every removed edge of a
    triangle lowers its survivors)."""
    m = len(tri)
    s = [len(t) for t in tri]
    removed_in = [0] * m          # 0 = alive, r = removed in round r
    truss = [0] * m
    r, k = 1, k_first

    def live_triangles(x):
        return sum(1 for f, g in tri[x] if removed_in[f] == 0 and removed_in[g] == 0)

    while True:
        thr = k - 2
        alive = [e for e in range(m) if removed_in[e] == 0]
        frontier = [e for e in alive if s[e] < thr]
        if not frontier:
            if single or not alive:
                break
            k = max(k + 1, min(s[e] for e in alive) + 3)
            continue
        while frontier:
            for e in frontier:
                removed_in[e] = r
            dying = set(frontier)
            lowered = set()
            for e in frontier:
                for f, g in tri[e]:
                    if 0 < removed_in[f] < r or 0 < removed_in[g] < r:
                        continue  # destroyed in an earlier round
                    if owner_rule and min(x for x in (e, f, g) if x in dying) != e:
                        continue  # another removed edge of this round owns it
                    for x in (f, g):
                        if removed_in[x] == 0:
                            s[x] -= 1
                            lowered.add(x)
            for e in frontier:
                truss[e] = k - 1
            # every surviving support is the edge's number of live triangles
            for x in range(m):
                if removed_in[x] == 0:
                    assert s[x] == live_triangles(x), (x, s[x], live_triangles(x))
            frontier = sorted(x for x in lowered if s[x] < thr)
            r += 1
        if single:
            break
        if not any(removed_in[e] == 0 for e in range(m)):
            break
        k += 1
    mask = np.array([removed_in[e] == 0 for e in range(m)], dtype=np.uint8)
    return mask, max(truss, default=0), np.array(truss, dtype=np.int32)


def graphs():
    yield "er", graphgen.er(60, 420, seed=7)
    yield "rmat8", graphgen.rmat(8, edgefactor=8, seed=11)
    yield "K9", graphgen.complete(9)
    yield "king6", graphgen.king(6)
    s1, d1, _ = graphgen.complete(6)
    # two 6-cliques joined by a path of three edges, plus a pendant star
    src = np.concatenate([s1, s1 + 6, np.array([5, 12, 13, 0, 0, 0], np.int32)])
    dst = np.concatenate([d1, d1 + 6, np.array([12, 13, 6, 14, 15, 16], np.int32)])
    yield "cliques", (src.astype(np.int32), dst.astype(np.int32), 17)
    rng = np.random.default_rng(5)
    n = 24
    a = rng.integers(0, n, 200).astype(np.int32)
    b = rng.integers(0, n, 200).astype(np.int32)
    yield "dense24", (a, b, n)


@pytest.mark.parametrize("name,g", list(graphs()), ids=[n for n, _ in graphs()])
def test_bulk_rules_give_the_oracle_trusses(name, g):
    src, dst, n = g
    og = oracle.OracleGraph.from_edges(src, dst, n)
    lo, hi = oracle.canonical_edges(src, dst, n)
    tri = triangles_of_edges(n, lo, hi)
    assert sum(len(t) for t in tri) == 3 * og.count()
    for k in (3, 4, 5, 6):
        mask, _, _ = bulk_peel(tri, k, single=True)
        omask, _, _ = og.ktruss(k)
        assert np.array_equal(mask, omask), (name, k)
    _, kmax, truss = bulk_peel(tri, 3, single=False)
    okmax, otruss = og.truss_decomposition()
    assert kmax == okmax, name
    # the decomposition removes every edge, each with its truss number
    assert (truss >= 2).all(), name
    assert np.array_equal(truss, otruss), name


def test_dropping_the_ownership_rule_is_caught():
    """Without the ownership rule a triangle with two removed edges in one
    round lowers its third edge twice; the live-triangle invariant fails."""
    src, dst, n = graphgen.er(60, 420, seed=7)
    lo, hi = oracle.canonical_edges(src, dst, n)
    tri = triangles_of_edges(n, lo, hi)
    bulk_peel(tri, 3, single=False)
    with pytest.raises(AssertionError):
        bulk_peel(tri, 3, single=False, owner_rule=False)


def windowed_peel(tri, window):
    """The decomposition with the device's scan structure: full scans that
    collect the alive list and the window, windowed scans in between.  At
    every scan the frontier found must equal the one a scan of all alive
    edges finds.  Returns the truss numbers."""
    m = len(tri)
    s = [len(t) for t in tri]
    removed = [False] * m
    truss = [0] * m
    k, bound = 3, None
    alive_list = list(range(m))
    win = []
    while not all(removed):
        thr = k - 2
        full = bound is None or thr > bound
        if full:
            bound = thr + window
        scan = alive_list if full else win
        scanned = [e for e in scan if not removed[e]]
        if full:
            alive_list = scanned
        next_win = [e for e in scanned if s[e] < bound]
        frontier = [e for e in scanned if s[e] < thr]
        truth = [e for e in range(m) if not removed[e] and s[e] < thr]
        assert sorted(frontier) == truth, (k, full)
        if not frontier:
            m0 = min(s[e] for e in scanned) if scanned else bound
            if not full:
                m0 = min(m0, bound)   # edges outside the window have s >= bound
            k = max(k + 1, m0 + 3)
            win = next_win
            continue
        while frontier:
            dying = set(frontier)
            lowered = []
            for e in frontier:
                for f, g in tri[e]:
                    if (removed[f] and f not in dying) or (removed[g] and g not in dying):
                        continue
                    if min(x for x in (e, f, g) if x in dying) != e:
                        continue
                    for x in (f, g):
                        if x not in dying and not removed[x]:
                            old = s[x]
                            s[x] -= 1
                            if old == bound:
                                next_win.append(x)   # just fell below the window bound
                            if old == thr:
                                lowered.append(x)    # just fell below the threshold
            for e in frontier:
                removed[e] = True
                truss[e] = k - 1
            frontier = sorted(lowered)
        win = next_win
        k += 1
    return np.array(truss, dtype=np.int32)


@pytest.mark.parametrize("window", [1, 2, 3, 16])
@pytest.mark.parametrize("name,g", list(graphs()), ids=[n for n, _ in graphs()])
def test_windowed_scans_find_every_frontier(name, g, window):
    src, dst, n = g
    og = oracle.OracleGraph.from_edges(src, dst, n)
    lo, hi = oracle.canonical_edges(src, dst, n)
    truss = windowed_peel(triangles_of_edges(n, lo, hi), window)
    assert np.array_equal(truss, og.truss_decomposition()[1]), (name, window)
