"""The oracle's pins catch plausible mistakes.

Each case compiles a copy of tc_oracle.c with one planted mistake (a wrong
comparison, a dropped term, a wrong index, a missing guard) into a temporary
directory and checks that at least one pin from test_oracle_pins fails on it.
Mistakes are planted in the oracle, on the CPU; the GPU library is not
involved.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import graphgen
import oracle
from conftest import ROOT
from test_oracle_pins import (brute_support, brute_triangles, closure_components, dense_adj,
                              king_support, literal_algorithm4, small_random_graphs,
                              two_cliques_and_a_bridge)

SRC = os.path.join(ROOT, "oracle", "tc_oracle.c")

MUTANTS = [
    ("count keeps w > a instead of w > b",
     "if (g->nbr[pa[i]] > b) ++total;", "if (g->nbr[pa[i]] > a) ++total;"),
    ("merge advances the wrong list",
     "else if (g->nbr[i] > g->nbr[j]) ++j;", "else if (g->nbr[i] > g->nbr[j]) ++i;"),
    ("binary search overshoots equal keys",
     "if (g->nbr[mid] < w) lo = mid + 1;", "if (g->nbr[mid] <= w) lo = mid + 1;"),
    ("peel threshold <= instead of <",
     "if (s[e] < k - 2 && !queued[e]) {", "if (s[e] <= k - 2 && !queued[e]) {"),
    ("destroyed triangle decremented again",
     "if (!alive[f] || !alive[h]) continue; /* triangle already destroyed */", ""),
    ("one of the two surviving edges not decremented",
     "            --s[h];\n", ""),
    ("truss number off by one",
     "if (level) level[e] = k - 1;", "if (level) level[e] = k;"),
    ("components ignore the edge subset",
     "if (alive[g->eid[p]] && lab[y] < 0) {", "if (lab[y] < 0) {"),
    ("component start vertex labelled apart from the rest",
     "lab[v] = v;\n        stack[top++] = v;", "lab[v] = v + 1;\n        stack[top++] = v;"),
    ("adjacency drops the reverse direction",
     "tmp[g->off[b] + fill[b]++] = (nbr_entry){a, (int32_t)e};",
     "tmp[g->off[b] + fill[b]++] = (nbr_entry){b, (int32_t)e};"),
]


def pins_fail(lib) -> bool:
    """True if any of a compact set of pins fails (or the library misbehaves)."""
    try:
        for n, lo, hi in small_random_graphs(25, 30, seed=11):
            g = oracle.OracleGraph(n, lo, hi, lib=lib)
            tris = brute_triangles(n, dense_adj(n, lo, hi))
            if g.count() != len(tris):
                return True
            if not np.array_equal(g.support(), brute_support(lo, hi, tris)):
                return True
            if len(lo) and len(lo) < 120:
                for k in (3, 4, 5):
                    mref, sref = literal_algorithm4(n, lo, hi, k)
                    mask, sup, _ = g.ktruss(k)
                    if not (np.array_equal(mask, mref) and np.array_equal(sup, sref)):
                        return True
        for n, lo, hi in small_random_graphs(10, 20, seed=12):
            g = oracle.OracleGraph(n, lo, hi, lib=lib)
            mk = g.ktruss(3)[0]
            got = g.components(mk)
            want = closure_components(n, lo, hi, mk)
            if got[2] != want[2] or not (np.array_equal(got[0], want[0])
                                         and np.array_equal(got[1], want[1])):
                return True
        s, d, n = two_cliques_and_a_bridge()
        g = oracle.OracleGraph.from_edges(s, d, n, lib=lib)
        if g.ktruss_components(5)[2] != 2:
            return True
        for M in (4, 9):
            s, d, n = graphgen.king(M)
            g = oracle.OracleGraph.from_edges(s, d, n, lib=lib)
            if g.count() != 4 * (M - 1) ** 2:
                return True
            if not np.array_equal(g.support(), king_support(M, g.lo, g.hi)):
                return True
            kmax, t = g.truss_decomposition()
            if kmax != 4 or not (t == 4).all():
                return True
        s, d, n = graphgen.rmat(9, seed=2)
        g = oracle.OracleGraph.from_edges(s, d, n, lib=lib)
        kmax, t = g.truss_decomposition()
        for k in range(3, kmax + 2):
            mask, sup, _ = g.ktruss(k)
            if not np.array_equal(mask.astype(bool), t >= k):
                return True
            if (sup[mask == 1] < k - 2).any():
                return True
    except (ValueError, OSError):
        return True
    return False


def test_unmodified_oracle_passes_the_compact_pins():
    assert not pins_fail(oracle.load())


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, desc, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site not unique: {desc}"
    path = tmp_path / "mutant.c"
    path.write_text(text.replace(old, new))
    so = str(tmp_path / "mutant.so")
    subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11", str(path), "-o",
                    so], check=True)
    assert pins_fail(oracle.load(so)), desc
