"""The seeded input generators: deterministic, in range, right sizes."""
import numpy as np

import graphgen


def test_rmat_deterministic_and_in_range():
    a = graphgen.rmat(12, seed=3)
    b = graphgen.rmat(12, seed=3)
    c = graphgen.rmat(12, seed=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    s, d, n = a
    assert n == 4096 and len(s) == 16 * 4096
    assert s.min() >= 0 and s.max() < n and d.min() >= 0 and d.max() < n


def test_rmat_quadrant_skew():
    # without the permutation, the top bit of src is 1 with probability c + d = 0.24
    s, d, n = graphgen.rmat(16, seed=1, permute=False)
    top_src = (s >> 15) & 1
    top_dst = (d >> 15) & 1
    assert abs(top_src.mean() - 0.24) < 0.01
    assert abs(top_dst.mean() - 0.24) < 0.01   # b + d


def test_permutation_is_a_permutation():
    p = graphgen.permutation(1000, 7)
    assert np.array_equal(np.sort(p), np.arange(1000))
    assert not np.array_equal(p, np.arange(1000))


def test_rmat_n_respects_bound():
    s, d, n = graphgen.rmat_n(1000, 8, seed=2)
    assert len(s) == 8000 and s.max() < 1000 and d.max() < 1000


def test_er_simple_graph():
    s, d, n = graphgen.er(4096, 32768, seed=0)
    assert len(s) == 32768
    assert (s != d).all()
    key = np.minimum(s, d).astype(np.int64) << 32 | np.maximum(s, d)
    assert len(np.unique(key)) == 32768


def test_king_sizes():
    for M in (2, 5, 16):
        s, d, n = graphgen.king(M)
        assert n == M * M and len(s) == (M - 1) * (4 * M - 2)


def test_workload_table():
    assert graphgen.WORKLOADS["rmat24"].truss_ks == (3, 4, 6, 8)
    assert graphgen.WORKLOADS["er4096"].m == 32768
