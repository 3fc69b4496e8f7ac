"""Full-size workloads in the bench's launch configuration.

The 8192 x 8192 image graph (268M edges) is checked in full against the
closed forms of Section IV-C.  R-MAT scale 24 (268M generated pairs) is
checked in full against the oracle's stored results: SHA-256 hashes of the
canonical edge list, of every per-edge support and of each k-truss mask
(k = 3, 4, 6, 8), written once by tests/golden/make_oracle_fixtures.py (the
oracle's serial peel takes over an hour at this size).
"""
import hashlib
import os

import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1708_06866_gb300 as tc  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


def _fixture(name):
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", f"{name}_oracle.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                out.setdefault(line[0], []).append(line[1:])
    return out


def test_rmat24_full_size_against_stored_oracle():
    """The bench's scale-24 sequence (count, supports, then ktruss at
    k = 3, 4, 6, 8, each call resuming from the previous truss, in the
    automatic form: triangle lists for the edges of support below the bound,
    intersections for the rest) equals the oracle bit for bit; so do fresh
    peels in the intersection form and in the bounded-list form."""
    fx = _fixture("rmat24")
    w = graphgen.WORKLOADS["rmat24"]
    s, d, n = w.generate()
    g = tc.tc_build_csr(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
    del s, d
    assert g.m == int(fx["m"][0][0])
    lo, hi = tc.tc_edges(g)
    assert [_sha(lo.cpu().numpy()), _sha(hi.cpu().numpy())] == fx["lo_hi_sha256"][0]
    del lo, hi
    T = tc.tc_count(g)
    assert T == int(fx["triangles"][0][0])
    sup, T2 = tc.tc_edge_support(g)
    assert T2 == T
    assert int(sup.sum(dtype=torch.int64)) == int(fx["support_sum"][0][0])
    assert _sha(sup.cpu().numpy()) == fx["support_sha256"][0][0]
    del sup
    want = {int(k): (int(left), h) for k, left, h in fx["ktruss"]}
    assert sorted(want) == list(w.truss_ks)
    for k in w.truss_ks:                      # as the bench calls them
        mask, c = tc.ktruss(g, k)
        assert (c, _sha(mask.cpu().numpy().astype(np.int32))) == want[k], k
    for mode in (2, 3):                       # intersections; bounded lists
        prev = tc.tc_debug_peel_mode(mode)
        try:
            for k in (8, 4):                  # descending: each a fresh peel
                mask, c = tc.ktruss(g, k)
                assert (c, _sha(mask.cpu().numpy().astype(np.int32))) == want[k], (mode, k)
        finally:
            tc.tc_debug_peel_mode(prev)
    g.free()


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
