"""GPU parity: every C-ABI call against the CPU oracle, bit-exact.

All outputs are integers (int64 triangle counts, int32 supports and truss
numbers, uint8 masks, int32 canonical edge lists), so the bar is equality.
Inputs are seeded synthetic graphs: the paper's examples, closed-form
families, Erdős–Rényi and R-MAT graphs at sizes that span many radix-sort
tiles and compaction chunks with ragged tails, edge lists with self-loops,
repeats and reversed pairs, and the degenerate cases (no edges, one vertex,
a maximum-degree star).
"""
import hashlib
import os

import numpy as np
import pytest

import graphgen
import oracle
from conftest import ROOT, read_fixture

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1708_06866_gb300 as tc  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


PEEL_MODES = {"lists": 1, "intersect": 2, "hybrid": 3}
PEEL_INFO = {"lists": 1, "intersect": 0, "hybrid": 2}   # tc_graph_info's peel_lists


def gpu_all(src, dst, n, ks=(2, 3, 4, 5, 6)):
    """Every ABI call on one graph; the peel runs in each of its forms (all
    triangle lists, intersections, lists only below the support bound)."""
    g = tc.tc_build_csr(dev(src), dev(dst), n)
    lo, hi = tc.tc_edges(g)
    # the edge-per-warp kernel first, the thread-per-edge and the row
    # kernels, then the default (column kernel), whose supports the peel
    # then reuses
    prev = tc.tc_debug_intersect_mode(2)
    try:
        T_warp = tc.tc_count(g)
        s_warp, _ = tc.tc_edge_support(g)
        s_warp = s_warp.cpu().numpy()
        tc.tc_debug_intersect_mode(3)   # the thread-per-edge kernel
        T_thread = tc.tc_count(g)
        s_thread, _ = tc.tc_edge_support(g)
        s_thread = s_thread.cpu().numpy()
        tc.tc_debug_intersect_mode(4)   # the row kernel
        T_rows = tc.tc_count(g)
        s_rows, _ = tc.tc_edge_support(g)
        s_rows = s_rows.cpu().numpy()
        tc.tc_debug_intersect_mode(1)   # the column kernel (forced)
        T_cols = tc.tc_count(g)
        s_cols, _ = tc.tc_edge_support(g)
        s_cols = s_cols.cpu().numpy()
    finally:
        tc.tc_debug_intersect_mode(prev)
    T = tc.tc_count(g)
    s, T2 = tc.tc_edge_support(g)
    out = dict(m=g.m, lo=lo.cpu().numpy(), hi=hi.cpu().numpy(), T=T, T2=T2,
               s=s.cpu().numpy(), peel={}, T_warp=T_warp, s_warp=s_warp, T_thread=T_thread,
               s_thread=s_thread, T_rows=T_rows, s_rows=s_rows, T_cols=T_cols, s_cols=s_cols)
    for name, mode in PEEL_MODES.items():
        prev = tc.tc_debug_peel_mode(mode)
        try:
            masks = {}
            for k in ks:                    # ascending: each call resumes from the last
                mk, c = tc.ktruss(g, k)
                masks[k] = (mk.cpu().numpy(), c)
            for k in sorted(ks, reverse=True):   # descending: fresh peels, same trusses
                mk, c = tc.ktruss(g, k)
                assert c == masks[k][1] and np.array_equal(mk.cpu().numpy(), masks[k][0]), k
            kmax, truss = tc.ktruss_max(g)
            info = tc.tc_graph_info(g)
        finally:
            tc.tc_debug_peel_mode(prev)
        if g.m:
            assert info["peel_lists"] == PEEL_INFO[name], (name, info["peel_lists"])
        out["peel"][name] = dict(masks=masks, kmax=kmax, truss=truss.cpu().numpy())
    tc.tc_graph_free(g)
    return out


def check(src, dst, n, ks=(2, 3, 4, 5, 6)):
    got = gpu_all(src, dst, n, ks)
    og = oracle.OracleGraph.from_edges(src, dst, n)
    assert got["m"] == og.m
    assert np.array_equal(got["lo"], og.lo) and np.array_equal(got["hi"], og.hi)
    T = og.count()
    assert got["T"] == T and got["T2"] == T and got["T_warp"] == T
    assert np.array_equal(got["s"], og.support())
    assert np.array_equal(got["s_warp"], got["s"])
    assert got["T_thread"] == T and np.array_equal(got["s_thread"], got["s"])
    assert got["T_rows"] == T and np.array_equal(got["s_rows"], got["s"])
    assert got["T_cols"] == T and np.array_equal(got["s_cols"], got["s"])
    kmax, truss = og.truss_decomposition()
    for name, res in got["peel"].items():
        for k in ks:
            mask, sup, left = og.ktruss(k)
            gm, gc = res["masks"][k]
            assert np.array_equal(gm, mask), f"{name} k={k}"
            assert gc == left, f"{name} k={k}"
        assert res["kmax"] == kmax, name
        assert np.array_equal(res["truss"], truss), name
    got["masks"] = got["peel"]["lists"]["masks"]
    got["kmax"] = got["peel"]["lists"]["kmax"]
    got["truss"] = got["peel"]["lists"]["truss"]
    return got


def test_fig1_and_fig2_examples():
    fx = read_fixture("fig1_diamond.txt")
    e = np.array(fx["edge"], dtype=np.int32)
    got = check(e[:, 0], e[:, 1], 4)
    assert got["T"] == fx["triangles"][0][0]
    assert got["s"].tolist() == fx["support"][0]
    fx = read_fixture("fig2_pendant.txt")
    e = np.array(fx["edge"], dtype=np.int32)
    got = check(e[:, 0], e[:, 1], 4)
    assert got["masks"][3][0].tolist() == fx["truss3"][0]


@pytest.mark.parametrize("n", [3, 4, 9, 33, 64])
def test_complete_graphs(n):
    s, d, _ = graphgen.complete(n)
    got = check(s, d, n, ks=(2, 3, n, n + 1))
    assert got["kmax"] == n


@pytest.mark.parametrize("M", [2, 3, 16, 100])
def test_image_graphs(M):
    s, d, n = graphgen.king(M)
    got = check(s, d, n)
    assert got["T"] == 4 * (M - 1) ** 2 and got["kmax"] == 4


@pytest.mark.parametrize("maker", [
    lambda: graphgen.star(5000), lambda: graphgen.path(3000),
    lambda: graphgen.random_tree(4000, 1), lambda: graphgen.grid4(40)])
def test_triangle_free(maker):
    s, d, n = maker()
    got = check(s, d, n)
    assert got["T"] == 0 and got["kmax"] == 2


def test_er4096_workload():
    w = graphgen.WORKLOADS["er4096"]
    s, d, n = w.generate()
    check(s, d, n)


@pytest.mark.parametrize("scale,seed", [(6, 1), (9, 2), (12, 3), (14, 4), (16, 5)])
def test_rmat_graphs(scale, seed):
    s, d, n = graphgen.rmat(scale, seed=seed)
    check(s, d, n, ks=(3, 4, 6, 8))


@pytest.mark.parametrize("m_in", [1, 2, 31, 33, 2047, 2049, 4095, 4096, 4097, 3 * 4096 + 5,
                                  70001])
def test_ragged_sizes(m_in):
    rng = np.random.default_rng(m_in)
    n = max(2, int(np.sqrt(m_in) * 3))
    s = rng.integers(0, n, m_in).astype(np.int32)
    d = rng.integers(0, n, m_in).astype(np.int32)
    check(s, d, n)


def test_messy_inputs_clean_to_the_same_graph():
    s, d, n = graphgen.rmat(11, seed=7)
    ms, md = graphgen.messy(s, d, seed=3, loops=500, dup_frac=0.3, flip_frac=0.4)
    a = check(s, d, n)
    b = check(ms, md, n)
    assert np.array_equal(a["lo"], b["lo"]) and np.array_equal(a["s"], b["s"])


def test_star_plus_clique_max_degree():
    # hub adjacent to every vertex plus a dense core: maximum-degree vertex,
    # skewed list lengths in every intersection
    n = 20000
    s = [np.zeros(n - 1, np.int32)]
    d = [np.arange(1, n, dtype=np.int32)]
    cs, cd, _ = graphgen.complete(40)
    s.append(cs + 1)
    d.append(cd + 1)
    es, ed, _ = graphgen.er(n, 30000, seed=2)
    s.append(es)
    d.append(ed)
    check(np.concatenate(s), np.concatenate(d), n, ks=(3, 4, 10, 41, 42))


def test_degenerate_graphs():
    # no edges at all
    g = tc.tc_build_csr(dev(np.zeros(0)), dev(np.zeros(0)), 5)
    assert g.m == 0 and tc.tc_count(g) == 0
    s, T = tc.tc_edge_support(g)
    assert T == 0 and s.numel() == 0
    mask, left = tc.ktruss(g, 3)
    assert left == 0
    assert tc.ktruss_max(g)[0] == 0
    g.free()
    # only self-loops
    g = tc.tc_build_csr(dev([0, 1, 2]), dev([0, 1, 2]), 3)
    assert g.m == 0 and tc.ktruss_max(g)[0] == 0
    g.free()
    # one vertex
    g = tc.tc_build_csr(dev([0]), dev([0]), 1)
    assert g.m == 0 and tc.tc_count(g) == 0
    g.free()
    # single edge
    got = check(np.array([1]), np.array([0]), 2)
    assert got["kmax"] == 2 and got["truss"].tolist() == [2]


def test_host_inputs_and_outputs():
    s, d, n = graphgen.rmat(12, seed=11)
    g = tc.tc_build_csr(s, d, n)            # numpy (host) inputs
    og = oracle.OracleGraph.from_edges(s, d, n)
    out = torch.empty(g.m, dtype=torch.int32)          # host output
    sup, T = tc.tc_edge_support(g, out=out)
    assert sup is out and np.array_equal(out.numpy(), og.support())
    mask = torch.empty(g.m, dtype=torch.uint8)
    tc.ktruss(g, 4, out=mask)
    assert np.array_equal(mask.numpy(), og.ktruss(4)[0])
    truss = torch.empty(g.m, dtype=torch.int32).pin_memory()
    kmax, _ = tc.ktruss_max(g, out=truss)
    assert kmax == og.truss_decomposition()[0]
    assert np.array_equal(truss.numpy(), og.truss_decomposition()[1])
    lo, hi = tc.tc_edges(g, device="cpu")
    assert np.array_equal(lo.numpy(), og.lo)
    g.free()


def test_pinned_host_inputs_and_outputs_are_used_in_place():
    """Pinned host memory is read and written by the kernels themselves (no
    copy pass): a graph built from pinned pairs, with supports, k-truss
    masks and truss numbers written to pinned buffers, equals the oracle;
    pageable buffers of the same call give the same results."""
    s, d, n = graphgen.rmat(13, seed=12)
    og = oracle.OracleGraph.from_edges(s, d, n)
    ps = torch.from_numpy(np.ascontiguousarray(s, np.int32)).pin_memory()
    pd = torch.from_numpy(np.ascontiguousarray(d, np.int32)).pin_memory()
    for g in (tc.tc_build_csr(ps, pd, n), tc.tc_build_csr(s, d, n)):
        assert g.m == og.m
        lo, hi = tc.tc_edges(g, device="cpu")
        assert np.array_equal(lo.numpy(), og.lo) and np.array_equal(hi.numpy(), og.hi)
        sup = torch.full((g.m,), -1, dtype=torch.int32).pin_memory()
        _, T = tc.tc_edge_support(g, out=sup)
        assert T == og.count() and np.array_equal(sup.numpy(), og.support())
        for k in (3, 4, 5):
            mask = torch.full((g.m,), 7, dtype=torch.uint8).pin_memory()
            _, left = tc.ktruss(g, k, out=mask)
            want, _, wleft = og.ktruss(k)
            assert left == wleft and np.array_equal(mask.numpy(), want), k
        truss = torch.full((g.m,), -1, dtype=torch.int32).pin_memory()
        kmax, _ = tc.ktruss_max(g, out=truss)
        wk, wt = og.truss_decomposition()
        assert kmax == wk and np.array_equal(truss.numpy(), wt)
        g.free()


def test_streams():
    s, d, n = graphgen.rmat(13, seed=12)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        g = tc.tc_build_csr(dev(s), dev(d), n, stream=st)
        T = tc.tc_count(g, stream=st)
    assert T == oracle.OracleGraph.from_edges(s, d, n).count()
    g.free()


def test_errors_are_reported_and_leave_the_library_usable():
    with pytest.raises(tc.TCError) as ei:
        tc.tc_build_csr(dev([0, 1, 7]), dev([1, 2, 0]), 5)
    assert ei.value.code == tc.TC_ERANGE
    with pytest.raises(tc.TCError) as ei:
        tc.tc_build_csr(dev([0]), dev([1]), 0)
    assert ei.value.code == tc.TC_EINVAL
    g = tc.tc_build_csr(dev([0, 1, 2]), dev([1, 2, 0]), 3)
    with pytest.raises(tc.TCError) as ei:
        tc.ktruss(g, 1)
    assert ei.value.code == tc.TC_EINVAL
    # host-side fault injection: the 3rd device allocation fails
    tc.tc_debug_fail_alloc(3)
    with pytest.raises(tc.TCError) as ei:
        tc.tc_build_csr(dev([0, 1, 2]), dev([1, 2, 0]), 3)
    assert ei.value.code == tc.TC_ENOMEM
    tc.tc_debug_fail_alloc(0)
    assert tc.tc_count(g) == 1
    g.free()
    g = tc.tc_build_csr(dev([0, 1, 2]), dev([1, 2, 0]), 3)
    assert tc.ktruss_max(g)[0] == 3
    g.free()


# ------------------------------------------------- full-size R-MAT scale 20

def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


def _fixture(name):
    path = os.path.join(ROOT, "tests", "golden", f"{name}_oracle.txt")
    if not os.path.exists(path):
        pytest.skip(f"stored oracle results {path} not present")
    out = {}
    for line in open(path):
        line = line.split("#", 1)[0].split()
        if line:
            out.setdefault(line[0], []).append(line[1:])
    return out


def test_rmat20_full_size_against_stored_oracle():
    """R-MAT scale 20 in the bench's configuration: the whole path against the
    oracle's stored results (hashes of every per-edge array)."""
    fx = _fixture("rmat20")
    w = graphgen.WORKLOADS["rmat20"]
    s, d, n = w.generate()
    g = tc.tc_build_csr(dev(s), dev(d), n)
    assert g.m == int(fx["m"][0][0])
    lo, hi = tc.tc_edges(g)
    assert [_sha(lo.cpu().numpy()), _sha(hi.cpu().numpy())] == fx["lo_hi_sha256"][0]
    T = tc.tc_count(g)
    assert T == int(fx["triangles"][0][0])
    sup, T2 = tc.tc_edge_support(g)
    assert T2 == T
    assert _sha(sup.cpu().numpy()) == fx["support_sha256"][0][0]
    for k, left, h in fx.get("ktruss", []):
        mask, c = tc.ktruss(g, int(k))
        assert c == int(left)
        assert _sha(mask.cpu().numpy().astype(np.int32)) == h
    for mode in PEEL_MODES.values():
        prev = tc.tc_debug_peel_mode(mode)
        try:
            kmax, truss = tc.ktruss_max(g)
        finally:
            tc.tc_debug_peel_mode(prev)
        assert kmax == int(fx["kmax"][0][0])
        assert _sha(truss.cpu().numpy()) == fx["truss_sha256"][0][0]
    g.free()


def test_bounded_wait_expiry_is_reported():
    """A device-side wait that runs out returns TC_ETIMEDOUT and leaves the
    graph and the context usable (the waits are bounded; nothing faults)."""
    s, d, n = graphgen.rmat(12, seed=21)
    g = tc.tc_build_csr(dev(s), dev(d), n)
    og = oracle.OracleGraph.from_edges(s, d, n)
    old = tc.tc_debug_spin_limit_ns(1)
    try:
        with pytest.raises(tc.TCError) as ei:
            tc.ktruss_max(g)
        assert ei.value.code == tc.TC_ETIMEDOUT
    finally:
        tc.tc_debug_spin_limit_ns(old)
    kmax, truss = tc.ktruss_max(g)
    assert kmax == og.truss_decomposition()[0]
    assert np.array_equal(truss.cpu().numpy(), og.truss_decomposition()[1])
    assert tc.tc_graph_info(g)["peel_rounds"] > 0
    g.free()


def test_dense_graph_with_large_out_lists():
    """K_2100: all degrees tie, so out-lists take every size 0..2099 (both
    hash-table regimes, and a table above 48 KB of shared memory); count and
    supports against the closed forms C(n,3) and n-2, and the n-truss."""
    import math
    n = 2100
    s, d, _ = graphgen.complete(n)
    g = tc.tc_build_csr(dev(s), dev(d), n)
    assert tc.tc_graph_info(g)["max_out"] == n - 1
    assert tc.tc_count(g) == math.comb(n, 3)
    sup, T = tc.tc_edge_support(g)
    assert T == math.comb(n, 3)
    assert bool((sup == n - 2).all())
    mask, left = tc.ktruss(g, n)
    assert left == g.m and bool((mask == 1).all())
    g.free()


def test_memory_limit_selects_the_peel_form_and_keeps_results():
    """tc_graph_set_memory_limit bounds the optional memory: with 0 the peel
    runs without triangle lists or cached adjacency; a generous limit lets it
    keep lists; lowering the limit drops what is cached.  Results do not
    change."""
    src, dst, n = graphgen.rmat(12, 16, seed=21)
    og = oracle.OracleGraph.from_edges(src, dst, n)
    ref = {k: og.ktruss(k) for k in (3, 5)}
    g = tc.tc_build_csr(dev(src), dev(dst), n)
    base = tc.tc_graph_info(g)["device_bytes"]
    tc.tc_graph_set_memory_limit(g, 1 << 40)
    for k in (3, 5):
        mk, c = tc.ktruss(g, k)
        assert c == ref[k][2] and np.array_equal(mk.cpu().numpy(), ref[k][0])
    info = tc.tc_graph_info(g)
    assert info["peel_lists"] == 1
    held = info["device_bytes"]
    assert held > base
    tc.tc_graph_set_memory_limit(g, 0)
    for k in (3, 5):
        mk, c = tc.ktruss(g, k)
        assert c == ref[k][2] and np.array_equal(mk.cpu().numpy(), ref[k][0])
    info = tc.tc_graph_info(g)
    assert info["peel_lists"] == 0
    assert info["device_bytes"] < held
    kmax, truss = tc.ktruss_max(g)
    want_kmax, want_truss = og.truss_decomposition()
    assert kmax == want_kmax and np.array_equal(truss.cpu().numpy(), want_truss)
    assert tc.load_library().tc_graph_set_memory_limit(None, 0) == tc.TC_EINVAL
    tc.tc_graph_free(g)


def test_resume_across_forms():
    """A ktruss call resumes from the cached k-truss of an earlier call with
    a smaller k, whichever peel form made it; calls in between (a
    decomposition, a smaller k) leave results unchanged."""
    src, dst, n = graphgen.rmat(11, 16, seed=33)
    og = oracle.OracleGraph.from_edges(src, dst, n)
    want = {k: og.ktruss(k) for k in (3, 4, 5, 6)}
    want_kmax, want_truss = og.truss_decomposition()
    g = tc.tc_build_csr(dev(src), dev(dst), n)

    def check_k(k, mode):
        prev = tc.tc_debug_peel_mode(mode)
        try:
            mk, c = tc.ktruss(g, k)
        finally:
            tc.tc_debug_peel_mode(prev)
        assert c == want[k][2] and np.array_equal(mk.cpu().numpy(), want[k][0]), (k, mode)

    L, X, H = PEEL_MODES["lists"], PEEL_MODES["intersect"], PEEL_MODES["hybrid"]
    check_k(3, H)                             # hybrid, then full lists from its state
    check_k(4, L)
    check_k(3, L)
    prev = tc.tc_debug_peel_mode(L)
    try:
        kmax, truss = tc.ktruss_max(g)        # a decomposition in between
    finally:
        tc.tc_debug_peel_mode(prev)
    assert kmax == want_kmax and np.array_equal(truss.cpu().numpy(), want_truss)
    check_k(4, L)                             # resumes from k = 3
    check_k(5, X)                             # intersection form from the list state
    check_k(6, L)                             # list form from the intersection state
    check_k(4, L)                             # smaller k: fresh
    check_k(6, L)                             # resumes from k = 4
    check_k(4, H)                             # hybrid fresh, then resumed by every form
    check_k(5, H)
    check_k(6, X)
    tc.tc_graph_free(g)


def test_every_intersection_kernel_builds_the_same_lists():
    """The triangle lists of the peel, built by each intersection kernel
    (forced by the test hook, also on a skewed graph where the automatic
    choice would not take it), give the oracle's truss decomposition."""
    src, dst, n = graphgen.rmat(12, 16, seed=5)
    og = oracle.OracleGraph.from_edges(src, dst, n)
    want_kmax, want_truss = og.truss_decomposition()
    for imode in (1, 2, 3, 4):
        for pmode in ("lists", "hybrid"):
            g = tc.tc_build_csr(dev(src), dev(dst), n)
            pi = tc.tc_debug_intersect_mode(imode)
            pp = tc.tc_debug_peel_mode(PEEL_MODES[pmode])
            try:
                kmax, truss = tc.ktruss_max(g)
            finally:
                tc.tc_debug_intersect_mode(pi)
                tc.tc_debug_peel_mode(pp)
            assert kmax == want_kmax and np.array_equal(truss.cpu().numpy(), want_truss), \
                (imode, pmode)
            tc.tc_graph_free(g)


def test_column_list_build_counts_the_words_it_reads():
    """The column kernel's list build reports its algorithmic bytes from a
    count of the out-list words it read.  Building every edge's list reads
    each entry of N+(u) above v at most once per oriented edge (u, v), and
    reads the entry w of every triangle u < v < w, so the count lies between
    T and the column work (Section III-A's masked product by columns)."""
    src, dst, n = graphgen.rmat(14, 16, seed=7)
    og = oracle.OracleGraph.from_edges(src, dst, n)
    T = og.count()
    g = tc.tc_build_csr(dev(src), dev(dst), n)
    tc.tc_graph_wedge_work(g)
    pi = tc.tc_debug_intersect_mode(1)
    pp = tc.tc_debug_peel_mode(PEEL_MODES["lists"])
    try:
        tc.ktruss_max(g)
    finally:
        tc.tc_debug_intersect_mode(pi)
        tc.tc_debug_peel_mode(pp)
    inf = tc.tc_graph_info(g)
    rest = inf["lists_bytes"] - 24 * g.m - 24 * g.n - 16 * 3 * T
    assert rest % 4 == 0
    words = rest // 4
    assert T <= words <= inf["column_work"], (T, words, inf["column_work"])
    tc.tc_graph_free(g)


def test_from_a_tab_separated_file(tmp_path):
    """The Graph Challenge's input path: a 1-based tab-separated file with
    both directions of every edge and unit weights (Section II), read by
    tc_read_edges and built on the device: the 16 x 16 image graph gives
    Table II's edge count and the closed-form triangles."""
    M = 16
    s, d, n = graphgen.king(M)
    rows = np.concatenate([np.stack([s, d], 1), np.stack([d, s], 1)]) + 1
    path = tmp_path / "king16.tsv"
    path.write_text("".join(f"{u}\t{v}\t1\n" for u, v in rows.tolist()))
    src, dst, n2 = tc.tc_read_edges(str(path))
    assert n2 == n and len(src) == 2 * len(s)
    g = tc.tc_build_csr(dev(src), dev(dst), n2)
    assert g.m == (M - 1) * (4 * M - 2)
    assert tc.tc_count(g) == 4 * (M - 1) ** 2
    kmax, _ = tc.ktruss_max(g)
    assert kmax == 4
    tc.tc_graph_free(g)


def disjoint_union(parts):
    """Vertex-disjoint union of (src, dst, n) graphs, vertex ids shifted."""
    s_all, d_all, base = [], [], 0
    for s, d, n in parts:
        s_all.append(np.asarray(s, dtype=np.int64) + base)
        d_all.append(np.asarray(d, dtype=np.int64) + base)
        base += n
    return (np.concatenate(s_all).astype(np.int32), np.concatenate(d_all).astype(np.int32), base)


@pytest.mark.parametrize("case", ["cliques", "union", "rmat", "king", "er"])
def test_ktruss_components_against_oracle(case):
    """Connected trusses: every edge's and vertex's component label (its
    smallest vertex id) and the component count equal the oracle's, for k
    from 2 past kmax, with device and host outputs."""
    from test_oracle_pins import two_cliques_and_a_bridge
    if case == "cliques":
        src, dst, n = two_cliques_and_a_bridge()
    elif case == "union":
        src, dst, n = disjoint_union([graphgen.complete(6), graphgen.king(5),
                                      graphgen.rmat(8, seed=3), graphgen.complete(4),
                                      graphgen.star(9)])
    elif case == "rmat":
        src, dst, n = graphgen.rmat(12, seed=9)
    elif case == "king":
        src, dst, n = graphgen.king(33)
    else:
        src, dst, n = graphgen.er(3000, 30000, seed=4)
    og = oracle.OracleGraph.from_edges(src, dst, n)
    kmax, _ = og.truss_decomposition()
    g = tc.tc_build_csr(dev(src), dev(dst), n)
    for k in range(2, kmax + 2):
        wel, wvl, wc = og.ktruss_components(k)
        el, vl, c = tc.ktruss_components(g, k)
        assert c == wc, k
        assert np.array_equal(el.cpu().numpy(), wel), k
        assert np.array_equal(vl.cpu().numpy(), wvl), k
    # host outputs through the ABI
    k = max(3, kmax)
    wel, wvl, wc = og.ktruss_components(k)
    hel = np.empty(g.m, dtype=np.int32)
    hvl = np.empty(n, dtype=np.int32)
    import ctypes
    cnt = ctypes.c_int64()
    rc = tc.load_library().ktruss_components(g.handle, k, hel.ctypes.data, hvl.ctypes.data,
                                             ctypes.byref(cnt), None)
    assert rc == tc.TC_OK and cnt.value == wc
    assert np.array_equal(hel, wel) and np.array_equal(hvl, wvl)
    with pytest.raises(tc.TCError):
        tc.ktruss_components(g, 1)
    tc.tc_graph_free(g)


def test_ktruss_components_without_edges():
    g = tc.tc_build_csr(dev(np.array([2], np.int32)), dev(np.array([2], np.int32)), 5)
    el, vl, c = tc.ktruss_components(g, 3)
    assert c == 0 and len(el) == 0 and (vl.cpu().numpy() == -1).all()
    tc.tc_graph_free(g)


def test_support_without_count_then_peel_and_count():
    """tc_edge_support without triangles_out (asynchronous) leaves T unknown;
    a later peel and tc_count must still size and report everything from the
    true T, and repeated calls reuse the graph's supports."""
    src, dst, n = graphgen.rmat(11, seed=13)
    og = oracle.OracleGraph.from_edges(src, dst, n)
    g = tc.tc_build_csr(dev(src), dev(dst), n)
    s1, none = tc.tc_edge_support(g, triangles=False)
    assert none is None
    assert np.array_equal(s1.cpu().numpy(), og.support())
    for name, mode in PEEL_MODES.items():
        prev = tc.tc_debug_peel_mode(mode)
        try:
            kmax, truss = tc.ktruss_max(g)
        finally:
            tc.tc_debug_peel_mode(prev)
        want_kmax, want_truss = og.truss_decomposition()
        assert kmax == want_kmax and np.array_equal(truss.cpu().numpy(), want_truss), name
    assert tc.tc_count(g) == og.count()
    s2, T2 = tc.tc_edge_support(g)
    assert T2 == og.count() and np.array_equal(s2.cpu().numpy(), og.support())
    tc.tc_graph_free(g)
    # count first, then support: the support call knows T already
    g = tc.tc_build_csr(dev(src), dev(dst), n)
    assert tc.tc_count(g) == og.count()
    s3, T3 = tc.tc_edge_support(g)
    assert T3 == og.count() and np.array_equal(s3.cpu().numpy(), og.support())
    tc.tc_graph_free(g)


def test_kept_decomposition_answers_ktruss():
    """After ktruss_max the graph keeps its truss numbers; ktruss(k) for any
    k, ktruss_components and a second ktruss_max are answered from them and
    equal the oracle's peel."""
    src, dst, n = graphgen.rmat(12, seed=17)
    og = oracle.OracleGraph.from_edges(src, dst, n)
    want_kmax, want_truss = og.truss_decomposition()
    g = tc.tc_build_csr(dev(src), dev(dst), n)
    assert tc.tc_graph_info(g)["truss_cached"] == 0
    kmax, truss = tc.ktruss_max(g)
    assert kmax == want_kmax and np.array_equal(truss.cpu().numpy(), want_truss)
    assert tc.tc_graph_info(g)["truss_cached"] == 1
    for k in range(2, want_kmax + 2):
        mask, sup, left = og.ktruss(k)
        mk, c = tc.ktruss(g, k)
        assert c == left and np.array_equal(mk.cpu().numpy(), mask), k
        el, vl, cc = tc.ktruss_components(g, k)
        wel, wvl, wc = og.ktruss_components(k)
        assert cc == wc and np.array_equal(el.cpu().numpy(), wel), k
    kmax2, truss2 = tc.ktruss_max(g)
    assert kmax2 == want_kmax and np.array_equal(truss2.cpu().numpy(), want_truss)
    # a zero memory bound leaves nothing kept on a fresh graph
    g2 = tc.tc_build_csr(dev(src), dev(dst), n)
    tc.tc_graph_set_memory_limit(g2, 0)
    tc.ktruss_max(g2)
    assert tc.tc_graph_info(g2)["truss_cached"] == 0
    tc.tc_graph_free(g2)
    tc.tc_graph_free(g)


def test_memory_bound_counts_everything_kept_together():
    """With a bound that holds the triangle lists but not the lists and the
    truss numbers together, ktruss_max keeps the lists and not the truss
    numbers; results are unchanged and what the graph keeps stays within
    the bound."""
    src, dst, n = graphgen.rmat(11, seed=23)
    og = oracle.OracleGraph.from_edges(src, dst, n)
    want_kmax, want_truss = og.truss_decomposition()
    g = tc.tc_build_csr(dev(src), dev(dst), n)
    T = tc.tc_count(g)
    m = g.m
    lists = 24 * T + 8 * (m + 1)
    tc.tc_graph_set_memory_limit(g, lists + 2 * m)      # room for lists, not 4 B per edge more
    base = tc.tc_graph_info(g)["device_bytes"]
    kmax, truss = tc.ktruss_max(g)
    info = tc.tc_graph_info(g)
    assert kmax == want_kmax and np.array_equal(truss.cpu().numpy(), want_truss)
    assert info["peel_lists"] == 1 and info["truss_cached"] == 0
    # lowering the bound releases the lists at the next call
    tc.tc_graph_set_memory_limit(g, 4 * m)
    kmax, truss = tc.ktruss_max(g)
    info2 = tc.tc_graph_info(g)
    assert kmax == want_kmax and np.array_equal(truss.cpu().numpy(), want_truss)
    assert info2["peel_lists"] == 0 and info2["truss_cached"] == 1
    assert info2["device_bytes"] < info["device_bytes"]
    tc.tc_graph_free(g)


@pytest.mark.parametrize("case", ["rmat", "er", "king", "complete"])
def test_ktruss_sizes_against_oracle(case):
    """The sizes of the k-trusses for a range of k (one peel over levels
    k_lo..k_hi) equal the oracle's decomposition levels, in every peel form,
    with results not kept (a peel per call) and from kept truss numbers."""
    if case == "rmat":
        s, d, n = graphgen.rmat(12, seed=41)
    elif case == "er":
        s, d, n = graphgen.er(2000, 16000, seed=42)
    elif case == "king":
        s, d, n = graphgen.king(40)
    else:
        s, d, n = graphgen.complete(30)
    og = oracle.OracleGraph.from_edges(s, d, n)
    want = [og.m] + og.truss_levels(12)          # k = 2 .. 12
    g = tc.tc_build_csr(dev(s), dev(d), n)
    tc.tc_graph_set_result_cache(g, False)
    for mode in PEEL_MODES.values():
        prev = tc.tc_debug_peel_mode(mode)
        try:
            assert tc.ktruss_sizes(g, 2, 12) == want, mode
            assert tc.ktruss_sizes(g, 5, 7) == want[3:6], mode
            assert tc.ktruss_sizes(g, 9, 9) == [want[7]], mode
        finally:
            tc.tc_debug_peel_mode(prev)
    tc.tc_graph_set_result_cache(g, True)
    tc.ktruss_max(g)                              # kept truss numbers answer now
    assert tc.tc_graph_info(g)["truss_cached"] == 1
    assert tc.ktruss_sizes(g, 2, 12) == want
    assert tc.ktruss_sizes(g, 4, 10) == want[2:9]
    for bad in ((1, 5), (3, 2), (3, 67)):
        with pytest.raises(tc.TCError) as ei:
            tc.ktruss_sizes(g, *bad)
        assert ei.value.code == tc.TC_EINVAL
    tc.tc_graph_free(g)
