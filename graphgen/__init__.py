"""Seeded synthetic graph inputs shared by the tests, the oracle and the bench.

This module generates raw edge lists only (int32 ``src``/``dst`` arrays with
0-based vertex ids).  It performs none of the method's arithmetic: lists may
hold self-loops, repeated pairs and both directions of a pair, and cleaning
them (Section II of the paper) is left to the code under test.

Families:
  * R-MAT / Graph500-style Kronecker graphs with a seeded vertex permutation
    (Section II names Graph500 among the synthetic sources);
  * Erdős–Rényi G(n, m);
  * the paper's 8-neighbour "image" graphs (Section IV-C, Table II);
  * small closed-form families (complete graphs, stars, paths, trees, grids).

The random streams are SplitMix64 in counter mode, implemented in
``graphgen.c`` and compiled on first use with the host C compiler.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "_graphgen.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile graphgen.c into an in-tree shared library; returns its path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int, i32p, i32p]
            lib.gg_rmat_n.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                      ctypes.c_int, i32p, i32p]
            lib.gg_er.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, i32p, i32p]
            lib.gg_permutation.argtypes = [ctypes.c_int32, ctypes.c_uint64, i32p]
            lib.gg_king.argtypes = [ctypes.c_int32, i32p, i32p]
            vp = ctypes.c_void_p
            lib.gg_batch.argtypes = [ctypes.c_int32, vp, vp, vp, vp, ctypes.c_uint64,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, i32p, i32p]
            lib.gg_batch.restype = ctypes.c_int
            for f in (lib.gg_rmat, lib.gg_rmat_n, lib.gg_er):
                f.restype = ctypes.c_int
            lib.gg_permutation.restype = None
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def permutation(n: int, seed: int) -> np.ndarray:
    """Seeded Fisher–Yates permutation of range(n)."""
    perm = np.empty(n, dtype=np.int32)
    _load().gg_permutation(n, seed, _p(perm))
    return perm


def rmat(scale: int, edgefactor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 0, permute: bool = True):
    """R-MAT on n = 2**scale vertices with edgefactor * n draws.

    Returns (src, dst, n).  Each draw descends ``scale`` levels of the
    adjacency matrix, choosing a quadrant with probabilities (a, b, c, d).
    """
    n = 1 << scale
    m = edgefactor * n
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    rc = _load().gg_rmat(scale, m, a, b, c, seed, int(permute), _p(src), _p(dst))
    if rc != 0:
        raise ValueError(f"gg_rmat failed ({rc})")
    return src, dst, n


def rmat_n(n: int, edgefactor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
           seed: int = 0, permute: bool = True):
    """R-MAT on an arbitrary n (draws with an endpoint >= n are rejected)."""
    m = edgefactor * n
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    rc = _load().gg_rmat_n(n, m, a, b, c, seed, int(permute), _p(src), _p(dst))
    if rc != 0:
        raise ValueError(f"gg_rmat_n failed ({rc})")
    return src, dst, n


def er(n: int, m: int, seed: int = 0):
    """Erdős–Rényi G(n, m): m distinct pairs without loops; returns (src, dst, n)."""
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    rc = _load().gg_er(n, m, seed, _p(src), _p(dst))
    if rc != 0:
        raise ValueError(f"gg_er failed ({rc})")
    return src, dst, n


def king(M: int):
    """The paper's M x M image graph: each pixel joined to its 8 neighbours.

    Vertex id = row * M + col.  Each undirected edge is emitted once, so the
    list has (M - 1)(4M - 2) entries (Table II's edge column).
    """
    m = (M - 1) * (4 * M - 2)
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    if _load().gg_king(M, _p(src), _p(dst)) != 0:
        raise ValueError(f"gg_king failed for M={M}")
    return src, dst, M * M


def complete(n: int):
    """K_n, each pair once."""
    iu, ju = np.triu_indices(n, 1)
    return iu.astype(np.int32), ju.astype(np.int32), n


def star(n: int):
    """K_{1,n-1}: vertex 0 joined to every other vertex."""
    return np.zeros(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32), n


def path(n: int):
    return np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32), n


def random_tree(n: int, seed: int = 0):
    """Random recursive tree: vertex i > 0 attaches to a uniform earlier vertex."""
    rng = np.random.default_rng(seed)
    parent = np.array([rng.integers(0, i) for i in range(1, n)], dtype=np.int32)
    return parent, np.arange(1, n, dtype=np.int32), n


def grid4(M: int):
    """M x M grid with 4-neighbour edges (bipartite, so triangle-free)."""
    r, c = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    r = r.ravel()
    c = c.ravel()
    src, dst = [], []
    for dr, dc in ((0, 1), (1, 0)):
        ok = (r + dr < M) & (c + dc < M)
        src.append(r[ok] * M + c[ok])
        dst.append((r[ok] + dr) * M + (c[ok] + dc))
    return (np.concatenate(src).astype(np.int32), np.concatenate(dst).astype(np.int32), M * M)


def messy(src: np.ndarray, dst: np.ndarray, seed: int = 0, loops: int = 0,
          dup_frac: float = 0.0, flip_frac: float = 0.0):
    """Add self-loops, repeated pairs and reversed copies to a list, then shuffle.

    Used to exercise the cleaning rules of Section II (drop loops, one
    undirected edge per pair).
    """
    rng = np.random.default_rng(seed)
    n_nodes = int(max(src.max(initial=-1), dst.max(initial=-1))) + 1
    parts_s, parts_d = [src], [dst]
    k = len(src)
    if loops and n_nodes > 0:
        v = rng.integers(0, n_nodes, loops).astype(np.int32)
        parts_s.append(v)
        parts_d.append(v)
    if dup_frac and k:
        i = rng.integers(0, k, int(dup_frac * k))
        parts_s.append(src[i])
        parts_d.append(dst[i])
    if flip_frac and k:
        i = rng.integers(0, k, int(flip_frac * k))
        parts_s.append(dst[i])
        parts_d.append(src[i])
    s = np.concatenate(parts_s).astype(np.int32)
    d = np.concatenate(parts_d).astype(np.int32)
    order = rng.permutation(len(s))
    return s[order], d[order]


def batch(num_graphs: int = 10_000, seed: int = 3, n_min: int = 64, n_max: int = 65_536,
          er_degree=(8.0, 32.0), edgefactor: int = 16, a: float = 0.57, b: float = 0.19,
          c: float = 0.19):
    """Many independent graphs: n log-uniform in [n_min, n_max]; even-indexed
    graphs Erdős–Rényi with average degree uniform in er_degree, odd-indexed
    R-MAT with edgefactor * n draws (endpoints >= n rejected), permuted.

    Returns (n, edge_off, src, dst, kind): per-graph vertex counts, offsets
    into the concatenated pair lists (ids local to each graph), the kinds.
    """
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(n_min), np.log(n_max), num_graphs)).round().astype(np.int64)
    n = np.clip(n, n_min, n_max)
    kind = (np.arange(num_graphs) % 2).astype(np.int32)
    deg = rng.uniform(er_degree[0], er_degree[1], num_graphs)
    m = np.where(kind == 0, np.round(n * deg / 2.0), edgefactor * n).astype(np.int64)
    m = np.where(kind == 0, np.minimum(m, (n * (n - 1)) // 4), m)   # ER: at most half the pairs
    off = np.zeros(num_graphs + 1, dtype=np.int64)
    np.cumsum(m, out=off[1:])
    src = np.empty(off[-1], dtype=np.int32)
    dst = np.empty(off[-1], dtype=np.int32)
    n32 = np.ascontiguousarray(n, dtype=np.int32)
    rc = _load().gg_batch(num_graphs, kind.ctypes.data, n32.ctypes.data, m.ctypes.data,
                          off.ctypes.data, seed, a, b, c, _p(src), _p(dst))
    if rc != 0:
        raise ValueError("gg_batch failed")
    return n32, off, src, dst, kind


def rmat_pool(num_graphs: int = 64, seed: int = 4, n_min: int = 1 << 10, n_max: int = 1 << 22,
              edgefactor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19):
    """A pool of R-MAT graphs for serving: n log-uniform in [n_min, n_max],
    edgefactor * n draws each (endpoints >= n rejected), permuted.

    Returns {graph id: (src, dst, n)} (views into two concatenated arrays).
    """
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(n_min), np.log(n_max), num_graphs)).round().astype(np.int64)
    n = np.clip(n, n_min, n_max)
    m = edgefactor * n
    off = np.zeros(num_graphs + 1, dtype=np.int64)
    np.cumsum(m, out=off[1:])
    src = np.empty(off[-1], dtype=np.int32)
    dst = np.empty(off[-1], dtype=np.int32)
    kind = np.ones(num_graphs, dtype=np.int32)
    n32 = np.ascontiguousarray(n, dtype=np.int32)
    rc = _load().gg_batch(num_graphs, kind.ctypes.data, n32.ctypes.data, m.ctypes.data,
                          off.ctypes.data, seed, a, b, c, _p(src), _p(dst))
    if rc != 0:
        raise ValueError("gg_batch failed")
    return {g: (src[off[g]:off[g + 1]], dst[off[g]:off[g + 1]], int(n[g]))
            for g in range(num_graphs)}


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named synthetic workload: generator family, sizes and seed."""
    name: str
    family: str
    n: int
    seed: int
    scale: int = 0
    edgefactor: int = 16
    m: int = 0
    a: float = 0.57
    b: float = 0.19
    c: float = 0.19
    truss_ks: tuple = ()       # () means the full decomposition k = 3..kmax
    description: str = ""

    def generate(self):
        if self.family == "er":
            return er(self.n, self.m, self.seed)
        if self.family == "rmat":
            return rmat(self.scale, self.edgefactor, self.a, self.b, self.c, self.seed, True)
        if self.family == "king":
            return king(self.scale)
        raise ValueError(self.family)


WORKLOADS = {
    "er4096": Workload(
        "er4096", "er", n=4096, m=32768, seed=0,
        description="Erdős–Rényi G(n=4096, m=32768), avg degree 16; count + per-edge support"),
    "rmat20": Workload(
        "rmat20", "rmat", n=1 << 20, scale=20, seed=1,
        description="R-MAT scale 20, edgefactor 16, a/b/c/d=.57/.19/.19/.05, permuted; "
                    "count + support + full truss decomposition k=3..kmax"),
    "rmat18": Workload(
        "rmat18", "rmat", n=1 << 18, scale=18, seed=1,
        description="R-MAT scale 18, edgefactor 16, permuted; count + support + full truss "
                    "decomposition (the small case for hardware-counter captures)"),
    "rmat22": Workload(
        "rmat22", "rmat", n=1 << 22, scale=22, seed=1, truss_ks=(3, 4, 6, 8),
        description="R-MAT scale 22, edgefactor 16, permuted; count + support + k-truss at "
                    "k=3,4,6,8 (3T >= 2^32, so the scale-24 path at a quarter of its size: the "
                    "small case for hardware-counter captures of that path)"),
    "king8192": Workload(
        "king8192", "king", n=8192 * 8192, scale=8192, seed=0,
        description="the 8192 x 8192 8-neighbour image graph (Section IV-C, Table II's family): "
                    "268M edges, T = 4(M-1)^2; count + support + full truss decomposition"),
    "rmat24": Workload(
        "rmat24", "rmat", n=1 << 24, scale=24, seed=2, truss_ks=(3, 4, 6, 8),
        description="R-MAT scale 24, edgefactor 16 (268M draws), permuted; "
                    "count + support + k-truss at k=3,4,6,8"),
}
