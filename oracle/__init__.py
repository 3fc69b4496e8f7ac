"""CPU oracle for triangle counting, edge support and k-truss (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg are the only callers.  The GPU library never imports
this package and shares no code with it.

Two parts:
  * :func:`canonical_edges` applies the cleaning rules of Section II of the
    paper (vertex ids in [0, n), self-loops dropped, one undirected edge per
    pair, unit weights) with numpy's sort as the sorting step and adjacent-repeat removal, giving
    the canonical edge list: pairs (lo, hi), lo < hi, in lexicographic order.
    An edge's position in this list is its id in every per-edge output.
  * :class:`OracleGraph` wraps ``tc_oracle.c``: serial (OpenMP over edges for
    the independent per-edge loops) statements of the triangle count, the
    per-edge support |N(a) ∩ N(b)| and the k-truss peel of Section III.

Parity status of each function is recorded with its pins in the test suite;
every function here is pinned (brute force, closed forms, the paper's
Table II and Fig. 1, a literal Algorithm 4 and a float64 trace(A^3)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_tc_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile tc_oracle.c into a shared library next to it; returns its path."""
    if (not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", src, "-o", tmp],
                   check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    vp = ctypes.c_void_p
    lib.oracle_open.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p,
                                ctypes.POINTER(ctypes.c_int)]
    lib.oracle_open.restype = vp
    lib.oracle_free.argtypes = [vp]
    lib.oracle_free.restype = None
    lib.oracle_count.argtypes = [vp]
    lib.oracle_count.restype = ctypes.c_int64
    lib.oracle_support.argtypes = [vp, i32p]
    lib.oracle_support.restype = None
    lib.oracle_support_of.argtypes = [vp, i64p, ctypes.c_int64, i32p]
    lib.oracle_support_of.restype = None
    lib.oracle_support_within.argtypes = [vp, u8p, i32p]
    lib.oracle_support_within.restype = None
    lib.oracle_support_within_of.argtypes = [vp, u8p, i64p, ctypes.c_int64, i32p]
    lib.oracle_support_within_of.restype = None
    lib.oracle_ktruss.argtypes = [vp, ctypes.c_int32, u8p, i32p]
    lib.oracle_ktruss.restype = ctypes.c_int64
    lib.oracle_truss_decomposition.argtypes = [vp, i32p]
    lib.oracle_truss_decomposition.restype = ctypes.c_int32
    lib.oracle_truss_components.argtypes = [vp, u8p, i32p, i32p]
    lib.oracle_truss_components.restype = ctypes.c_int64
    lib.oracle_truss_levels.argtypes = [vp, ctypes.c_int32, i64p]
    lib.oracle_truss_levels.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library; ``path`` loads another build."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def canonical_edges(src, dst, n: int):
    """Cleaning of Section II: returns (lo, hi) int32 arrays, lo < hi, sorted, unique.

    Raises ValueError if any id lies outside [0, n).
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    if n < 0:
        raise ValueError("n < 0")
    if len(src) and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("vertex id out of range")
    keep = src != dst
    lo = np.minimum(src[keep], dst[keep])
    hi = np.maximum(src[keep], dst[keep])
    key = np.sort((lo << 32) | hi)
    if len(key):
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    return (key >> 32).astype(np.int32), (key & 0xFFFFFFFF).astype(np.int32)


class OracleGraph:
    """A canonical edge list with the oracle's adjacency lists built."""

    def __init__(self, n: int, lo, hi, lib=None):
        self._lib = lib if lib is not None else load()
        self.n = int(n)
        self.lo = np.ascontiguousarray(lo, dtype=np.int32)
        self.hi = np.ascontiguousarray(hi, dtype=np.int32)
        self.m = len(self.lo)
        err = ctypes.c_int(0)
        self._h = self._lib.oracle_open(self.n, self.m, _ptr(self.lo, ctypes.c_int32),
                                        _ptr(self.hi, ctypes.c_int32), ctypes.byref(err))
        if not self._h:
            raise ValueError(f"not a canonical edge list (code {err.value})")

    @classmethod
    def from_edges(cls, src, dst, n: int, lib=None) -> "OracleGraph":
        lo, hi = canonical_edges(src, dst, n)
        return cls(n, lo, hi, lib=lib)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def count(self) -> int:
        """Number of triangles (Section III-A)."""
        return int(self._lib.oracle_count(self._h))

    def support(self) -> np.ndarray:
        """int32 support of every edge, canonical order (Algorithm 4, s = (R == 2) 1)."""
        s = np.empty(self.m, dtype=np.int32)
        self._lib.oracle_support(self._h, _ptr(s, ctypes.c_int32))
        return s

    def support_of(self, edges) -> np.ndarray:
        """Support of the listed edge ids only."""
        e = np.ascontiguousarray(edges, dtype=np.int64)
        s = np.empty(len(e), dtype=np.int32)
        self._lib.oracle_support_of(self._h, _ptr(e, ctypes.c_int64), len(e),
                                    _ptr(s, ctypes.c_int32))
        return s

    def support_within(self, mask) -> np.ndarray:
        """Support of each edge counting only triangles whose edges all have mask != 0."""
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        s = np.empty(self.m, dtype=np.int32)
        self._lib.oracle_support_within(self._h, _ptr(mk, ctypes.c_uint8),
                                        _ptr(s, ctypes.c_int32))
        return s

    def support_within_of(self, mask, edges) -> np.ndarray:
        """For the listed edge ids: triangles through the edge whose two other edges are in mask."""
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        e = np.ascontiguousarray(edges, dtype=np.int64)
        s = np.empty(len(e), dtype=np.int32)
        self._lib.oracle_support_within_of(self._h, _ptr(mk, ctypes.c_uint8),
                                           _ptr(e, ctypes.c_int64), len(e),
                                           _ptr(s, ctypes.c_int32))
        return s

    def ktruss(self, k: int):
        """(mask uint8[m], support-within-truss int32[m], edges left) for the k-truss."""
        mask = np.empty(self.m, dtype=np.uint8)
        sup = np.empty(self.m, dtype=np.int32)
        left = self._lib.oracle_ktruss(self._h, int(k), _ptr(mask, ctypes.c_uint8),
                                       _ptr(sup, ctypes.c_int32))
        if left < 0:
            raise ValueError("k < 2")
        return mask, sup, int(left)

    def components(self, mask):
        """Connected components of the subgraph of the edges with mask 1:
        (edge labels int32[m], vertex labels int32[n], count); a label is the
        smallest vertex id of the component, -1 outside the subgraph."""
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        el = np.empty(self.m, dtype=np.int32)
        vl = np.empty(self.n, dtype=np.int32)
        c = self._lib.oracle_truss_components(self._h, _ptr(mk, ctypes.c_uint8),
                                              _ptr(el, ctypes.c_int32), _ptr(vl, ctypes.c_int32))
        return el, vl, int(c)

    def ktruss_components(self, k: int):
        """Connected components of the k-truss (see components)."""
        mask, _, _ = self.ktruss(k)
        return self.components(mask)

    def truss_levels(self, kmax: int):
        """Sizes of the k-trusses for k = 3 .. kmax (the decomposition's first
        levels, each continuing from the previous level's survivors)."""
        sizes = np.zeros(max(int(kmax) - 2, 0), dtype=np.int64)
        if self._lib.oracle_truss_levels(self._h, int(kmax), _ptr(sizes, ctypes.c_int64)) != 0:
            raise ValueError("kmax < 3")
        return [int(x) for x in sizes]

    def truss_decomposition(self):
        """(kmax, truss int32[m]): truss[e] = largest k whose k-truss holds e."""
        t = np.zeros(self.m, dtype=np.int32)
        kmax = self._lib.oracle_truss_decomposition(self._h, _ptr(t, ctypes.c_int32))
        return int(kmax), t
