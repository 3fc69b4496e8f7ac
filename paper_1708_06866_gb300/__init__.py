"""Python binding of the GB300 triangle-counting / k-truss library.

Thin ctypes marshalling over the C ABI in ``include/tc.h``: the functions
here carry the ABI's names and do no computation of their own.  Every step
of triangle counting, edge support and k-truss peeling runs in the CUDA
kernels of ``libtc_gb300.so``; if that library is missing this module raises
on first use instead of falling back to anything else.

PyTorch supplies device buffers and streams: arrays are ``torch.Tensor``
objects (CUDA or CPU) or numpy arrays (host); ``stream`` is a
``torch.cuda.Stream`` (default: the current stream).

Kernels of the Static Graph Challenge (Samsi et al. 2017):
  * :func:`tc_count` — triangle count, Section III-A;
  * :func:`tc_edge_support` — per-edge support, Algorithm 4's s = (R == 2) 1;
  * :func:`ktruss` / :func:`ktruss_max` — k-truss and truss decomposition,
    Section III-B.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = [
    "TCError", "Graph", "load_library", "library_path", "tc_build_csr", "tc_count",
    "tc_edge_support", "ktruss", "ktruss_sizes", "ktruss_max", "ktruss_components", "tc_num_edges",
    "tc_num_vertices", "tc_edges",
    "tc_graph_info", "tc_graph_wedge_work", "tc_launch_count", "tc_batch_run",
    "tc_graph_set_memory_limit", "tc_graph_set_result_cache", "tc_read_edges",
    "tc_debug_server_fake", "GraphSource",
    "ServeRequest", "ServeResponse", "ServerStats", "TC_REQ_COUNT", "TC_REQ_KTRUSS",
    "tc_graph_free", "tc_strerror", "tc_last_error", "tc_debug_fail_alloc",
    "tc_debug_spin_limit_ns", "tc_debug_peel_mode", "tc_debug_intersect_mode", "TC_OK", "TC_EINVAL", "TC_ERANGE", "TC_ENOMEM", "TC_ECUDA",
    "TC_ETIMEDOUT", "TC_EOVERFLOW", "TC_INPUT_AUTO", "TC_INPUT_DEVICE", "TC_INPUT_HOST",
]

TC_OK, TC_EINVAL, TC_ERANGE, TC_ENOMEM, TC_ECUDA, TC_ETIMEDOUT, TC_EOVERFLOW = 0, -1, -2, -3, -4, -5, -6
TC_INPUT_AUTO, TC_INPUT_DEVICE, TC_INPUT_HOST = 0, 1, 2

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Loads libtc_gb300.so (compiling it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library not built: {_build.LIB}")
        lib = ctypes.CDLL(_build.LIB)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sig = {
            "tc_build_csr": (ctypes.c_int, [vp, vp, i64, i32, ctypes.c_int, vp,
                                            ctypes.POINTER(vp)]),
            "tc_count": (ctypes.c_int, [vp, ctypes.POINTER(i64), vp]),
            "tc_edge_support": (ctypes.c_int, [vp, vp, ctypes.POINTER(i64), vp]),
            "ktruss": (ctypes.c_int, [vp, i32, vp, ctypes.POINTER(i64), vp]),
            "ktruss_max": (ctypes.c_int, [vp, ctypes.POINTER(i32), vp, vp]),
            "tc_num_edges": (i64, [vp]),
            "tc_num_vertices": (i32, [vp]),
            "tc_edges": (ctypes.c_int, [vp, vp, vp, vp]),
            "tc_graph_free": (None, [vp]),
            "tc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "tc_last_error": (ctypes.c_char_p, []),
            "tc_graph_info": (ctypes.c_int, [vp, ctypes.POINTER(GraphInfo), vp]),
            "tc_launch_count": (i64, []),
            "tc_graph_set_memory_limit": (ctypes.c_int, [vp, i64]),
            "tc_graph_set_result_cache": (ctypes.c_int, [vp, i32]),
            "ktruss_sizes": (ctypes.c_int, [vp, i32, i32, ctypes.POINTER(i64), vp]),
            "tc_server_set_result_cache": (ctypes.c_int, [vp, i32]),
            "ktruss_components": (ctypes.c_int, [vp, i32, vp, vp, ctypes.POINTER(i64), vp]),
            "tc_read_edges": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, vp, vp, i64,
                                             ctypes.POINTER(i64), ctypes.POINTER(i32)]),
            "tc_server_create": (ctypes.c_int, [ctypes.POINTER(GraphSource), i32, i64, i64,
                                                i32, ctypes.POINTER(vp)]),
            "tc_server_run": (ctypes.c_int, [vp, ctypes.POINTER(ServeRequest), i64, i32, i32,
                                             ctypes.POINTER(ServeResponse),
                                             ctypes.POINTER(ctypes.c_double)]),
            "tc_server_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(ServerStats)]),
            "tc_server_destroy": (None, [vp]),
            "tc_debug_server_fake": (ctypes.c_int, [ctypes.c_int]),
            "tc_batch_run": (ctypes.c_int, [ctypes.POINTER(BatchDesc), vp]),
            "tc_graph_wedge_work": (ctypes.c_int, [vp, ctypes.POINTER(i64), vp]),
            "tc_debug_fail_alloc": (i64, [i64]),
            "tc_debug_spin_limit_ns": (i64, [i64]),
            "tc_debug_peel_mode": (ctypes.c_int, [ctypes.c_int]),
            "tc_debug_intersect_mode": (ctypes.c_int, [ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


class GraphSource(ctypes.Structure):
    """Mirror of tc_graph_source."""
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("m_in", ctypes.c_int64),
                ("n", ctypes.c_int32), ("pad", ctypes.c_int32)]


class ServeRequest(ctypes.Structure):
    """Mirror of tc_request."""
    _fields_ = [("graph", ctypes.c_int32), ("kind", ctypes.c_int32), ("k", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("arrival_s", ctypes.c_double)]


class ServeResponse(ctypes.Structure):
    """Mirror of tc_response."""
    _fields_ = [("result", ctypes.c_int64), ("start_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("status", ctypes.c_int32), ("slot", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    """Mirror of tc_server_stats."""
    _fields_ = [(f, ctypes.c_int64) for f in
                ("builds", "evictions", "max_concurrent", "peak_reserved_bytes", "errors",
                 "violations", "reserved_bytes", "resident_graphs")]


TC_REQ_COUNT, TC_REQ_KTRUSS = 0, 1


class GraphInfo(ctypes.Structure):
    """Mirror of tc_graph_info_t."""
    _fields_ = [(f, ctypes.c_int64) for f in
                ("n", "m_in", "m", "max_degree", "max_out", "wedge_work", "device_bytes",
                 "peel_rounds", "peel_lists", "count_kernel_ns", "support_kernel_ns",
                 "lists_kernel_ns", "peel_kernel_ns", "peel_bytes", "peel_scanned",
                 "peel_entries", "peel_searches", "peel_lookups", "peel_lowered",
                 "truss_cached", "column_work", "product_form", "lists_bytes")]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class BatchStats(ctypes.Structure):
    """Mirror of tc_batch_stats_t."""
    _fields_ = [("build_ns", ctypes.c_int64), ("query_ns", ctypes.c_int64),
                ("m", ctypes.c_int64), ("triangles", ctypes.c_int64),
                ("intersect_form", ctypes.c_int32), ("peel_form", ctypes.c_int32),
                ("tuned_from_cache", ctypes.c_int32), ("captured", ctypes.c_int32),
                ("peel_blocks", ctypes.c_int32), ("light_degree", ctypes.c_int32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class BatchDesc(ctypes.Structure):
    """Mirror of tc_batch_desc."""
    _fields_ = [("num_graphs", ctypes.c_int32), ("n", ctypes.c_void_p),
                ("edge_off", ctypes.c_void_p), ("src", ctypes.c_void_p),
                ("dst", ctypes.c_void_p), ("k", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("triangles_out", ctypes.c_void_p), ("edges_out", ctypes.c_void_p),
                ("truss_edges_out", ctypes.c_void_p), ("stats_out", ctypes.c_void_p)]


class TCError(RuntimeError):
    """A TC_E* status returned by the C ABI."""

    def __init__(self, code: int, message: str):
        super().__init__(f"{message} (code {code})")
        self.code = code


def tc_strerror(code: int) -> str:
    return load_library().tc_strerror(int(code)).decode()


def tc_last_error() -> str:
    return load_library().tc_last_error().decode()


def _check(rc: int, what: str):
    if rc != TC_OK:
        raise TCError(rc, f"{what}: {tc_strerror(rc)}: {tc_last_error()}")


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _ptr(a):
    """Raw address of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data or None
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr() or None


class Graph:
    """A device-resident graph built by :func:`tc_build_csr` (owned handle)."""

    def __init__(self, handle: int, device):
        self._h = handle
        self.device = device

    @property
    def handle(self):
        if not self._h:
            raise ValueError("graph was freed")
        return self._h

    @property
    def m(self) -> int:
        return tc_num_edges(self)

    @property
    def n(self) -> int:
        return tc_num_vertices(self)

    def free(self):
        if getattr(self, "_h", None):
            load_library().tc_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _as_int32(a):
    torch = _torch()
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.int32)
    if a.dtype != torch.int32:
        a = a.to(torch.int32)
    return a.contiguous()


def tc_build_csr(src, dst, n: int, stream=None, flags: int = TC_INPUT_AUTO) -> Graph:
    """Cleans an edge list (Section II rules) and builds the device graph.

    src, dst: int32 endpoints, 0-based, as CUDA or CPU tensors or numpy arrays.
    """
    lib = load_library()
    torch = _torch()
    src = _as_int32(src)
    dst = _as_int32(dst)
    if len(src) != len(dst):
        raise ValueError("src and dst differ in length")
    h = ctypes.c_void_p()
    rc = lib.tc_build_csr(_ptr(src), _ptr(dst), len(src), int(n), int(flags),
                          _stream_handle(stream), ctypes.byref(h))
    _check(rc, "tc_build_csr")
    return Graph(h.value, torch.device("cuda", torch.cuda.current_device()))


def tc_count(g: Graph, stream=None) -> int:
    """Number of triangles."""
    out = ctypes.c_int64(0)
    _check(load_library().tc_count(g.handle, ctypes.byref(out), _stream_handle(stream)),
           "tc_count")
    return out.value


def tc_edge_support(g: Graph, out=None, stream=None, triangles: bool = True):
    """Per-edge triangle support (int32, edge-id order) and the triangle count.

    Returns (support, T); T is None when ``triangles`` is False.  ``out`` may
    be a CUDA or CPU int32 tensor of m entries (allocated on the device if None).
    """
    torch = _torch()
    m = g.m
    if out is None:
        out = torch.empty(m, dtype=torch.int32, device=g.device)
    t = ctypes.c_int64(0)
    rc = load_library().tc_edge_support(g.handle, _ptr(out), ctypes.byref(t) if triangles else None,
                                        _stream_handle(stream))
    _check(rc, "tc_edge_support")
    return out, (t.value if triangles else None)


def ktruss(g: Graph, k: int, out=None, stream=None):
    """The k-truss as a uint8 mask over edge ids, and its edge count."""
    torch = _torch()
    if out is None:
        out = torch.empty(g.m, dtype=torch.uint8, device=g.device)
    left = ctypes.c_int64(0)
    rc = load_library().ktruss(g.handle, int(k), _ptr(out), ctypes.byref(left),
                               _stream_handle(stream))
    _check(rc, "ktruss")
    return out, left.value


def ktruss_components(g: Graph, k: int, stream=None, vertices: bool = True):
    """Connected components of the k-truss: (edge labels int32[m] in
    canonical order, vertex labels int32[n] or None, count); a label is the
    component's smallest vertex id, -1 outside the k-truss."""
    torch = _torch()
    dev = g.device
    el = torch.empty(max(g.m, 0), dtype=torch.int32, device=dev)
    vl = torch.empty(g.n, dtype=torch.int32, device=dev) if vertices else None
    c = ctypes.c_int64()
    _check(load_library().ktruss_components(g.handle, int(k), _ptr(el) if g.m else None,
                                            _ptr(vl) if vl is not None else None,
                                            ctypes.byref(c), _stream_handle(stream)),
           "ktruss_components")
    return el, vl, c.value


def ktruss_sizes(g: Graph, k_lo: int, k_hi: int, stream=None):
    """Sizes of the k-trusses for k = k_lo .. k_hi (one peel for the range)."""
    nk = int(k_hi) - int(k_lo) + 1
    out = (ctypes.c_int64 * max(nk, 1))()
    _check(load_library().ktruss_sizes(g.handle, int(k_lo), int(k_hi), out,
                                       _stream_handle(stream)), "ktruss_sizes")
    return [int(out[i]) for i in range(nk)]


def ktruss_max(g: Graph, out=None, stream=None, want_truss: bool = True):
    """Truss decomposition: (kmax, per-edge truss numbers or None)."""
    torch = _torch()
    if out is None and want_truss:
        out = torch.empty(g.m, dtype=torch.int32, device=g.device)
    kmax = ctypes.c_int32(0)
    rc = load_library().ktruss_max(g.handle, ctypes.byref(kmax), _ptr(out) if want_truss else None,
                                   _stream_handle(stream))
    _check(rc, "ktruss_max")
    return kmax.value, out


def tc_num_edges(g: Graph) -> int:
    return int(load_library().tc_num_edges(g.handle))


def tc_num_vertices(g: Graph) -> int:
    return int(load_library().tc_num_vertices(g.handle))


def tc_edges(g: Graph, stream=None, device=None):
    """The canonical edge list (lo, hi) in original ids, edge-id order."""
    torch = _torch()
    dev = g.device if device is None else device
    lo = torch.empty(g.m, dtype=torch.int32, device=dev)
    hi = torch.empty(g.m, dtype=torch.int32, device=dev)
    _check(load_library().tc_edges(g.handle, _ptr(lo), _ptr(hi), _stream_handle(stream)),
           "tc_edges")
    return lo, hi


def tc_graph_info(g: Graph, stream=None) -> dict:
    """Sizes of the graph: n, m_in, m, max_degree, max_out, wedge_work, device_bytes."""
    info = GraphInfo()
    _check(load_library().tc_graph_info(g.handle, ctypes.byref(info), _stream_handle(stream)),
           "tc_graph_info")
    return info.as_dict()


def tc_graph_wedge_work(g: Graph, stream=None) -> int:
    """Sum over oriented edges (u, v) of |N+(u)| + |N+(v)| (one kernel, cached)."""
    out = ctypes.c_int64(0)
    _check(load_library().tc_graph_wedge_work(g.handle, ctypes.byref(out), _stream_handle(stream)),
           "tc_graph_wedge_work")
    return out.value


def tc_graph_set_result_cache(g: Graph, keep: bool):
    """Whether the graph keeps results (truss numbers, the latest k-truss) between calls."""
    _check(load_library().tc_graph_set_result_cache(g.handle, 1 if keep else 0),
           "tc_graph_set_result_cache")


def tc_graph_set_memory_limit(g: Graph, nbytes: int):
    """Bound on the optional device memory (triangle lists, caches) for this graph; <0 = auto."""
    _check(load_library().tc_graph_set_memory_limit(g.handle, int(nbytes)),
           "tc_graph_set_memory_limit")


def tc_read_edges(path: str, fmt: int = 0):
    """Edge list of a tab-separated or Matrix Market file (1-based ids in the
    file) as 0-based int32 numpy arrays: returns (src, dst, n)."""
    lib = load_library()
    m = ctypes.c_int64()
    n = ctypes.c_int32()
    bpath = os.fsencode(path)
    _check(lib.tc_read_edges(bpath, int(fmt), None, None, 0, ctypes.byref(m), ctypes.byref(n)),
           "tc_read_edges")
    src = np.empty(m.value, dtype=np.int32)
    dst = np.empty(m.value, dtype=np.int32)
    _check(lib.tc_read_edges(bpath, int(fmt), src.ctypes.data, dst.ctypes.data, m.value,
                             ctypes.byref(m), ctypes.byref(n)), "tc_read_edges")
    return src, dst, n.value


def tc_launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load_library().tc_launch_count())


def tc_batch_run(n, edge_off, src, dst, k: int = 0, use_graph: bool = True, stream=None):
    """Triangle counts (and k-truss sizes if k >= 2) of many graphs in one pass.

    n: vertices per graph; edge_off: num_graphs + 1 offsets into the
    concatenated src/dst (ids local to each graph).  Returns a dict with
    numpy arrays "triangles", "edges", "truss_edges" and "stats".
    """
    n = np.ascontiguousarray(n, dtype=np.int32)
    edge_off = np.ascontiguousarray(edge_off, dtype=np.int64)
    G = len(n)
    if len(edge_off) != G + 1:
        raise ValueError("edge_off must have num_graphs + 1 entries")
    src = _as_int32(src)
    dst = _as_int32(dst)
    tri = np.zeros(G, dtype=np.int64)
    edges = np.zeros(G, dtype=np.int64)
    truss = np.zeros(G, dtype=np.int64)
    stats = BatchStats()
    d = BatchDesc(G, n.ctypes.data, edge_off.ctypes.data, _ptr(src), _ptr(dst), int(k),
                  int(bool(use_graph)), tri.ctypes.data, edges.ctypes.data, truss.ctypes.data,
                  ctypes.addressof(stats))
    _check(load_library().tc_batch_run(ctypes.byref(d), _stream_handle(stream)), "tc_batch_run")
    return {"triangles": tri, "edges": edges, "truss_edges": truss, "stats": stats.as_dict()}


def tc_graph_free(g: Graph):
    g.free()


def tc_debug_fail_alloc(nth: int) -> int:
    return int(load_library().tc_debug_fail_alloc(int(nth)))


def tc_debug_server_fake(on: bool) -> bool:
    """Test hook: servers created while on sleep instead of using the GPU."""
    return bool(load_library().tc_debug_server_fake(1 if on else 0))


def tc_debug_peel_mode(mode: int) -> int:
    """0 automatic, 1 triangle lists, 2 intersections; returns the previous mode."""
    return int(load_library().tc_debug_peel_mode(int(mode)))


def tc_debug_intersect_mode(mode: int) -> int:
    """0 automatic, 1 row/hash kernel, 2 edge-per-warp kernel; returns the previous mode."""
    return int(load_library().tc_debug_intersect_mode(int(mode)))


def tc_debug_spin_limit_ns(ns: int) -> int:
    return int(load_library().tc_debug_spin_limit_ns(int(ns)))
