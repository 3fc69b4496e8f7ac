"""Serving: triangle-count and k-truss queries on device-resident graphs.

A thin wrapper over the library's native request loop (``tc_server_*`` in
``include/tc.h``): requests (graph id, query) arrive over time and are
served with continuous batching by a fixed number of worker threads, each
with its own CUDA stream; a free slot takes the oldest request whose graph
is idle and resident, or can be made resident within the device-memory
budget after evicting least-recently-used idle graphs.  Graphs are built on
first use and kept resident; a graph serves one call at a time, requests for
different graphs overlap.  Latency runs from a request's arrival to its
result on the host.

This module only marshals: traces in, results out.  It also generates
Poisson traces and summarises latencies.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Dict, List, Optional

import numpy as np

import paper_1708_06866_gb300 as tc


@dataclasses.dataclass
class Request:
    rid: int
    graph: int
    kind: str             # "count" or "ktruss"
    k: int = 0
    arrival: float = 0.0  # seconds after the run start
    start: float = 0.0
    done: float = 0.0
    result: Optional[int] = None
    error: Optional[str] = None
    slot: int = -1

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class NativeServer:
    """The library's server over a pool of graphs {id: (src, dst, n)} with
    host int32 edge lists (kept referenced while the server lives)."""

    def __init__(self, pool: Dict[int, tuple], slots: int = 8, budget_bytes: int = 120 << 30,
                 optional_bytes_per_pair: int = 40, keep_results: bool = True):
        self.lib = tc.load_library()
        self.handle = None
        self.ids = sorted(pool)
        self.index = {g: i for i, g in enumerate(self.ids)}
        self._keep = []
        src = (tc.GraphSource * max(1, len(self.ids)))()
        for i, g in enumerate(self.ids):
            s, d, n = pool[g]
            s = np.ascontiguousarray(s, dtype=np.int32)
            d = np.ascontiguousarray(d, dtype=np.int32)
            self._keep += [s, d]
            src[i].src = s.ctypes.data or None
            src[i].dst = d.ctypes.data or None
            src[i].m_in = len(s)
            src[i].n = int(n)
        self._src = src
        self.m_in = {g: int(pool[g][0].shape[0]) for g in self.ids}
        h = ctypes.c_void_p()
        tc._check(self.lib.tc_server_create(src, len(self.ids), int(budget_bytes),
                                            int(optional_bytes_per_pair), int(slots),
                                            ctypes.byref(h)), "tc_server_create")
        self.handle = h.value
        self.slots = slots
        if not keep_results:
            self.set_result_cache(False)

    def set_result_cache(self, keep: bool):
        """keep=False: every k-truss request peels on the device (no kept
        truss decompositions or k-truss states)."""
        tc._check(self.lib.tc_server_set_result_cache(self.handle, 1 if keep else 0),
                  "tc_server_set_result_cache")

    def run(self, trace, open_loop: bool = True, slots: int = 0) -> float:
        """Serves [(arrival seconds, Request)] in order; fills each Request's
        result, times, slot and error.  slots: how many of the server's slots
        serve (0 = all; 1 = the plain one-at-a-time loop).  Returns the run's
        wall time (s)."""
        n = len(trace)
        reqs = (tc.ServeRequest * max(1, n))()
        for i, (at, r) in enumerate(trace):
            reqs[i].graph = self.index[r.graph]
            reqs[i].kind = tc.TC_REQ_COUNT if r.kind == "count" else tc.TC_REQ_KTRUSS
            reqs[i].k = int(r.k)
            reqs[i].arrival_s = float(at) if open_loop else 0.0
        out = (tc.ServeResponse * max(1, n))()
        wall = ctypes.c_double()
        rc = self.lib.tc_server_run(self.handle, reqs, n, 1 if open_loop else 0, int(slots), out,
                                    ctypes.byref(wall))
        if rc not in (tc.TC_OK, tc.TC_ECUDA):
            tc._check(rc, "tc_server_run")
        for i, (at, r) in enumerate(trace):
            o = out[i]
            r.arrival = float(at) if open_loop else 0.0
            r.start, r.done, r.slot = o.start_s, o.done_s, o.slot
            if o.status == tc.TC_OK:
                r.result, r.error = int(o.result), None
            else:
                r.result, r.error = None, f"{tc.tc_strerror(o.status)} (code {o.status})"
        return wall.value

    def stats(self) -> dict:
        st = tc.ServerStats()
        tc._check(self.lib.tc_server_get_stats(self.handle, ctypes.byref(st)),
                  "tc_server_get_stats")
        return {f: int(getattr(st, f)) for f, _ in st._fields_}

    def close(self):
        if self.handle:
            self.lib.tc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poisson_trace(num: int, rate: float, graph_ids, seed: int, ks=(3, 4, 5, 6, 7, 8),
                  count_share: float = 0.5):
    """Requests with exponential inter-arrival gaps (rate per second; 0 = all
    at once): half triangle counts, half k-truss queries with k uniform in
    ks, on graphs drawn uniformly from graph_ids."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, num) if rate > 0 else np.zeros(num)
    times = np.cumsum(gaps) - gaps[0]
    gids = rng.choice(np.asarray(graph_ids), num)
    is_count = rng.random(num) < count_share
    kk = rng.choice(np.asarray(ks), num)
    return [(float(times[i]), Request(i, int(gids[i]), "count" if is_count[i] else "ktruss",
                                      0 if is_count[i] else int(kk[i]))) for i in range(num)]


def fresh(trace):
    """The same requests, unserved (for another run)."""
    return [(at, Request(r.rid, r.graph, r.kind, r.k)) for at, r in trace]


def summarize(reqs: List[Request], wall: float) -> dict:
    lat = np.array([r.latency for r in reqs]) * 1e3
    return {"requests": len(reqs), "errors": sum(r.error is not None for r in reqs),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "throughput_rps": len(reqs) / wall, "wall_s": wall}
