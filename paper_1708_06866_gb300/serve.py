"""Serving loop: triangle-count and k-truss queries on device-resident graphs.

Requests (graph id, query) arrive over time and are served with continuous
batching: a fixed number of worker slots, each with its own CUDA stream,
take the oldest admissible request as soon as they are free, so work of
requests that arrive while others run overlaps on the device.  Graphs are
built on first use and kept resident (their CSR and cached supports) under
an HBM budget; least-recently-used idle graphs are evicted to admit a new
one, and a request whose graph cannot be admitted yet waits while requests
on resident graphs go ahead.  A graph serves one call at a time (the ABI's
rule); requests for different graphs overlap.

The scheduler talks to a backend (build / free / query); ``GpuBackend`` runs
the library's kernels.  Latency is measured on the host from a request's
arrival to its result.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    graph: int
    kind: str             # "count" or "ktruss"
    k: int = 0
    arrival: float = 0.0  # host clock (time.perf_counter) at submission
    start: float = 0.0
    done: float = 0.0
    result: Optional[int] = None
    error: Optional[str] = None
    slot: int = -1
    event: threading.Event = dataclasses.field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class GpuBackend:
    """Builds graphs with tc_build_csr and answers queries with tc_count /
    ktruss on the caller's stream.  Graph inputs stay on the host until
    built (the build copies them in)."""

    def __init__(self, graphs: Dict[int, tuple], device: int = 0):
        import torch
        import paper_1708_06866_gb300 as tc
        self.tc = tc
        self.torch = torch
        self.graphs = graphs
        self.device = device
        torch.cuda.set_device(device)

    def new_stream(self):
        return self.torch.cuda.Stream(device=self.device)

    # per input pair: CSR and edge arrays (~40 B), call scratch of a peel
    # (~60 B), and the optional memory (triangle lists, caches) the graph may
    # use (OPTIONAL_PER_PAIR, enforced through tc_graph_set_memory_limit)
    OPTIONAL_PER_PAIR = 40

    def estimate_bytes(self, gid: int) -> int:
        """Device bytes a graph may need while it is used."""
        src, _, _ = self.graphs[gid]
        return (100 + self.OPTIONAL_PER_PAIR) * len(src) + (1 << 20)

    def build(self, gid: int, stream):
        src, dst, n = self.graphs[gid]
        with self.torch.cuda.stream(stream):
            g = self.tc.tc_build_csr(src, dst, n, stream=stream)
        self.tc.tc_graph_set_memory_limit(g, self.OPTIONAL_PER_PAIR * len(src))
        return g

    def free(self, handle):
        handle.free()

    def held_bytes(self, handle) -> int:
        """Device bytes the graph holds now (it keeps supports and triangle
        lists between queries)."""
        return int(self.tc.tc_graph_info(handle)["device_bytes"])

    def query(self, handle, req: Request, stream) -> int:
        with self.torch.cuda.stream(stream):
            if req.kind == "count":
                return self.tc.tc_count(handle, stream=stream)
            _, left = self.tc.ktruss(handle, req.k, stream=stream)
            return left


class Server:
    """Continuous-batching scheduler over a backend."""

    def __init__(self, backend, slots: int = 8, budget_bytes: int = 120 << 30):
        self.backend = backend
        self.slots = slots
        self.budget = budget_bytes
        self.cv = threading.Condition()
        self.pending: collections.deque = collections.deque()
        self.resident: "collections.OrderedDict[int, dict]" = collections.OrderedDict()
        self.reserved = 0
        self.busy_graphs = set()
        self.building = set()
        self.stop = False
        self.completed: List[Request] = []
        self.evictions = 0
        self.builds = 0
        self.max_concurrent = 0
        self.running = 0
        self.threads = [threading.Thread(target=self._worker, args=(i,), daemon=True)
                        for i in range(slots)]
        for t in self.threads:
            t.start()

    # ---------------------------------------------------------- client side
    def submit(self, req: Request) -> Request:
        req.arrival = time.perf_counter()
        with self.cv:
            self.pending.append(req)
            self.cv.notify_all()
        return req

    def shutdown(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for t in self.threads:
            t.join(timeout=60)
        for gid, ent in list(self.resident.items()):
            if ent["handle"] is not None:
                self.backend.free(ent["handle"])
        self.resident.clear()

    # ---------------------------------------------------------- scheduling
    def _admissible(self, req: Request) -> bool:
        """The graph is resident and idle, or can be made resident (budget
        after evicting idle graphs) and nobody is building it."""
        g = req.graph
        if g in self.busy_graphs or g in self.building:
            return False
        if g in self.resident:
            return True
        need = self.backend.estimate_bytes(g)
        freeable = sum(e["bytes"] for gid, e in self.resident.items()
                       if gid not in self.busy_graphs)
        return self.reserved - freeable + need <= self.budget or not self.resident

    def _take(self) -> Optional[Request]:
        """Oldest admissible request (FIFO among those that can run now)."""
        for i, req in enumerate(self.pending):
            if self._admissible(req):
                del self.pending[i]
                return req
        return None

    def _make_room(self, need: int) -> List:
        """Evicts least-recently-used idle graphs until `need` fits; returns
        their handles for freeing outside the lock."""
        out = []
        for gid in list(self.resident.keys()):
            if self.reserved + need <= self.budget:
                break
            if gid in self.busy_graphs:
                continue
            ent = self.resident.pop(gid)
            self.reserved -= ent["bytes"]
            self.evictions += 1
            out.append(ent["handle"])
        return out

    def _worker(self, slot: int):
        stream = self.backend.new_stream()
        while True:
            with self.cv:
                req = None
                while not self.stop:
                    req = self._take()
                    if req is not None:
                        break
                    self.cv.wait(timeout=0.05)
                if req is None:
                    return
                g = req.graph
                self.busy_graphs.add(g)
                handle = None
                to_free = []
                if g in self.resident:
                    self.resident.move_to_end(g)
                    handle = self.resident[g]["handle"]
                else:
                    need = self.backend.estimate_bytes(g)
                    to_free = self._make_room(need)
                    self.reserved += need
                    self.building.add(g)
                self.running += 1
                self.max_concurrent = max(self.max_concurrent, self.running)
            for h in to_free:
                self.backend.free(h)
            req.slot = slot
            req.start = time.perf_counter()
            try:
                if handle is None:
                    handle = self.backend.build(g, stream)
                    with self.cv:
                        self.builds += 1
                        self.building.discard(g)
                        self.resident[g] = {"handle": handle,
                                            "bytes": self.backend.estimate_bytes(g)}
                req.result = self.backend.query(handle, req, stream)
                held = getattr(self.backend, "held_bytes", None)
                if held is not None:
                    now_bytes = max(held(handle), self.backend.estimate_bytes(g))
                    with self.cv:
                        ent = self.resident.get(g)
                        if ent is not None and now_bytes != ent["bytes"]:
                            self.reserved += now_bytes - ent["bytes"]
                            ent["bytes"] = now_bytes
            except Exception as exc:  # reported per request, the server keeps going
                req.error = repr(exc)
                with self.cv:
                    if g in self.building:
                        self.building.discard(g)
                        self.reserved -= self.backend.estimate_bytes(g)
            req.done = time.perf_counter()
            with self.cv:
                self.busy_graphs.discard(g)
                self.running -= 1
                self.completed.append(req)
                self.cv.notify_all()
            req.event.set()


def poisson_trace(num: int, rate: float, graph_ids, seed: int, ks=(3, 4, 5, 6, 7, 8),
                  count_share: float = 0.5):
    """Requests with exponential inter-arrival gaps (rate per second): half
    triangle counts, half k-truss queries with k uniform in ks, on graphs
    drawn uniformly from graph_ids."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, num) if rate > 0 else np.zeros(num)
    times = np.cumsum(gaps) - gaps[0]
    gids = rng.choice(np.asarray(graph_ids), num)
    is_count = rng.random(num) < count_share
    kk = rng.choice(np.asarray(ks), num)
    return [(float(times[i]), Request(i, int(gids[i]), "count" if is_count[i] else "ktruss",
                                      0 if is_count[i] else int(kk[i]))) for i in range(num)]


def replay(server: Server, trace, timeout: float = 600.0,
           clock: Callable[[], float] = time.perf_counter):
    """Submits each request at its scheduled offset and waits for all."""
    t0 = clock()
    for at, req in trace:
        delay = at - (clock() - t0)
        if delay > 0:
            time.sleep(delay)
        server.submit(req)
    deadline = time.perf_counter() + timeout
    for _, req in trace:
        if not req.event.wait(max(0.0, deadline - time.perf_counter())):
            raise TimeoutError(f"request {req.rid} not served in time")
    return clock() - t0


def summarize(reqs: List[Request], wall: float) -> dict:
    lat = np.array([r.latency for r in reqs]) * 1e3
    return {"requests": len(reqs), "errors": sum(r.error is not None for r in reqs),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "throughput_rps": len(reqs) / wall, "wall_s": wall}
