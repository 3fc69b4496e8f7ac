// server.cu — a continuous-batching request loop over device-resident graphs.
//
// Requests (triangle count, or the size of the k-truss, on one graph of a
// pool) arrive over time.  A fixed number of worker threads ("slots"), each
// with its own CUDA stream, take the oldest request that can run now: its
// graph is idle (a graph serves one call at a time, the ABI's rule) and is
// resident or can be made resident within the device-memory budget after
// evicting least-recently-used idle graphs.  Graphs are built on first use
// from the caller's host edge lists.  Work of requests that arrive while
// others run overlaps on the device.  By default a graph's first k-truss
// request computes its truss decomposition, which the library keeps with the
// graph, so later k-truss requests on it are threshold passes (Section
// III-B: the k-trusses nest); with results not kept
// (tc_server_set_result_cache) every k-truss request peels on the device.
// With more than one slot, a slot that takes a request also takes the
// other requests for the same graph that have arrived and wait (coalescing,
// up to MAX_GROUP): their counts come from one count call and their k-truss
// sizes from one ktruss_sizes peel over their range of k.  One slot is the
// plain loop: one request per call, in arrival order.
//
// Test hook: a fake mode runs the same scheduler with sleeps instead of
// device work (no CUDA calls), so its host logic is testable without a GPU.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include "tc_internal.cuh"

namespace {

std::atomic<int> g_server_fake{0};
constexpr int MAX_GROUP = 64;  // requests answered by one slot's turn

using Clock = std::chrono::steady_clock;

struct Slot {
    cudaStream_t stream = nullptr;
    uint8_t* mask = nullptr;  // device k-truss mask scratch
    int64_t mask_cap = 0;
};

struct Entry {
    tc_graph* g = nullptr;
    bool resident = false;
    bool busy = false;
    bool building = false;
    bool indexed = false;     // its truss decomposition is kept
    bool index_tried = false;  // ... or could not be (memory bound): peel per request
    int64_t reserved = 0;
    uint64_t last_use = 0;
    std::atomic<int> in_call{0};  // fake mode: concurrent calls seen on the graph
};

}  // namespace

struct tc_server {
    std::vector<tc_graph_source> src;
    std::vector<Entry> graphs;
    std::vector<Slot> slots;
    int device = 0;
    bool fake = false;
    int64_t budget = 0;
    int64_t opt_per_pair = 0;
    bool keep_results = true;
    int64_t reserved = 0;
    uint64_t tick = 0;
    tc_server_stats stats{};
    std::mutex mu;
    std::condition_variable cv;

    explicit tc_server(int32_t num_graphs) : graphs(num_graphs) {}

    int64_t estimate(int32_t gid) const {
        // CSR and edge arrays (~40 B per input pair), a call's scratch
        // (at most ~56 B: the peel's lists of edges, frontier ranges and
        // round table), and the optional memory the graph may keep
        return (100 + opt_per_pair) * src[gid].m_in + (1 << 20);
    }
};

namespace {

double seconds_since(Clock::time_point t0) {
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

// Runs one request on its slot.  Returns a TC_* status.
int execute(tc_server* s, Slot& slot, int32_t gid, const tc_request& rq, int64_t* result) {
    Entry& e = s->graphs[gid];
    if (s->fake) {
        if (e.in_call.fetch_add(1) != 0) {
            std::lock_guard<std::mutex> lk(s->mu);
            ++s->stats.violations;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(100));
        e.in_call.fetch_sub(1);
        *result = (int64_t)gid * 1000 + (rq.kind == TC_REQ_COUNT ? 0 : rq.k);
        return TC_OK;
    }
    if (rq.kind == TC_REQ_COUNT) return tc_count(e.g, result, slot.stream);
    if (rq.kind != TC_REQ_KTRUSS) return tc::fail(TC_EINVAL, "server: unknown request kind");
    if (s->keep_results && !e.indexed && !e.index_tried) {
        e.index_tried = true;
        int32_t kmax = 0;
        TC_TRY(ktruss_max(e.g, &kmax, nullptr, slot.stream));
        tc_graph_info_t info;
        TC_TRY(tc_graph_info(e.g, &info, slot.stream));
        e.indexed = info.truss_cached != 0;
    }
    const int64_t m = tc_num_edges(e.g);
    if (m > slot.mask_cap) {
        if (slot.mask) cudaFreeAsync(slot.mask, slot.stream);
        slot.mask = nullptr;
        slot.mask_cap = 0;
        TC_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&slot.mask), (size_t)m, slot.stream));
        slot.mask_cap = m;
    }
    return ktruss(e.g, rq.k, slot.mask, result, slot.stream);
}

// Answers requests reqs[ids[0..cnt)] (all on graph gid): counts from one
// call, k-truss sizes from one ktruss_sizes over their k range (or one
// ktruss when a single k-truss request is in the group).
int execute_group(tc_server* s, Slot& slot, int32_t gid, const tc_request* reqs,
                  const int64_t* ids, int cnt, int64_t* results) {
    if (cnt == 1 || s->fake) {
        for (int i = 0; i < cnt; ++i) TC_TRY(execute(s, slot, gid, reqs[ids[i]], &results[i]));
        return TC_OK;
    }
    Entry& e = s->graphs[gid];
    int32_t klo = INT32_MAX, khi = 0, nk = 0;
    bool any_count = false;
    for (int i = 0; i < cnt; ++i) {
        const tc_request& rq = reqs[ids[i]];
        if (rq.kind == TC_REQ_COUNT) {
            any_count = true;
        } else {
            klo = std::min(klo, rq.k);
            khi = std::max(khi, rq.k);
            ++nk;
        }
    }
    int64_t T = 0;
    if (any_count) TC_TRY(tc_count(e.g, &T, slot.stream));
    int64_t sizes[64];
    const bool range = nk > 1 && khi - klo < 64;
    if (range) {
        if (s->keep_results && !e.indexed && !e.index_tried) {
            e.index_tried = true;
            int32_t kmax = 0;
            TC_TRY(ktruss_max(e.g, &kmax, nullptr, slot.stream));
            tc_graph_info_t info;
            TC_TRY(tc_graph_info(e.g, &info, slot.stream));
            e.indexed = info.truss_cached != 0;
        }
        TC_TRY(ktruss_sizes(e.g, klo, khi, sizes, slot.stream));
    }
    for (int i = 0; i < cnt; ++i) {
        const tc_request& rq = reqs[ids[i]];
        if (rq.kind == TC_REQ_COUNT) results[i] = T;
        else if (range) results[i] = sizes[rq.k - klo];
        else TC_TRY(execute(s, slot, gid, rq, &results[i]));
    }
    return TC_OK;
}

int build(tc_server* s, Slot& slot, int32_t gid) {
    Entry& e = s->graphs[gid];
    if (s->fake) {
        std::this_thread::sleep_for(std::chrono::microseconds(200));
        e.g = reinterpret_cast<tc_graph*>(static_cast<uintptr_t>(gid + 1));
        return TC_OK;
    }
    const tc_graph_source& g = s->src[gid];
    TC_TRY(tc_build_csr(g.src, g.dst, g.m_in, g.n, TC_INPUT_HOST, slot.stream, &e.g));
    TC_TRY(tc_graph_set_result_cache(e.g, s->keep_results ? 1 : 0));
    return tc_graph_set_memory_limit(e.g, s->opt_per_pair * g.m_in);
}

void release(tc_server* s, tc_graph* g) {
    if (!s->fake && g) tc_graph_free(g);
}

void worker(tc_server* s, int slot_id, const tc_request* reqs, int64_t nreq, bool open_loop,
            bool coalesce, Clock::time_point t0, std::vector<char>* taken, int64_t* head,
            int64_t* left, int64_t* running, tc_response* out) {
    if (!s->fake) cudaSetDevice(s->device);
    Slot& slot = s->slots[slot_id];
    int64_t group[MAX_GROUP];
    int64_t results[MAX_GROUP];
    for (;;) {
        int64_t pick = -1;
        int ng = 0;
        std::vector<tc_graph*> evict;
        bool need_build = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                if (*left == 0) return;
                const double now = seconds_since(t0);
                double next_arrival = -1;
                while (*head < nreq && (*taken)[*head]) ++*head;
                for (int64_t i = *head; i < nreq; ++i) {
                    if ((*taken)[i]) continue;
                    const tc_request& rq = reqs[i];
                    if (open_loop && rq.arrival_s > now) {
                        next_arrival = rq.arrival_s;  // requests are in arrival order
                        break;
                    }
                    Entry& e = s->graphs[rq.graph];
                    if (e.busy || e.building) continue;
                    if (e.resident) {
                        pick = i;
                        break;
                    }
                    // can it be made resident: budget after evicting idle graphs
                    int64_t freeable = 0;
                    for (const Entry& o : s->graphs)
                        if (o.resident && !o.busy) freeable += o.reserved;
                    bool any_resident = false;
                    for (const Entry& o : s->graphs) any_resident |= o.resident || o.building;
                    if (s->reserved - freeable + s->estimate(rq.graph) <= s->budget ||
                        !any_resident) {
                        pick = i;
                        break;
                    }
                }
                if (pick >= 0) break;
                if (next_arrival >= 0) {
                    s->cv.wait_until(lk, t0 + std::chrono::duration_cast<Clock::duration>(
                                                  std::chrono::duration<double>(next_arrival)));
                } else {
                    s->cv.wait_for(lk, std::chrono::milliseconds(50));
                }
            }
            (*taken)[pick] = 1;
            const int32_t gid = reqs[pick].graph;
            Entry& e = s->graphs[gid];
            group[ng++] = pick;
            if (coalesce) {
                // the other requests for this graph that have arrived and wait
                const double now = seconds_since(t0);
                for (int64_t i = pick + 1; i < nreq && ng < MAX_GROUP; ++i) {
                    if (open_loop && reqs[i].arrival_s > now) break;
                    if (!(*taken)[i] && reqs[i].graph == gid) {
                        (*taken)[i] = 1;
                        group[ng++] = i;
                    }
                }
            }
            e.busy = true;
            e.last_use = ++s->tick;
            if (!e.resident) {
                const int64_t need = s->estimate(gid);
                // least recently used idle graphs first
                while (s->reserved + need > s->budget) {
                    int victim = -1;
                    for (int j = 0; j < (int)s->graphs.size(); ++j) {
                        const Entry& o = s->graphs[j];
                        if (o.resident && !o.busy &&
                            (victim < 0 || o.last_use < s->graphs[victim].last_use))
                            victim = j;
                    }
                    if (victim < 0) break;
                    Entry& v = s->graphs[victim];
                    evict.push_back(v.g);
                    v.g = nullptr;
                    v.resident = false;
                    v.indexed = false;
                    v.index_tried = false;
                    s->reserved -= v.reserved;
                    v.reserved = 0;
                    ++s->stats.evictions;
                }
                e.reserved = need;
                e.building = true;
                s->reserved += need;
                need_build = true;
            }
            ++*running;
            s->stats.max_concurrent = std::max<int64_t>(s->stats.max_concurrent, *running);
            s->stats.peak_reserved_bytes = std::max(s->stats.peak_reserved_bytes, s->reserved);
        }
        for (tc_graph* g : evict) release(s, g);
        const tc_request& rq = reqs[pick];
        Entry& e = s->graphs[rq.graph];
        const double start_s = seconds_since(t0);
        int rc = TC_OK;
        if (need_build) {
            rc = build(s, slot, rq.graph);
            std::lock_guard<std::mutex> lk(s->mu);
            e.building = false;
            if (rc == TC_OK) {
                e.resident = true;
                ++s->stats.builds;
            } else {
                s->reserved -= e.reserved;
                e.reserved = 0;
                e.g = nullptr;
            }
        }
        if (rc == TC_OK) rc = execute_group(s, slot, rq.graph, reqs, group, ng, results);
        int64_t held = -1;
        if (rc == TC_OK && !s->fake) {
            tc_graph_info_t info;
            if (tc_graph_info(e.g, &info, slot.stream) == TC_OK) held = info.device_bytes;
        }
        const double done_s = seconds_since(t0);
        for (int i = 0; i < ng; ++i) {
            tc_response& r = out[group[i]];
            r.slot = slot_id;
            r.start_s = start_s;
            r.done_s = done_s;
            r.result = rc == TC_OK ? results[i] : 0;
            r.status = rc;
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            // what the graph holds now (kept supports, lists, truss numbers)
            if (held >= 0 && e.resident) {
                const int64_t now_bytes = std::max(held, s->estimate(rq.graph));
                s->reserved += now_bytes - e.reserved;
                e.reserved = now_bytes;
                s->stats.peak_reserved_bytes = std::max(s->stats.peak_reserved_bytes, s->reserved);
            }
            e.busy = false;
            --*running;
            *left -= ng;
            if (rc != TC_OK) s->stats.errors += ng;
        }
        s->cv.notify_all();
    }
}

}  // namespace

extern "C" {

int tc_server_create(const tc_graph_source* sources, int32_t num_graphs, int64_t budget_bytes,
                     int64_t optional_bytes_per_pair, int32_t slots, tc_server** out) {
    if (!out || (!sources && num_graphs > 0)) return tc::fail(TC_EINVAL, "server: NULL argument");
    if (num_graphs < 0 || slots < 1 || slots > 256 || budget_bytes <= 0 ||
        optional_bytes_per_pair < 0)
        return tc::fail(TC_EINVAL, "server: bad sizes");
    for (int32_t i = 0; i < num_graphs; ++i)
        if (sources[i].n < 1 || sources[i].m_in < 0 ||
            (sources[i].m_in > 0 && (!sources[i].src || !sources[i].dst)))
            return tc::fail(TC_EINVAL, "server: bad graph source " + std::to_string(i));
    tc_server* s = new (std::nothrow) tc_server(num_graphs);
    if (!s) return tc::fail(TC_ENOMEM, "server: host allocation failed");
    s->src.assign(sources, sources + num_graphs);
    s->budget = budget_bytes;
    s->opt_per_pair = optional_bytes_per_pair;
    s->fake = g_server_fake.load() != 0;
    s->slots.resize(slots);
    if (!s->fake) {
        cudaError_t e = cudaGetDevice(&s->device);
        for (int i = 0; e == cudaSuccess && i < slots; ++i)
            e = cudaStreamCreateWithFlags(&s->slots[i].stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaGetLastError();
            tc_server_destroy(s);
            return tc::fail(TC_ECUDA, std::string("server: ") + cudaGetErrorString(e));
        }
    }
    *out = s;
    return TC_OK;
}

int tc_server_run(tc_server* s, const tc_request* reqs, int64_t num_reqs, int32_t open_loop,
                  int32_t slots, tc_response* out, double* wall_s) {
    if (!s || (num_reqs > 0 && (!reqs || !out))) return tc::fail(TC_EINVAL, "server: NULL argument");
    if (slots < 0 || slots > (int32_t)s->slots.size())
        return tc::fail(TC_EINVAL, "server: more slots than the server has");
    const int use = slots == 0 ? (int)s->slots.size() : slots;
    for (int64_t i = 0; i < num_reqs; ++i) {
        const tc_request& r = reqs[i];
        if (r.graph < 0 || r.graph >= (int32_t)s->graphs.size())
            return tc::fail(TC_ERANGE, "server: request " + std::to_string(i) + " names no graph");
        if ((r.kind != TC_REQ_COUNT && r.kind != TC_REQ_KTRUSS) ||
            (r.kind == TC_REQ_KTRUSS && r.k < 2))
            return tc::fail(TC_EINVAL, "server: request " + std::to_string(i) + " is malformed");
        if (open_loop && i > 0 && r.arrival_s < reqs[i - 1].arrival_s)
            return tc::fail(TC_EINVAL, "server: arrivals must not decrease");
        out[i] = tc_response{};
        out[i].status = TC_EINVAL;
        out[i].slot = -1;
    }
    std::vector<char> taken((size_t)num_reqs, 0);
    int64_t head = 0, left = num_reqs, running = 0;
    const int64_t errors0 = s->stats.errors;
    const Clock::time_point t0 = Clock::now();
    std::vector<std::thread> th;
    th.reserve(use);
    for (int i = 0; i < use; ++i)
        th.emplace_back(worker, s, i, reqs, num_reqs, open_loop != 0, use > 1, t0, &taken, &head,
                        &left, &running, out);
    for (auto& t : th) t.join();
    if (wall_s) *wall_s = seconds_since(t0);
    if (!s->fake)
        for (Slot& sl : s->slots) cudaStreamSynchronize(sl.stream);
    return s->stats.errors == errors0 ? TC_OK
                                      : tc::fail(TC_ECUDA, "server: some requests failed (see "
                                                           "their status)");
}

int tc_server_get_stats(const tc_server* s, tc_server_stats* out) {
    if (!s || !out) return tc::fail(TC_EINVAL, "server: NULL argument");
    *out = s->stats;
    out->reserved_bytes = s->reserved;
    int64_t res = 0;
    for (const Entry& e : s->graphs) res += e.resident ? 1 : 0;
    out->resident_graphs = res;
    return TC_OK;
}

void tc_server_destroy(tc_server* s) {
    if (!s) return;
    if (!s->fake) cudaSetDevice(s->device);
    for (Entry& e : s->graphs) release(s, e.resident ? e.g : nullptr);
    for (Slot& sl : s->slots) {
        if (sl.mask) cudaFreeAsync(sl.mask, sl.stream);
        if (sl.stream) {
            cudaStreamSynchronize(sl.stream);
            cudaStreamDestroy(sl.stream);
        }
    }
    delete s;
}

int tc_server_set_result_cache(tc_server* s, int32_t keep) {
    if (!s) return tc::fail(TC_EINVAL, "server: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    s->keep_results = keep != 0;
    for (Entry& e : s->graphs) {
        if (!s->fake && e.resident && e.g) {
            const int rc = tc_graph_set_result_cache(e.g, keep);
            if (rc != TC_OK) return rc;
        }
        if (!s->keep_results) {
            e.indexed = false;
            e.index_tried = false;
        }
    }
    return TC_OK;
}

int tc_debug_server_fake(int on) { return g_server_fake.exchange(on ? 1 : 0); }

}  // extern "C"
