// batch.cu — many independent graphs in one pass.
//
// The disjoint union of the batch's graphs is itself a graph, and its
// triangles and k-trusses are exactly those of the individual graphs (a
// triangle or a truss never spans two components).  So the batch is cleaned
// and built as one graph whose vertex ids are offset per graph, and every
// phase — supports (Algorithm 4's s), per-graph triangle counts (Section
// III-A), the k-truss peel (Section III-B) and per-graph truss sizes — is one
// launch over all graphs.  The query phase can be captured into one CUDA
// graph and launched once.  An autotuner picks the masked-product kernel,
// the peel form and the peel's grid size by timing them on the batch, and
// caches the choice by a signature of the union graph's size and degree
// classes.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "tc_internal.cuh"

namespace tc {
namespace {

// Global vertex id of every endpoint; local ids outside [0, n_g) flag
// DEV_ERR_RANGE.  The graph of edge i is found by binary search in the
// edge offsets.
__global__ void k_remap(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                        int64_t m_in, const int64_t* __restrict__ eoff,
                        const int64_t* __restrict__ voff, int32_t G, int32_t* __restrict__ gsrc,
                        int32_t* __restrict__ gdst, int* __restrict__ err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_in; i += stride) {
        int32_t lo = 0, hi = G;  // last g with eoff[g] <= i
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (eoff[mid] <= i) lo = mid;
            else hi = mid;
        }
        const int64_t base = voff[lo], nv = voff[lo + 1] - voff[lo];
        const int32_t u = src[i], v = dst[i];
        if (u < 0 || u >= nv || v < 0 || v >= nv) {
            bad = true;
            gsrc[i] = 0;
            gdst[i] = 0;
        } else {
            gsrc[i] = (int32_t)(base + u);
            gdst[i] = (int32_t)(base + v);
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, DEV_ERR_RANGE);
}

// First canonical edge of each graph: edges are sorted by (lo, hi) in global
// ids and each graph's vertices are a contiguous id range.
__global__ void k_graph_edge_ranges(const int32_t* __restrict__ lo, int64_t m,
                                    const int64_t* __restrict__ voff, int32_t G,
                                    int64_t* __restrict__ ge) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += stride) {
        if (g == G) {
            ge[G] = m;
            continue;
        }
        const int64_t key = voff[g];
        int64_t a = 0, b = m;
        while (a < b) {
            const int64_t mid = (a + b) >> 1;
            if ((int64_t)lo[mid] < key) a = mid + 1;
            else b = mid;
        }
        ge[g] = a;
    }
}

// Per-graph sums over contiguous canonical edge ranges, one warp per graph:
// MODE 0: sum of supports / 3 (triangles); MODE 1: k-truss mask bytes.
template <int MODE, typename T>
__global__ void k_segment_sums(const T* __restrict__ x, const int64_t* __restrict__ ge,
                               int32_t G, long long* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = w0; g < G; g += nw) {
        unsigned long long acc = 0;
        for (int64_t e = ge[g] + lane; e < ge[g + 1]; e += 32)
            acc += (unsigned long long)x[e];
        acc = warp_sum(acc);
        if (lane == 0) out[g] = MODE == 0 ? (long long)(acc / 3) : (long long)acc;
    }
}

struct Choice {
    int intersect = 1;    // 1 columns, 2 edge-per-warp, 3 edge-per-thread, 4 rows
    int light = LIGHT_DEG;  // columns: the degree bound of warp-per-column (light) columns
    int peel = PEEL_AUTO;
    int peel_blocks = 0;  // cap on the peel's grid (0 = its own rule)
};
std::mutex g_tune_mu;
std::map<uint64_t, Choice> g_tune;

uint64_t signature(const Graph* g, int32_t k) {
    return ((uint64_t)bits_for((uint64_t)g->m) << 40) | ((uint64_t)bits_for(g->max_out) << 32) |
           ((uint64_t)bits_for(g->max_deg) << 24) | (uint64_t)std::min(k, 255);
}

unsigned grid_items(int64_t n, int per = 256) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per,
                                                            (int64_t)num_sms() * 16));
}

// Times each candidate on the batch itself and keeps the fastest.  The
// peel candidates must agree on the number of surviving edges.
int autotune(Graph* g, int32_t k, Choice* c, cudaStream_t s) {
    // masked-product kernel and, for the column kernel, the degree bucket
    // boundary: columns up to `light` take a warp each, heavier ones a block
    struct Cand {
        int form, light;
    };
    const Cand cands[] = {{1, 32}, {1, 64}, {1, LIGHT_DEG}, {4, 0}, {2, 0}, {3, 0}};
    int64_t best_ns = -1;
    for (const Cand& cd : cands) {
        if ((cd.form == 1 || cd.form == 4) && !triangle_lists_supported(g)) continue;  // table size
        if (cd.form == 1 && cd.light > LIGHT_DEG) continue;
        if (cd.form == 3 && g->max_out > 64) continue;  // merges grow with the out-lists
        g->col_light_deg = cd.form == 1 ? cd.light : LIGHT_DEG;
        int64_t T = 0;
        TC_TRY(compute_support(g, g->support, true, &T, s, cd.form));
        g->triangles = T;
        g->support_valid = true;
        const int64_t ns = g->stats.support_ns;
        if (best_ns < 0 || (ns >= 0 && ns < best_ns)) {
            best_ns = ns;
            c->intersect = cd.form;
            c->light = cd.form == 1 ? cd.light : LIGHT_DEG;
        }
    }
    g->col_light_deg = c->light;
    if (k < 2) return TC_OK;
    // peel form
    best_ns = -1;
    int64_t left_ref = -1;
    Scratch sc(s);
    int32_t* t;
    TC_TRY(sc.alloc(&t, g->m));
    // peel form and grid: the full grid, half and a quarter of the SMs
    // (the peel is latency-bound, so a smaller grid with cheaper barriers can win)
    const int grids[3] = {0, std::max(1, num_sms() / 2), std::max(1, num_sms() / 4)};
    for (int trial = 0; trial < 6; ++trial) {
        const int form = trial < 3 ? PEEL_LISTS : PEEL_INTERSECT;
        const int cap = grids[trial % 3];
        PeelPlan* p = peel_plan_new();
        if (!p) return fail(TC_ENOMEM, "peel plan");
        int64_t left = 0;
        int rc;
        {
            Scratch psc(s);
            rc = peel_plan(p, psc, g, k, true, t, form, false, false, cap);
            const bool skip = rc == TC_OK && form == PEEL_LISTS && !peel_uses_lists(p);
            if (rc == TC_OK && !skip) {
                rc = peel_enqueue(p, s);
                if (rc == TC_OK) rc = peel_finish(p, s, &left, nullptr);
                if (rc == TC_OK) {
                    if (left_ref >= 0 && left != left_ref)
                        rc = fail(TC_ECUDA, "autotune: peel forms disagree");
                    left_ref = left;
                    const int64_t ns = g->stats.peel_ns +
                                       (form == PEEL_LISTS ? std::max<int64_t>(0, g->stats.lists_ns) : 0);
                    if (best_ns < 0 || ns < best_ns) {
                        best_ns = ns;
                        c->peel = form;
                        c->peel_blocks = cap;
                    }
                }
            }
        }
        peel_plan_delete(p);
        TC_TRY(rc);
    }
    return TC_OK;
}

}  // namespace

int batch_run(const tc_batch_desc* d, cudaStream_t user_stream) {
    const int32_t G = d->num_graphs;
    if (G < 1 || !d->n || !d->edge_off || !d->triangles_out)
        return fail(TC_EINVAL, "batch: num_graphs, n, edge_off and triangles_out are required");
    if (d->k != 0 && d->k < 2) return fail(TC_EINVAL, "batch: k must be 0 or >= 2");
    std::vector<int64_t> voff(G + 1, 0);
    for (int32_t g = 0; g < G; ++g) {
        if (d->n[g] < 1) return fail(TC_EINVAL, "batch: every graph needs n >= 1");
        if (d->edge_off[g + 1] < d->edge_off[g]) return fail(TC_EINVAL, "batch: edge_off decreases");
        voff[g + 1] = voff[g] + d->n[g];
    }
    if (d->edge_off[0] != 0) return fail(TC_EINVAL, "batch: edge_off[0] must be 0");
    if (voff[G] > 0x7fffffffLL) return fail(TC_EOVERFLOW, "batch: more than 2^31-1 vertices");
    const int64_t m_in = d->edge_off[G];
    if (m_in > 0 && (!d->src || !d->dst)) return fail(TC_EINVAL, "batch: src/dst is NULL");
    if (m_in >= (1ll << 32)) return fail(TC_EOVERFLOW, "batch: 2^32 or more input pairs");

    // the legacy default stream cannot be captured: run on a private stream then
    cudaStream_t s = user_stream;
    cudaStream_t own = nullptr;
    if (s == nullptr || s == cudaStreamLegacy) {
        TC_CUDA_TRY(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
        s = own;
    }
    struct StreamGuard {
        cudaStream_t st;
        ~StreamGuard() {
            if (st) {
                cudaStreamSynchronize(st);
                cudaStreamDestroy(st);
            }
        }
    } sguard{own};

    Graph g;
    g.n = (int32_t)voff[G];
    g.m_in = m_in;
    g.last_stream = s;
    cudaGetDevice(&g.device);
    struct GraphGuard {
        Graph* g;
        ~GraphGuard() { free_graph(g); }
    } gguard{&g};
    TC_TRY(dev_alloc_n(&g.dev_err, 1, s));
    TC_TRY(dev_alloc_n(&g.dev_scalars, 8, s));

    KernelTimer build_timer;
    TC_TRY(build_timer.start(s));
    {
        Scratch sc(s);
        int64_t *eoff_d, *voff_d;
        TC_TRY(sc.alloc(&eoff_d, G + 1));
        TC_TRY(sc.alloc(&voff_d, G + 1));
        TC_CUDA_TRY(cudaMemcpyAsync(eoff_d, d->edge_off, sizeof(int64_t) * (G + 1),
                                    cudaMemcpyHostToDevice, s));
        TC_CUDA_TRY(cudaMemcpyAsync(voff_d, voff.data(), sizeof(int64_t) * (G + 1),
                                    cudaMemcpyHostToDevice, s));
        const int32_t* src = d->src;
        const int32_t* dst = d->dst;
        int32_t *gsrc = nullptr, *gdst = nullptr;
        TC_TRY(sc.alloc(&gsrc, m_in));
        TC_TRY(sc.alloc(&gdst, m_in));
        if (m_in > 0 && (is_host_pointer(src) || is_host_pointer(dst))) {
            int32_t *s2, *d2;
            TC_TRY(sc.alloc(&s2, m_in));
            TC_TRY(sc.alloc(&d2, m_in));
            TC_CUDA_TRY(cudaMemcpyAsync(s2, src, 4 * m_in, cudaMemcpyHostToDevice, s));
            TC_CUDA_TRY(cudaMemcpyAsync(d2, dst, 4 * m_in, cudaMemcpyHostToDevice, s));
            src = s2;
            dst = d2;
        }
        TC_CUDA_TRY(cudaMemsetAsync(g.dev_err, 0, sizeof(int), s));
        if (m_in > 0) {
            k_remap<<<grid_items(m_in), 256, 0, s>>>(src, dst, m_in, eoff_d, voff_d, G, gsrc, gdst,
                                                     g.dev_err);
            TC_LAUNCH_CHECK("k_remap");
            TC_TRY(check_dev_err(g.dev_err, s));
        }
        TC_TRY(build_graph(&g, gsrc, gdst, s));
    }
    TC_TRY(build_timer.stop(s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));

    // per-graph edge ranges and outputs on the device
    Scratch sc(s);
    int64_t *voff_d, *ge;
    long long *tri_d, *left_d;
    int32_t* sup_can;       // supports in canonical order (graphs are contiguous there)
    uint8_t* mask_can;      // k-truss mask in canonical order
    TC_TRY(sc.alloc(&sup_can, g.m));
    TC_TRY(sc.alloc(&mask_can, g.m));
    TC_TRY(sc.alloc(&voff_d, G + 1));
    TC_TRY(sc.alloc(&ge, G + 1));
    TC_TRY(sc.alloc(&tri_d, G));
    TC_TRY(sc.alloc(&left_d, G));
    TC_CUDA_TRY(cudaMemcpyAsync(voff_d, voff.data(), sizeof(int64_t) * (G + 1),
                                cudaMemcpyHostToDevice, s));
    k_graph_edge_ranges<<<grid_items(G + 1), 256, 0, s>>>(g.lo, g.m, voff_d, G, ge);
    TC_LAUNCH_CHECK("k_graph_edge_ranges");
    TC_TRY(dev_alloc_n(&g.support, g.m, s));

    // autotuned kernel forms (cached by signature); the trials also leave
    // valid supports and T, which size the peel's plan
    Choice choice;
    bool cached = false;
    const uint64_t sig = signature(&g, d->k);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(sig);
        if (it != g_tune.end()) {
            choice = it->second;
            cached = true;
        }
    }
    if (!cached && g.m > 0) {
        TC_TRY(autotune(&g, d->k, &choice, s));
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[sig] = choice;
    } else if (g.m > 0) {
        g.col_light_deg = choice.light;
        if (d->k >= 2 && choice.peel != PEEL_INTERSECT) {
            // the triangle-list form is sized by T: count before planning
            int64_t T = 0;
            TC_TRY(compute_support(&g, g.support, true, &T, s, choice.intersect));
            g.triangles = T;
        }
        // otherwise the supports are computed inside the query, ahead of the
        // peel on the same stream; the plan needs no count
        g.support_valid = true;
    }

    // plan the query (every allocation happens here, outside any capture)
    const bool peel = d->k >= 2 && g.m > 0;
    int32_t* t = nullptr;
    PeelPlan* plan = nullptr;
    struct PlanGuard {
        PeelPlan* p;
        ~PlanGuard() {
            if (p) peel_plan_delete(p);
        }
    } pguard{nullptr};
    if (peel) {
        TC_TRY(sc.alloc(&t, g.m));
        plan = peel_plan_new();
        if (!plan) return fail(TC_ENOMEM, "peel plan");
        pguard.p = plan;
        TC_TRY(peel_plan(plan, sc, &g, d->k, true, t, choice.peel, false, false,
                         choice.peel_blocks));
    }
    KernelTimer query_timer;
    auto enqueue_query = [&]() -> int {
        if (g.m > 0) {
            TC_TRY(compute_support(&g, g.support, true, nullptr, s, choice.intersect));
            TC_TRY(to_canonical_i32(g.support, g.inv, g.m, sup_can, s));
            k_segment_sums<0, int32_t><<<grid_items((int64_t)G * 32), 256, 0, s>>>(sup_can, ge, G,
                                                                                  tri_d);
            TC_LAUNCH_CHECK("k_segment_sums");
        } else {
            TC_CUDA_TRY(cudaMemsetAsync(tri_d, 0, sizeof(long long) * G, s));
        }
        if (peel) {
            TC_TRY(peel_enqueue(plan, s));
            TC_TRY(mask_from_state(t, g.inv, g.m, mask_can, s));
            k_segment_sums<1, uint8_t><<<grid_items((int64_t)G * 32), 256, 0, s>>>(mask_can, ge, G,
                                                                                  left_d);
            TC_LAUNCH_CHECK("k_segment_sums");
        }
        return TC_OK;
    };
    if (d->use_graph) {
        cudaGraph_t cg = nullptr;
        cudaGraphExec_t ge_exec = nullptr;
        TC_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        const int rc = enqueue_query();
        const cudaError_t ec = cudaStreamEndCapture(s, &cg);
        if (rc != TC_OK) {
            if (cg) cudaGraphDestroy(cg);
            return rc;
        }
        if (ec != cudaSuccess) return fail(TC_ECUDA, std::string("capture: ") + cudaGetErrorString(ec));
        const cudaError_t ei = cudaGraphInstantiate(&ge_exec, cg, 0);
        cudaGraphDestroy(cg);
        if (ei != cudaSuccess)
            return fail(TC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
        TC_TRY(query_timer.start(s));
        const cudaError_t el = cudaGraphLaunch(ge_exec, s);
        count_launch();
        TC_TRY(query_timer.stop(s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
        cudaGraphExecDestroy(ge_exec);
        if (el != cudaSuccess) return fail(TC_ECUDA, std::string("graph launch: ") + cudaGetErrorString(el));
    } else {
        TC_TRY(query_timer.start(s));
        TC_TRY(enqueue_query());
        TC_TRY(query_timer.stop(s));
    }
    int64_t left_total = 0;
    if (peel) TC_TRY(peel_finish(plan, s, &left_total, nullptr));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    TC_TRY(check_dev_err(g.dev_err, s));

    // outputs
    std::vector<int64_t> ge_h(G + 1);
    TC_CUDA_TRY(cudaMemcpyAsync(ge_h.data(), ge, sizeof(int64_t) * (G + 1), cudaMemcpyDeviceToHost, s));
    std::vector<long long> tri_h(G), left_h(G, 0);
    TC_CUDA_TRY(cudaMemcpyAsync(tri_h.data(), tri_d, sizeof(long long) * G, cudaMemcpyDeviceToHost, s));
    if (peel)
        TC_CUDA_TRY(cudaMemcpyAsync(left_h.data(), left_d, sizeof(long long) * G,
                                    cudaMemcpyDeviceToHost, s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t tri_total = 0;
    for (int32_t i = 0; i < G; ++i) {
        d->triangles_out[i] = tri_h[i];
        tri_total += tri_h[i];
        if (d->edges_out) d->edges_out[i] = ge_h[i + 1] - ge_h[i];
        if (d->truss_edges_out) d->truss_edges_out[i] = peel ? left_h[i] : (ge_h[i + 1] - ge_h[i]);
    }
    if (d->stats_out) {
        tc_batch_stats_t* st = d->stats_out;
        st->build_ns = build_timer.elapsed_ns();
        st->query_ns = query_timer.elapsed_ns();
        st->m = g.m;
        st->triangles = tri_total;
        st->intersect_form = choice.intersect;
        st->peel_form = peel ? (peel_uses_lists(plan) ? 1 : 2) : 0;
        st->peel_blocks = peel ? choice.peel_blocks : 0;
        st->light_degree = choice.intersect == 1 ? choice.light : 0;
        st->tuned_from_cache = cached ? 1 : 0;
        st->captured = d->use_graph ? 1 : 0;
    }
    return TC_OK;
}

}  // namespace tc

extern "C" int tc_batch_run(const tc_batch_desc* d, void* cuda_stream) {
    if (!d) return tc::fail(TC_EINVAL, "batch descriptor is NULL");
    return tc::batch_run(d, reinterpret_cast<cudaStream_t>(cuda_stream));
}
