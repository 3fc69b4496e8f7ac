// tc_abi.cu — the extern "C" entry points declared in include/tc.h: argument
// checks, host/device marshalling of caller buffers, the graph object, error
// reporting, and the library's stream-ordered device allocator.
#include <atomic>
#include <cstring>
#include <new>
#include <string>

#include "tc_internal.cuh"


namespace tc {

namespace {
thread_local std::string t_last_error;
std::atomic<int64_t> g_fail_alloc{0};
std::atomic<int64_t> g_spin_ns{2000000000LL};
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_peel_mode{0};
std::atomic<int> g_intersect_mode{0};
}  // namespace

int peel_mode() { return g_peel_mode.load(); }
int intersect_mode() { return g_intersect_mode.load(); }

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int fail(int code, const std::string& what) {
    t_last_error = what;
    return code;
}

int64_t spin_limit_ns() { return g_spin_ns.load(); }

// The library allocates from the device's default stream-ordered pool.  Its
// release threshold is raised once per device so that memory freed by one
// call is kept for the next instead of being unmapped at every
// synchronisation (the peel's scratch runs to gigabytes).
void keep_pool_memory() {
    static std::atomic<unsigned long long> done_mask{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return;
    const unsigned long long bit = 1ull << dev;
    if (done_mask.load() & bit) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done_mask.fetch_or(bit);
}

int dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    keep_pool_memory();
    int64_t c = g_fail_alloc.load();
    while (c > 0) {
        if (g_fail_alloc.compare_exchange_weak(c, c - 1)) {
            if (c == 1) return fail(TC_ENOMEM, "injected device allocation failure");
            break;
        }
    }
    const cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? TC_ENOMEM : TC_ECUDA,
                    std::string("cudaMallocAsync(") + std::to_string(bytes) +
                        " bytes): " + cudaGetErrorString(e));
    }
    return TC_OK;
}

void dev_free(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

bool is_host_pointer(const void* p) {
    cudaPointerAttributes a;
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

// The device's address of host memory the GPU can reach directly (pinned or
// registered memory, mapped into the device's address space), else nullptr
// (pageable memory: the caller copies).  On a GB300's coherent host link a
// kernel reads or writes such memory itself, so inputs and outputs in it
// skip the separate copy pass.
void* host_device_view(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int check_dev_err(int* dev_err, cudaStream_t s) {
    int h = 0;
    TC_CUDA_TRY(cudaMemcpyAsync(&h, dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    if (h == 0) return TC_OK;
    TC_CUDA_TRY(cudaMemsetAsync(dev_err, 0, sizeof(int), s));
    if (h & DEV_ERR_RANGE) return fail(TC_ERANGE, "vertex id outside [0, n)");
    if (h & DEV_ERR_TIMEOUT) return fail(TC_ETIMEDOUT, "a device-side wait ran out of time");
    return fail(TC_ECUDA, "internal device bounds check failed");
}

void free_graph(Graph* g) {
    cudaStream_t s = g->last_stream;
    dev_free(g->lo, s);
    dev_free(g->hi, s);
    dev_free(g->ends, s);
    dev_free(g->rowptr, s);
    dev_free(g->upper, s);
    dev_free(g->col, s);
    dev_free(g->eid, s);
    dev_free(g->inv, s);
    dev_free(g->head, s);
    dev_free(g->iend, s);
    dev_free(g->oshift, s);
    dev_free(g->support, s);
    dev_free(g->tri_off, s);
    dev_free(g->tri_pairs, s);
    dev_free(g->truss_cache, s);
    dev_free(g->kt_state, s);
    dev_free(g->kt_support, s);
    dev_free(g->kt_col, s);
    dev_free(g->kt_eid, s);
    dev_free(g->kt_rowlen, s);
    dev_free(g->dev_err, s);
    dev_free(g->dev_scalars, s);
    cudaStreamSynchronize(s);
}

}  // namespace tc

namespace {

using tc::fail;

struct DeviceGuard {  // makes `dev` current for the scope of a call
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

inline cudaStream_t as_stream(void* p) { return reinterpret_cast<cudaStream_t>(p); }

// Writes `count` elements of device array `src` to the caller's buffer `dst`
// (device or host).  Host destinations synchronise the stream.
template <typename T>
int deliver(T* dst, const T* src, int64_t count, cudaStream_t s) {
    if (count <= 0) return TC_OK;
    const bool host = tc::is_host_pointer(dst);
    TC_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(T) * count,
                                host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    if (host) TC_CUDA_TRY(cudaStreamSynchronize(s));
    return TC_OK;
}

int begin_call(tc_graph* g, void* stream) {
    if (!g) return fail(TC_EINVAL, "graph is NULL");
    g->g.last_stream = as_stream(stream);
    return TC_OK;
}

}  // namespace

extern "C" {

int tc_build_csr(const int32_t* src, const int32_t* dst, int64_t m_in, int32_t n, int flags,
                 void* cuda_stream, tc_graph** out) {
    if (!out) return fail(TC_EINVAL, "out is NULL");
    if (n < 1) return fail(TC_EINVAL, "n must be >= 1");
    if (m_in < 0) return fail(TC_EINVAL, "m_in must be >= 0");
    if (m_in > 0 && (!src || !dst)) return fail(TC_EINVAL, "src/dst is NULL");
    if (flags != TC_INPUT_AUTO && flags != TC_INPUT_DEVICE && flags != TC_INPUT_HOST)
        return fail(TC_EINVAL, "unknown flags");
    if (m_in >= (1ll << 32)) return fail(TC_EOVERFLOW, "m_in must be below 2^32");
    cudaStream_t s = as_stream(cuda_stream);
    int dev = 0;
    TC_CUDA_TRY(cudaGetDevice(&dev));

    bool host = flags == TC_INPUT_HOST;
    if (flags == TC_INPUT_AUTO && m_in > 0) host = tc::is_host_pointer(src) || tc::is_host_pointer(dst);

    tc_graph* h = new (std::nothrow) tc_graph();
    if (!h) return fail(TC_ENOMEM, "host allocation of the graph");
    tc::Graph* g = &h->g;
    g->device = dev;
    g->n = n;
    g->m_in = m_in;
    g->last_stream = s;
    int rc = tc::dev_alloc_n(&g->dev_err, 1, s);
    if (rc == TC_OK) rc = tc::dev_alloc_n(&g->dev_scalars, 8, s);
    if (rc == TC_OK) {
        const int32_t* sd = src;
        const int32_t* dd = dst;
        tc::Scratch sc(s);
        const int32_t* sv = host && m_in > 0 ? static_cast<const int32_t*>(tc::host_device_view(src))
                                              : nullptr;
        const int32_t* dv = host && m_in > 0 ? static_cast<const int32_t*>(tc::host_device_view(dst))
                                              : nullptr;
        if (sv && dv) {  // pinned input: the first kernel reads it in place
            sd = sv;
            dd = dv;
        } else if (host && m_in > 0) {
            int32_t *s2 = nullptr, *d2 = nullptr;
            rc = sc.alloc(&s2, m_in);
            if (rc == TC_OK) rc = sc.alloc(&d2, m_in);
            if (rc == TC_OK) {
                cudaError_t e = cudaMemcpyAsync(s2, src, sizeof(int32_t) * m_in,
                                                cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(d2, dst, sizeof(int32_t) * m_in, cudaMemcpyHostToDevice, s);
                if (e != cudaSuccess)
                    rc = fail(TC_ECUDA, std::string("input copy: ") + cudaGetErrorString(e));
            }
            sd = s2;
            dd = d2;
        }
        if (rc == TC_OK) rc = tc::build_graph(g, sd, dd, s);
    }
    if (rc != TC_OK) {
        tc::free_graph(g);
        delete h;
        return rc;
    }
    *out = h;
    return TC_OK;
}

int tc_count(tc_graph* g, int64_t* triangles_out, void* cuda_stream) {
    TC_TRY(begin_call(g, cuda_stream));
    if (!triangles_out) return fail(TC_EINVAL, "triangles_out is NULL");
    DeviceGuard dg(g->g.device);
    // the graph is immutable: once its supports are computed, T is known
    // (a kernel forced by the test hook is always run)
    if (g->g.triangles >= 0 && tc::intersect_mode() == 0) {
        *triangles_out = g->g.triangles;
        return TC_OK;
    }
    int64_t T = 0;
    TC_TRY(tc::compute_support(&g->g, nullptr, false, &T, as_stream(cuda_stream)));
    g->g.triangles = T;
    *triangles_out = T;
    return TC_OK;
}

int tc_edge_support(tc_graph* g, int32_t* support_out, int64_t* triangles_out,
                    void* cuda_stream) {
    TC_TRY(begin_call(g, cuda_stream));
    tc::Graph* gg = &g->g;
    if (!support_out && gg->m > 0) return fail(TC_EINVAL, "support_out is NULL");
    DeviceGuard dg(gg->device);
    cudaStream_t s = as_stream(cuda_stream);
    // computed once per graph and kept (the peel starts from them too); a
    // kernel forced by the test hook is always run
    const bool need_T = triangles_out && gg->triangles < 0;
    if (!gg->support_valid || need_T || tc::intersect_mode() != 0) {
        if (!gg->support) TC_TRY(tc::dev_alloc_n(&gg->support, gg->m, s));
        gg->support_valid = false;
        int64_t T = 0;
        // without triangles_out the call stays asynchronous (T not read back)
        TC_TRY(tc::compute_support(gg, gg->support, true, triangles_out ? &T : nullptr, s));
        if (triangles_out) gg->triangles = T;
        gg->support_valid = true;
    }
    if (triangles_out) *triangles_out = gg->triangles;
    // the cached supports are in internal edge order: gather them by edge id
    if (gg->m == 0) return TC_OK;
    if (!tc::is_host_pointer(support_out))
        return tc::to_canonical_i32(gg->support, gg->inv, gg->m, support_out, s);
    if (void* v = tc::host_device_view(support_out)) {  // pinned: written in place
        TC_TRY(tc::to_canonical_i32(gg->support, gg->inv, gg->m, static_cast<int32_t*>(v), s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
        return TC_OK;
    }
    tc::Scratch sc(s);
    int32_t* tmp;
    TC_TRY(sc.alloc(&tmp, gg->m));
    TC_TRY(tc::to_canonical_i32(gg->support, gg->inv, gg->m, tmp, s));
    return deliver(support_out, tmp, gg->m, s);
}

int ktruss(tc_graph* g, int32_t k, uint8_t* mask_out, int64_t* edges_out, void* cuda_stream) {
    TC_TRY(begin_call(g, cuda_stream));
    if (k < 2) return fail(TC_EINVAL, "k must be >= 2");
    tc::Graph* gg = &g->g;
    if (!mask_out && gg->m > 0) return fail(TC_EINVAL, "mask_out is NULL");
    DeviceGuard dg(gg->device);
    cudaStream_t s = as_stream(cuda_stream);
    bool host = gg->m > 0 && tc::is_host_pointer(mask_out);
    tc::Scratch sc(s);
    uint8_t* mask = mask_out;
    if (host) {
        if (void* v = tc::host_device_view(mask_out)) {  // pinned: written in place
            mask = static_cast<uint8_t*>(v);
            host = false;
        } else {
            TC_TRY(sc.alloc(&mask, gg->m));
        }
    }
    int64_t left = 0;
    TC_TRY(tc::peel_ktruss(gg, k, mask, &left, s));
    if (host) TC_TRY(deliver(mask_out, mask, gg->m, s));
    if (edges_out) *edges_out = left;
    return tc::check_dev_err(gg->dev_err, s);
}

int ktruss_components(tc_graph* g, int32_t k, int32_t* edge_label_out, int32_t* vertex_label_out,
                      int64_t* count_out, void* cuda_stream) {
    TC_TRY(begin_call(g, cuda_stream));
    if (k < 2) return fail(TC_EINVAL, "k must be >= 2");
    if (!count_out) return fail(TC_EINVAL, "count_out is NULL");
    tc::Graph* gg = &g->g;
    if (!edge_label_out && gg->m > 0) return fail(TC_EINVAL, "edge_label_out is NULL");
    DeviceGuard dg(gg->device);
    cudaStream_t s = as_stream(cuda_stream);
    tc::Scratch sc(s);
    int32_t* el = edge_label_out;
    int32_t* vl = vertex_label_out;
    const bool host_e = gg->m > 0 && tc::is_host_pointer(edge_label_out);
    const bool host_v = vertex_label_out && tc::is_host_pointer(vertex_label_out);
    if (host_e) TC_TRY(sc.alloc(&el, gg->m));
    if (host_v) TC_TRY(sc.alloc(&vl, gg->n));
    TC_TRY(tc::truss_components(gg, k, el, vl, count_out, s));
    if (host_e) TC_TRY(deliver(edge_label_out, el, gg->m, s));
    if (host_v) TC_TRY(deliver(vertex_label_out, vl, (int64_t)gg->n, s));
    return tc::check_dev_err(gg->dev_err, s);
}

int ktruss_max(tc_graph* g, int32_t* kmax_out, int32_t* truss_out, void* cuda_stream) {
    TC_TRY(begin_call(g, cuda_stream));
    if (!kmax_out) return fail(TC_EINVAL, "kmax_out is NULL");
    tc::Graph* gg = &g->g;
    DeviceGuard dg(gg->device);
    cudaStream_t s = as_stream(cuda_stream);
    tc::Scratch sc(s);
    int32_t* truss = truss_out;
    bool direct = truss_out && gg->m > 0 && !tc::is_host_pointer(truss_out);
    if (!direct && truss_out && gg->m > 0) {
        if (void* v = tc::host_device_view(truss_out)) {  // pinned: written in place
            truss = static_cast<int32_t*>(v);
            direct = true;
        }
    }
    if (!direct) TC_TRY(sc.alloc(&truss, gg->m));
    int32_t kmax = 0;
    TC_TRY(tc::peel_decompose(gg, truss, &kmax, s));
    if (truss_out && !direct) TC_TRY(deliver(truss_out, truss, gg->m, s));
    TC_TRY(tc::check_dev_err(gg->dev_err, s));
    *kmax_out = kmax;
    return TC_OK;
}

int ktruss_sizes(tc_graph* g, int32_t k_lo, int32_t k_hi, int64_t* sizes_out, void* cuda_stream) {
    TC_TRY(begin_call(g, cuda_stream));
    if (!sizes_out) return fail(TC_EINVAL, "sizes_out is NULL");
    if (k_lo < 2 || k_hi < k_lo || k_hi - k_lo >= 64)
        return fail(TC_EINVAL, "ktruss_sizes: need 2 <= k_lo <= k_hi < k_lo + 64");
    tc::Graph* gg = &g->g;
    DeviceGuard dg(gg->device);
    cudaStream_t s = as_stream(cuda_stream);
    TC_TRY(tc::peel_sizes(gg, k_lo, k_hi, sizes_out, s));
    return tc::check_dev_err(gg->dev_err, s);
}

int64_t tc_num_edges(const tc_graph* g) { return g ? g->g.m : -1; }

int32_t tc_num_vertices(const tc_graph* g) { return g ? g->g.n : -1; }

int tc_edges(const tc_graph* g, int32_t* lo, int32_t* hi, void* cuda_stream) {
    if (!g) return fail(TC_EINVAL, "graph is NULL");
    if (g->g.m > 0 && (!lo || !hi)) return fail(TC_EINVAL, "lo/hi is NULL");
    DeviceGuard dg(g->g.device);
    cudaStream_t s = as_stream(cuda_stream);
    TC_TRY(deliver(lo, g->g.lo, g->g.m, s));
    return deliver(hi, g->g.hi, g->g.m, s);
}

int tc_graph_info(const tc_graph* g, tc_graph_info_t* info, void* cuda_stream) {
    if (!g || !info) return fail(TC_EINVAL, "graph or info is NULL");
    tc::Graph* gg = const_cast<tc::Graph*>(&g->g);
    (void)cuda_stream;
    const int64_t ww = gg->wedge_work;
    info->n = gg->n;
    info->m_in = gg->m_in;
    info->m = gg->m;
    info->max_degree = gg->max_deg;
    info->max_out = gg->max_out;
    info->wedge_work = ww;
    const int64_t m = gg->m, n = gg->n;
    // lo, hi, ends, inv (m each) and col, eid (2m each); rowptr, upper, oshift
    info->device_bytes = m * (4 + 4 + 8 + 4 + 8 + 8 + 8) + 8 * (n + 1) + 8 * n + 8 * n +
                         (gg->support ? 4 * m : 0) +
                         (gg->tri_valid ? 8 * (m + 1) + 8 * gg->tri_entries : 0) +
                         (gg->kt_state ? 8 * m : 0) + (gg->truss_cache ? 4 * m : 0) + (gg->kt_col ? 16 * m + 4 * n : 0);
    info->peel_rounds = gg->last_peel_rounds;
    info->peel_lists = gg->last_peel_lists;
    info->count_kernel_ns = gg->stats.count_ns;
    info->support_kernel_ns = gg->stats.support_ns;
    info->lists_kernel_ns = gg->stats.lists_ns;
    info->peel_kernel_ns = gg->stats.peel_ns;
    info->peel_bytes = gg->stats.peel_bytes;
    info->peel_scanned = gg->stats.peel_scanned;
    info->peel_entries = gg->stats.peel_entries;
    info->peel_searches = gg->stats.peel_searches;
    info->peel_lookups = gg->stats.peel_lookups;
    info->peel_lowered = gg->stats.peel_lowered;
    info->truss_cached = gg->truss_valid ? 1 : 0;
    info->column_work = gg->column_work;
    info->product_form = gg->stats.product_form;
    info->lists_bytes = gg->stats.lists_bytes;
    return TC_OK;
}

int tc_graph_wedge_work(tc_graph* g, int64_t* out, void* cuda_stream) {
    TC_TRY(begin_call(g, cuda_stream));
    if (!out) return fail(TC_EINVAL, "out is NULL");
    DeviceGuard dg(g->g.device);
    return tc::graph_wedge_work(&g->g, out, as_stream(cuda_stream));
}

int tc_graph_set_memory_limit(tc_graph* g, int64_t bytes) {
    if (!g) return fail(TC_EINVAL, "graph is NULL");
    g->g.mem_limit = bytes < 0 ? -1 : bytes;
    return TC_OK;
}

int tc_graph_set_result_cache(tc_graph* g, int32_t keep) {
    if (!g) return fail(TC_EINVAL, "graph is NULL");
    DeviceGuard dg(g->g.device);
    tc::Graph* gg = &g->g;
    gg->keep_results = keep != 0;
    if (!gg->keep_results) {
        cudaStream_t s = gg->last_stream;
        tc::dev_free(gg->truss_cache, s);
        tc::dev_free(gg->kt_state, s);
        tc::dev_free(gg->kt_support, s);
        tc::dev_free(gg->kt_col, s);
        tc::dev_free(gg->kt_eid, s);
        tc::dev_free(gg->kt_rowlen, s);
        gg->truss_cache = nullptr;
        gg->kt_state = gg->kt_support = nullptr;
        gg->kt_col = gg->kt_eid = gg->kt_rowlen = nullptr;
        gg->truss_valid = false;
        gg->kt_k = 0;
        gg->kt_adj = false;
    }
    return TC_OK;
}

int64_t tc_launch_count(void) { return tc::g_launches.load(); }

void tc_graph_free(tc_graph* g) {
    if (!g) return;
    {
        DeviceGuard dg(g->g.device);
        tc::free_graph(&g->g);
    }
    delete g;
}

const char* tc_strerror(int code) {
    switch (code) {
        case TC_OK: return "ok";
        case TC_EINVAL: return "invalid argument";
        case TC_ERANGE: return "vertex id out of range";
        case TC_ENOMEM: return "out of memory";
        case TC_ECUDA: return "CUDA error";
        case TC_ETIMEDOUT: return "device-side wait timed out";
        case TC_EOVERFLOW: return "size overflow";
        default: return "unknown error";
    }
}

const char* tc_last_error(void) { return tc::t_last_error.c_str(); }

int64_t tc_debug_fail_alloc(int64_t nth) { return tc::g_fail_alloc.exchange(nth < 0 ? 0 : nth); }

int tc_debug_intersect_mode(int mode) {
    if (mode < 0 || mode > 4) return tc::g_intersect_mode.load();
    return tc::g_intersect_mode.exchange(mode);
}

int tc_debug_peel_mode(int mode) {
    if (mode < 0 || mode > 3) return tc::g_peel_mode.load();
    return tc::g_peel_mode.exchange(mode);
}

int64_t tc_debug_spin_limit_ns(int64_t ns) {
    if (ns <= 0) return tc::g_spin_ns.load();
    return tc::g_spin_ns.exchange(ns);
}

}  // extern "C"
