// tc_internal.cuh — shared declarations of the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/tc.h"

namespace tc {

// ---------------------------------------------------------------- errors

// Records a failure for tc_last_error() and returns `code`.
int fail(int code, const std::string& what);

#define TC_CUDA_TRY(expr)                                                              \
    do {                                                                               \
        cudaError_t err__ = (expr);                                                    \
        if (err__ != cudaSuccess)                                                      \
            return ::tc::fail(err__ == cudaErrorMemoryAllocation ? TC_ENOMEM : TC_ECUDA, \
                              std::string(#expr) + ": " + cudaGetErrorString(err__));  \
    } while (0)

#define TC_TRY(expr)                 \
    do {                             \
        int rc__ = (expr);           \
        if (rc__ != TC_OK) return rc__; \
    } while (0)

// Every kernel launch is followed by this check, which also counts it.
void count_launch();
#define TC_LAUNCH_CHECK(name)            \
    do {                                 \
        ::tc::count_launch();            \
        TC_CUDA_TRY(cudaGetLastError()); \
    } while (0)

// Device-side error word: kernels OR these bits into it, the host maps them.
enum : int {
    DEV_ERR_RANGE = 1,     // vertex id outside [0, n)
    DEV_ERR_TIMEOUT = 2,   // a bounded spin wait gave up
    DEV_ERR_BOUNDS = 4,    // an internal index check failed (a library bug)
};

int64_t spin_limit_ns();

// Columns of the masked product whose vertex has at most this degree are
// processed by one warp each (warp-private table); the others by one block.
#ifndef TC_LIGHT_DEG
#define TC_LIGHT_DEG 128
#endif
constexpr int LIGHT_DEG = TC_LIGHT_DEG;

// Which form of the peel to use (test hook; PEEL_AUTO by default).
// PEEL_HYBRID: triangle lists for the edges whose support is below
// LIST_BOUND, intersections of live neighbour lists for the others.
enum : int { PEEL_AUTO = 0, PEEL_LISTS = 1, PEEL_INTERSECT = 2, PEEL_HYBRID = 3 };
#ifndef TC_LIST_BOUND
#define TC_LIST_BOUND 8
#endif
constexpr int LIST_BOUND = TC_LIST_BOUND;
int peel_mode();
// Which count/support kernel to use (test hook): 0 automatic, 1 column
// kernel where the graph allows it, 2 edge-per-warp binary search, 3 thread
// per edge, 4 row kernel where the graph allows it.
int intersect_mode();

// ---------------------------------------------------------------- memory

// Stream-ordered device allocation with the fault-injection hook.
int dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

template <typename T>
int dev_alloc_n(T** p, int64_t count, cudaStream_t s) {
    return dev_alloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)(count > 0 ? count : 1), s);
}

// RAII holder for scratch buffers freed (stream-ordered) at scope exit.
struct Scratch {
    static constexpr int kMax = 48;
    cudaStream_t s;
    void* ptrs[kMax];
    int n = 0;
    explicit Scratch(cudaStream_t st) : s(st) {}
    template <typename T>
    int alloc(T** p, int64_t count) {
        if (n == kMax) return fail(TC_ENOMEM, "internal: too many scratch buffers");
        int rc = dev_alloc_n(p, count, s);
        if (rc == TC_OK) ptrs[n++] = *p;
        return rc;
    }
    ~Scratch() {
        for (int i = 0; i < n; ++i) dev_free(ptrs[i], s);
    }
};

// Pointer location: true if `p` is host memory the device cannot address
// directly as device memory (pageable, or pinned/registered host memory).
bool is_host_pointer(const void* p);
void* host_device_view(const void* p);  // device address of pinned host memory, else nullptr

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Relaxed (coherent, unordered) 64-bit load and store: for flag words that
// carry their whole message, so no other memory needs ordering with them.
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v));
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide exclusive scan of one uint32 per thread (blockDim.x <= 1024,
// a multiple of 32).  `sh` must hold 33 entries of shared memory.  Returns the
// exclusive prefix; *total receives the block sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* sh,
                                                         uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < nwarps ? sh[lane] : 0u;
        uint32_t tt = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, tt, o);
            if (lane >= o) tt += y;
        }
        if (lane < nwarps) sh[lane] = tt - t;
        if (lane == 31) sh[32] = tt;
    }
    __syncthreads();
    const uint32_t res = sh[warp] + x - v;
    *total = sh[32];
    __syncthreads();
    return res;
}

inline int num_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

inline int bits_for(uint64_t maxval) {  // bits needed to hold values 0..maxval (>= 1)
    int b = 1;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b;
}

// Times one kernel launch with CUDA events on the launching stream.
struct KernelTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    int start(cudaStream_t s) {
        TC_CUDA_TRY(cudaEventCreate(&a));
        TC_CUDA_TRY(cudaEventCreate(&b));
        TC_CUDA_TRY(cudaEventRecord(a, s));
        return TC_OK;
    }
    int stop(cudaStream_t s) {
        TC_CUDA_TRY(cudaEventRecord(b, s));
        return TC_OK;
    }
    // valid once the stream has passed the stop event
    int64_t elapsed_ns() {
        float ms = 0.f;
        if (a && b && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) return (int64_t)(ms * 1e6);
        cudaGetLastError();
        return -1;
    }
    ~KernelTimer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// ---------------------------------------------------------------- primitives

// LSD radix sort of uint64 keys on bits [0, key_bits), stable, optionally
// carrying uint32 values.  keys/vals are sorted in place (alt buffers are
// scratch of the same size, provided by the caller).  vals may be NULL.
int radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                   int64_t n, int key_bits, int* dev_err, cudaStream_t s);

// Exclusive scan of `count` uint32 block totals in place (one kernel).
int scan_block_totals(uint32_t* totals, int64_t count, uint64_t* grand_total_dev,
                      cudaStream_t s);

// Reads the device error word, maps it to a TC code, clears it.
int check_dev_err(int* dev_err, cudaStream_t s);

// ---------------------------------------------------------------- the graph

struct Graph {
    int device = 0;
    int32_t n = 0;
    int64_t m_in = 0;
    int64_t m = 0;       // undirected edges after cleaning
    int bits = 1;        // bits per vertex id in packed keys
    // canonical edge list (original ids), edge-id order
    int32_t* lo = nullptr;
    int32_t* hi = nullptr;
    // Internal edge ids: j = position in the oriented (u, v) order, u < v in
    // rank; inv[c] is the internal id of canonical edge c (the ABI's edge
    // id).  Everything below that is per edge is in internal order.
    // endpoints in rank ids, (u, v), internal order
    int2* ends = nullptr;
    // symmetric CSR over rank ids: row r = [rowptr[r], rowptr[r+1]); its part
    // above r (the oriented out-list N+(r)) starts at upper[r]
    int64_t* rowptr = nullptr;
    int64_t* upper = nullptr;
    int32_t* col = nullptr;   // 2m neighbour rank ids
    int32_t* eid = nullptr;   // 2m internal edge ids
    int32_t* inv = nullptr;   // internal id of each canonical edge
    // for the column kernel: head[e] = the higher-rank end of internal edge
    // e (the out-lists laid out by edge id); iend[i] = one past the last
    // out-edge id of the i-th in-neighbour entry's neighbour, in-entries
    // numbered row by row (row v's start at rowptr[v] - first edge id of v)
    int32_t* head = nullptr;  // m
    int32_t* iend = nullptr;  // m
    // internal ids follow the out-lists: the out-entry at position p of row r
    // is edge p - oshift[r] (n entries)
    int64_t* oshift = nullptr;
    int32_t max_out = 0;      // max |N+(u)|
    int32_t max_deg = 0;
    // rows of degree <= 16, 32, 64, 128 (LIGHT_DEG): the lowest ranks
    int32_t light_rows[4] = {0, 0, 0, 0};
    // the column kernel's light columns: degree <= this bound (16..LIGHT_DEG)
    int32_t col_light_deg = LIGHT_DEG;
    int64_t wedge_work = -1;  // sum of |N+(u)| + |N+(v)| over oriented edges (lazy)
    int64_t column_work = -1; // sum over u of |N+(u)| (|N+(u)| - 1) / 2 (lazy, with wedge_work)
    int64_t last_peel_rounds = 0;  // bulk rounds of the most recent peel
    int last_peel_lists = 0;       // 1: it used triangle lists, 2: lists below a bound
    struct {
        int64_t count_ns = -1, support_ns = -1, lists_ns = -1, peel_ns = -1;
        int64_t product_form = 0;  // masked-product kernel of the latest count/support
        int64_t lists_bytes = -1;  // algorithmic bytes of the latest column-kernel list build
        int64_t peel_bytes = -1;
        int64_t peel_scanned = 0, peel_entries = 0, peel_searches = 0, peel_lookups = 0,
                peel_lowered = 0;
    } stats;  // device time of the latest launch of each main kernel
    // cached support (internal order) and triangle count
    int32_t* support = nullptr;
    bool support_valid = false;
    // cached per-edge triangle lists (kept after the first peel that builds
    // them, when they fit): list of edge e = tri_pairs[tri_off[e] .. tri_off[e+1])
    unsigned long long* tri_off = nullptr;
    int2* tri_pairs = nullptr;
    bool tri_valid = false;
    int32_t tri_bound = 0;     // 0: every edge has its list; B: only edges of support < B
    int64_t tri_entries = 0;   // pairs allocated
    // the latest single-level k-truss (ktruss): internal edge states (0 = in
    // the truss), supports within it and, for the intersection form, its
    // compacted adjacency; a later ktruss with a k at least as large resumes
    // from it (the (k+1)-truss lies inside the k-truss)
    int32_t* kt_state = nullptr;
    int32_t* kt_support = nullptr;
    int32_t kt_k = 0;  // 0 = nothing cached
    int32_t* kt_col = nullptr;
    int32_t* kt_eid = nullptr;
    int32_t* kt_rowlen = nullptr;
    bool kt_adj = false;
    // the truss decomposition of the latest ktruss_max (canonical order),
    // kept when it fits: later ktruss calls threshold it instead of peeling
    int32_t* truss_cache = nullptr;
    int32_t truss_kmax = 0;
    bool truss_valid = false;
    // bound on optional device memory for this graph (triangle lists, their
    // cache, the cached compacted adjacency); -1 = a share of free memory
    int64_t mem_limit = -1;
    // keep results between calls (truss numbers, the latest k-truss state)
    bool keep_results = true;
    // cap on the peel's grid (0: none): a server shares the device between
    // concurrent requests
    int peel_max_blocks = 0;
    int64_t triangles = -1;
    int* dev_err = nullptr;
    unsigned long long* dev_scalars = nullptr;  // small device scratch (8 words)
    cudaStream_t last_stream = nullptr;
};

// Scratch of a triangle-list build (planned before, enqueued later).
struct ListsPlan {
    unsigned long long* sums = nullptr;  // per-chunk sums of the offset scan
    int64_t chunks = 0;
    unsigned int* top = nullptr;         // per-edge fill positions from the list's end
    bool thread = false;                 // built by the thread-per-edge kernel
    int form = 1;                        // the intersection kernel that builds them
    int32_t bound = 0;                   // lists only for edges of support < bound (0: all)
    int64_t entries = 0;                 // pairs the lists hold
    int64_t low_edges = 0;               // ... edges with support in (0, bound)
    unsigned int* lowbits = nullptr;     // ... one bit per such edge
    unsigned int* lowpos = nullptr;      // ... their exclusive prefix count by edge id
    unsigned long long* lowsums = nullptr;
    int2* lowlist = nullptr;             // ... {head, edge id} of each, by edge id
    unsigned long long* partials = nullptr;
    int blocks = 0;
    KernelTimer timer;
};
int plan_triangle_lists(Graph* g, Scratch& sc, ListsPlan* lp);
// out[i] = x[0] + ... + x[i-1] for i in [0, n] (n + 1 entries).
int exclusive_scan_i32(const int32_t* x, int64_t n, unsigned long long* out, Scratch& sc,
                       cudaStream_t s);
// Sum of the supports in (0, bound) (the entries of lists kept only for
// those edges) and the number of such edges; synchronises.
int partial_list_entries(Graph* g, int32_t bound, int64_t* entries, int64_t* low_edges,
                         cudaStream_t s);
int enqueue_triangle_lists(Graph* g, const int32_t* sup, unsigned long long* off, int2* pairs,
                           ListsPlan* lp, cudaStream_t s);

// Peel: plan (host decisions and allocations), enqueue (stream work only,
// capturable), finish (reads results back; synchronises).
struct PeelPlan;
PeelPlan* peel_plan_new();
void peel_plan_delete(PeelPlan* p);
// keep_lists: a triangle-list build is kept with the graph for later peels;
// use_cache (single level only): work in the graph's k-truss cache and
// resume from it when k is at least the cached k.
// max_blocks > 0 caps the peel's grid (the batch tuner tries several).
int peel_plan(PeelPlan* p, Scratch& sc, Graph* g, int32_t k_first, bool single, int32_t* t,
              int form, bool keep_lists = false, bool use_cache = false, int max_blocks = 0);
int peel_enqueue(PeelPlan* p, cudaStream_t s);
int peel_finish(PeelPlan* p, cudaStream_t s, int64_t* n_alive, int32_t* kmax);
bool peel_uses_lists(const PeelPlan* p);  // full lists
int peel_form_of(const PeelPlan* p);      // PEEL_LISTS, PEEL_INTERSECT or PEEL_HYBRID
int ensure_support(Graph* g, cudaStream_t s);
// Internal-order per-edge arrays -> canonical order (out[c] = in[inv[c]]: a
// gather, so the writes are coalesced).
int to_canonical_i32(const int32_t* in, const int32_t* inv, int64_t m, int32_t* out,
                     cudaStream_t s);
// k-truss mask in canonical order from internal edge states (alive = 0).
int mask_from_state(const int32_t* t, const int32_t* inv, int64_t m, uint8_t* mask,
                    cudaStream_t s);

int build_graph(Graph* g, const int32_t* src_d, const int32_t* dst_d, cudaStream_t s);
void free_graph(Graph* g);
// form: 0 = automatic (honours the test hook), 1 = row/hash kernel where the
// graph allows it, 2 = edge-per-warp kernel.
int compute_support(Graph* g, int32_t* s_out_dev, bool want_support, int64_t* triangles,
                    cudaStream_t s, int form = 0);
int peel_ktruss(Graph* g, int32_t k, uint8_t* mask_dev, int64_t* edges_left, cudaStream_t s);
int graph_wedge_work(Graph* g, int64_t* out, cudaStream_t s);
bool triangle_lists_supported(const Graph* g);
int build_triangle_lists(Graph* g, const int32_t* sup, unsigned long long* off, int2* pairs,
                         cudaStream_t s);
int peel_decompose(Graph* g, int32_t* truss_dev, int32_t* kmax, cudaStream_t s);
// Sizes of the k-trusses for k = k_lo .. k_hi (at most 64 values; host
// output): the decomposition's levels from one peel, stopping after k_hi.
int peel_sizes(Graph* g, int32_t k_lo, int32_t k_hi, int64_t* sizes, cudaStream_t s);
// Connected components of the k-truss: canonical-order edge labels (device,
// m), optional vertex labels (device, n); labels are smallest vertex ids.
int truss_components(Graph* g, int32_t k, int32_t* edge_label, int32_t* vertex_label,
                     int64_t* count, cudaStream_t s);

}  // namespace tc

// The ABI's opaque graph handle.
struct tc_graph {
    tc::Graph g;
};
