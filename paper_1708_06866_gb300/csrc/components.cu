// components.cu — the k-truss as a set of connected trusses (Section IV-A's
// enumeration of the k-trusses): connected components of the subgraph of
// the k-truss edges, each labelled by its smallest vertex id.
//
// Lock-free union-find over the original vertex ids: every k-truss edge
// (lo, hi) joins the roots of its endpoints by a compare-and-swap that links
// the larger root under the smaller one, so a root is always the smallest id
// of its set and parent pointers only ever lead to smaller ids (every find
// ends).  Finds halve their paths as they go; a halving step only rewrites
// the parent of a vertex that is not a root, so it never races with a link.
// A last pass points every vertex at its root.
#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int CC_THREADS = 256;

__device__ __forceinline__ int32_t cc_find(int32_t* parent, int32_t x) {
    for (;;) {
        const int32_t p = __ldcg(parent + x);
        if (p == x) return x;
        const int32_t gp = __ldcg(parent + p);
        if (gp != p) parent[x] = gp;
        x = gp;
    }
}

__global__ void k_cc_init(int32_t* __restrict__ parent, uint8_t* __restrict__ touched,
                          int32_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        parent[v] = (int32_t)v;
        touched[v] = 0;
    }
}

__global__ void k_cc_link(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                          const uint8_t* __restrict__ mask, int64_t m, int32_t* parent,
                          uint8_t* __restrict__ touched) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        if (!mask[e]) continue;
        const int32_t u = lo[e], v = hi[e];
        touched[u] = 1;
        touched[v] = 1;
        int32_t a = cc_find(parent, u), b = cc_find(parent, v);
        while (a != b) {
            if (a > b) {
                const int32_t t = a;
                a = b;
                b = t;
            }
            // link root b under the smaller root a; if b stopped being a root
            // meanwhile, retry from the roots as they are now
            const int32_t old = atomicCAS(parent + b, b, a);
            if (old == b) break;
            a = cc_find(parent, a);
            b = cc_find(parent, old);
        }
    }
}

__global__ void k_cc_label(int32_t* parent, const uint8_t* __restrict__ touched, int32_t n,
                           int32_t* __restrict__ vertex_label,
                           unsigned long long* __restrict__ roots) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t r = cc_find(parent, (int32_t)v);
        parent[v] = r;
        if (touched[v] && r == (int32_t)v) ++c;
        if (vertex_label) vertex_label[v] = touched[v] ? r : -1;
    }
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(roots, c);
}

__global__ void k_cc_edges(const int32_t* __restrict__ lo, const uint8_t* __restrict__ mask,
                           int64_t m, const int32_t* __restrict__ parent,
                           int32_t* __restrict__ edge_label) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
        edge_label[e] = mask[e] ? parent[lo[e]] : -1;
}

unsigned grid_for(int64_t items) {
    return (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)num_sms() * 8, (items + CC_THREADS - 1) / CC_THREADS));
}

}  // namespace

int truss_components(Graph* g, int32_t k, int32_t* edge_label, int32_t* vertex_label,
                     int64_t* count, cudaStream_t s) {
    const int64_t m = g->m;
    const int32_t n = g->n;
    Scratch sc(s);
    uint8_t* mask = nullptr;
    int32_t* parent;
    uint8_t* touched;
    unsigned long long* roots;
    TC_TRY(sc.alloc(&parent, n));
    TC_TRY(sc.alloc(&touched, n));
    TC_TRY(sc.alloc(&roots, 1));
    if (m > 0) {
        TC_TRY(sc.alloc(&mask, m));
        int64_t left = 0;
        TC_TRY(peel_ktruss(g, k, mask, &left, s));
    }
    TC_CUDA_TRY(cudaMemsetAsync(roots, 0, sizeof(unsigned long long), s));
    k_cc_init<<<grid_for(n), CC_THREADS, 0, s>>>(parent, touched, n);
    TC_LAUNCH_CHECK("k_cc_init");
    if (m > 0) {
        k_cc_link<<<grid_for(m), CC_THREADS, 0, s>>>(g->lo, g->hi, mask, m, parent, touched);
        TC_LAUNCH_CHECK("k_cc_link");
    }
    k_cc_label<<<grid_for(n), CC_THREADS, 0, s>>>(parent, touched, n, vertex_label, roots);
    TC_LAUNCH_CHECK("k_cc_label");
    if (m > 0) {
        k_cc_edges<<<grid_for(m), CC_THREADS, 0, s>>>(g->lo, mask, m, parent, edge_label);
        TC_LAUNCH_CHECK("k_cc_edges");
    }
    unsigned long long c = 0;
    TC_CUDA_TRY(cudaMemcpyAsync(&c, roots, sizeof(c), cudaMemcpyDeviceToHost, s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    *count = (int64_t)c;
    return TC_OK;
}

}  // namespace tc
