// intersect.cu — triangle count and per-edge support by the masked product
// (L L^T) ∘ L over the degree-oriented adjacency (Section III-A, Algorithm 3,
// with a degree order in place of the index order so that every triangle is
// found exactly once), and the support credit of Algorithm 4 (s = (R == 2) 1).
//
// For an oriented edge (u, v), (L L^T)(u, v) = |N+(u) ∩ N+(v)|: each common
// out-neighbour w closes the triangle u < v < w (in rank order), found only
// at its lowest edge (u, v).  The support pass credits all three edges of
// each triangle found: (u, v) by the count, (u, w) and (v, w) by atomics.
#include <algorithm>

#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int IX_THREADS = 256;

// One warp per oriented edge: lanes take the shorter out-list's elements and
// look each up in the longer list by binary search.
template <bool SUPPORT>
__global__ void __launch_bounds__(IX_THREADS) k_intersect_warp(
    const int32_t* __restrict__ fwd, const int2* __restrict__ ends,
    const int64_t* __restrict__ rowptr, const int64_t* __restrict__ upper,
    const int32_t* __restrict__ col, const int32_t* __restrict__ eid, int64_t m,
    int32_t* __restrict__ sup, unsigned long long* __restrict__ partials) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long acc = 0;
    for (int64_t j = wid; j < m; j += nw) {
        const int32_t e = fwd[j];
        const int2 uv = ends[e];
        int64_t s0 = upper[uv.x], s1 = rowptr[uv.x + 1];
        int64_t l0 = upper[uv.y], l1 = rowptr[uv.y + 1];
        if (s1 - s0 > l1 - l0) {
            int64_t t0 = s0, t1 = s1;
            s0 = l0;
            s1 = l1;
            l0 = t0;
            l1 = t1;
        }
        if (s0 == s1) continue;
        uint32_t cnt = 0;
        for (int64_t p = s0 + lane; p < s1; p += 32) {
            const int32_t w = col[p];
            int64_t lo = l0, hi = l1;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (col[mid] < w) lo = mid + 1;
                else hi = mid;
            }
            if (lo < l1 && col[lo] == w) {
                ++cnt;
                if (SUPPORT) {
                    atomicAdd(&sup[eid[p]], 1);
                    atomicAdd(&sup[eid[lo]], 1);
                }
            }
        }
        cnt = warp_sum(cnt);
        if (lane == 0) {
            acc += cnt;
            if (SUPPORT && cnt) atomicAdd(&sup[e], (int)cnt);
        }
    }
    __shared__ unsigned long long s_acc[IX_THREADS / 32];
    if (lane == 0) s_acc[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < IX_THREADS / 32; ++w) t += s_acc[w];
        partials[blockIdx.x] = t;
    }
}

// Sum of the per-block partial counts (one block, no atomics).
__global__ void __launch_bounds__(1024) k_reduce_partials(const unsigned long long* __restrict__ p,
                                                          int64_t count,
                                                          unsigned long long* __restrict__ out) {
    unsigned long long acc = 0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) acc += p[i];
    acc = warp_sum(acc);
    __shared__ unsigned long long s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        *out = t;
    }
}

__global__ void k_wedge_work(const int32_t* __restrict__ fwd, const int2* __restrict__ ends,
                             const int64_t* __restrict__ rowptr, const int64_t* __restrict__ upper,
                             int64_t m, unsigned long long* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long acc = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const int2 uv = ends[fwd[j]];
        acc += (unsigned long long)(rowptr[uv.x + 1] - upper[uv.x]) +
               (unsigned long long)(rowptr[uv.y + 1] - upper[uv.y]);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

}  // namespace

int graph_wedge_work(Graph* g, int64_t* out, cudaStream_t s) {
    if (g->wedge_work < 0) {
        unsigned long long h = 0;
        if (g->m > 0) {
            TC_CUDA_TRY(cudaMemsetAsync(g->dev_scalars + 2, 0, sizeof(unsigned long long), s));
            k_wedge_work<<<num_sms() * 8, 256, 0, s>>>(g->fwd, g->ends, g->rowptr, g->upper, g->m,
                                                       g->dev_scalars + 2);
            TC_LAUNCH_CHECK("k_wedge_work");
            TC_CUDA_TRY(cudaMemcpyAsync(&h, g->dev_scalars + 2, sizeof(h), cudaMemcpyDeviceToHost, s));
            TC_CUDA_TRY(cudaStreamSynchronize(s));
        }
        g->wedge_work = (int64_t)h;
    }
    *out = g->wedge_work;
    return TC_OK;
}

int compute_support(Graph* g, int32_t* sup, bool want_support, int64_t* triangles,
                    cudaStream_t s) {
    const int64_t m = g->m;
    if (m == 0) {
        if (triangles) *triangles = 0;
        return TC_OK;
    }
    const int blocks = num_sms() * 8;
    Scratch sc(s);
    unsigned long long* partials;
    TC_TRY(sc.alloc(&partials, blocks));
    if (want_support) {
        TC_CUDA_TRY(cudaMemsetAsync(sup, 0, sizeof(int32_t) * m, s));
        k_intersect_warp<true><<<blocks, IX_THREADS, 0, s>>>(g->fwd, g->ends, g->rowptr, g->upper,
                                                             g->col, g->eid, m, sup, partials);
    } else {
        k_intersect_warp<false><<<blocks, IX_THREADS, 0, s>>>(g->fwd, g->ends, g->rowptr, g->upper,
                                                              g->col, g->eid, m, nullptr, partials);
    }
    TC_LAUNCH_CHECK("k_intersect_warp");
    k_reduce_partials<<<1, 1024, 0, s>>>(partials, blocks, g->dev_scalars);
    TC_LAUNCH_CHECK("k_reduce_partials");
    if (triangles) {
        unsigned long long t = 0;
        TC_CUDA_TRY(cudaMemcpyAsync(&t, g->dev_scalars, sizeof(t), cudaMemcpyDeviceToHost, s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
        *triangles = (int64_t)t;
    }
    return TC_OK;
}

}  // namespace tc
