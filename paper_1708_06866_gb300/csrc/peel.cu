// peel.cu — k-truss peeling and the truss decomposition (Section III-B,
// Algorithm 4).
//
// Algorithm 4 removes, in each pass of its loop, every edge whose support is
// below k - 2, then lowers the supports of the remaining edges by the
// triangles those removals destroyed (R -= E [E_x^T E_x - diag(d_x)]).  Here
// one round does the same on the device:
//   frontier F = alive edges with s < k - 2 (state -1 = "dying this round");
//   for each e in F, every triangle {e, f, g} whose other two edges are not
//   yet removed is destroyed; it is handled once, by the dying edge of the
//   triangle with the smallest edge id, which lowers s of each of f, g that
//   is not dying.  An edge whose support falls from k - 2 to k - 3 (exactly
//   one atomic sees that) joins the next round's frontier;
//   then the dying edges are removed (state = truss number k - 1).
// The decomposition runs k = 3, 4, ... on the survivors of the previous level
// until no edge is left.
//
// Edge state t[e]: 0 = alive, -1 = in the current frontier, > 0 = removed.
#include <algorithm>
#include <utility>

#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int PL_THREADS = 256;

__device__ __forceinline__ void warp_append(bool take, int32_t value, int32_t* list,
                                            unsigned* count) {
    const unsigned mask = __ballot_sync(0xffffffffu, take);
    if (mask == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (take) list[base + __popc(mask & lanemask_lt())] = value;
}

// Level start: keep the edges of `in` that are still alive (-> out) and put
// those with s < thr into the frontier, marked dying.  in == NULL means all
// edges 0..n_in-1.
__global__ void __launch_bounds__(PL_THREADS) k_level_scan(
    const int32_t* __restrict__ in, int64_t n_in, int32_t* __restrict__ t,
    const int32_t* __restrict__ s, int32_t thr, int32_t* __restrict__ out,
    unsigned* __restrict__ n_out, int32_t* __restrict__ F, unsigned* __restrict__ nF) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t start = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t base = start - (threadIdx.x & 31); base < n_in; base += stride) {
        const int64_t i = base + (threadIdx.x & 31);
        bool alive = false, front = false;
        int32_t e = 0;
        if (i < n_in) {
            e = in ? in[i] : (int32_t)i;
            alive = t[e] == 0;
            front = alive && s[e] < thr;
            if (front) t[e] = -1;
        }
        warp_append(alive, e, out, n_out);
        warp_append(front, e, F, nF);
    }
}

// One round: one warp per frontier edge e = {a, b}; lanes take the shorter
// full neighbour list's entries and look each up in the longer list.
__global__ void __launch_bounds__(PL_THREADS) k_peel_round(
    const int32_t* __restrict__ F, unsigned nF, const int2* __restrict__ ends,
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const int32_t* __restrict__ eid, const int32_t* __restrict__ t, int32_t* __restrict__ s,
    int32_t thr, int32_t* __restrict__ Fn, unsigned* __restrict__ nFn) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = wid; j < (int64_t)nF; j += nw) {
        const int32_t e = F[j];
        const int2 ab = ends[e];
        int64_t s0 = rowptr[ab.x], s1 = rowptr[ab.x + 1];
        int64_t l0 = rowptr[ab.y], l1 = rowptr[ab.y + 1];
        if (s1 - s0 > l1 - l0) {
            const int64_t t0 = s0, t1 = s1;
            s0 = l0;
            s1 = l1;
            l0 = t0;
            l1 = t1;
        }
        for (int64_t p = s0 + lane; p < s1; p += 32) {
            const int32_t f = eid[p];
            const int32_t tf = t[f];
            if (tf > 0) continue;  // removed in an earlier round
            const int32_t w = col[p];
            int64_t lo = l0, hi = l1;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (col[mid] < w) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= l1 || col[lo] != w) continue;
            const int32_t g = eid[lo];
            const int32_t tg = t[g];
            if (tg > 0) continue;
            // the triangle is destroyed this round; its smallest dying edge owns it
            if ((tf < 0 && f < e) || (tg < 0 && g < e)) continue;
            if (tf == 0) {
                const int old = atomicSub(&s[f], 1);
                if (old == thr) Fn[atomicAdd(nFn, 1u)] = f;
            }
            if (tg == 0) {
                const int old = atomicSub(&s[g], 1);
                if (old == thr) Fn[atomicAdd(nFn, 1u)] = g;
            }
        }
    }
}

// Round end: remove the frontier (state = value), mark the next frontier.
__global__ void k_finalize(const int32_t* __restrict__ F, unsigned nF, int32_t value,
                           const int32_t* __restrict__ Fn, const unsigned* __restrict__ nFn,
                           int32_t* __restrict__ t) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = i0; i < (int64_t)nF; i += stride) t[F[i]] = value;
    const int64_t nn = *nFn;
    for (int64_t i = i0; i < nn; i += stride) t[Fn[i]] = -1;
}

__global__ void k_mask_from_state(const int32_t* __restrict__ t, int64_t m,
                                  uint8_t* __restrict__ mask) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
        mask[e] = t[e] == 0 ? 1 : 0;
}

inline unsigned blocks_for_warps(int64_t items) {
    const int64_t warps_per_block = PL_THREADS / 32;
    int64_t b = (items + warps_per_block - 1) / warps_per_block;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (b < 1) b = 1;
    return (unsigned)std::min(b, cap);
}

inline unsigned blocks_for_items(int64_t items) {
    int64_t b = (items + PL_THREADS - 1) / PL_THREADS;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (b < 1) b = 1;
    return (unsigned)std::min(b, cap);
}

// Working buffers of a peel.
struct PeelState {
    int32_t* s = nullptr;      // support within the current subgraph
    int32_t* t = nullptr;      // edge state
    int32_t* alive[2] = {nullptr, nullptr};
    int32_t* F = nullptr;
    int32_t* Fn = nullptr;
    unsigned* counters = nullptr;  // [0] alive out, [1] |F|, [2] |Fn|
    int64_t n_alive = 0;
    int cur = 0;
    bool first = true;
};

int alloc_state(Scratch& sc, Graph* g, PeelState* ps, cudaStream_t s) {
    const int64_t m = g->m;
    TC_TRY(sc.alloc(&ps->s, m));
    TC_TRY(sc.alloc(&ps->alive[0], m));
    TC_TRY(sc.alloc(&ps->alive[1], m));
    TC_TRY(sc.alloc(&ps->F, m));
    TC_TRY(sc.alloc(&ps->Fn, m));
    TC_TRY(sc.alloc(&ps->counters, 4));
    TC_CUDA_TRY(
        cudaMemcpyAsync(ps->s, g->support, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s));
    TC_CUDA_TRY(cudaMemsetAsync(ps->t, 0, sizeof(int32_t) * m, s));
    ps->n_alive = m;
    return TC_OK;
}

// Peels one level: removes edges until every alive edge has s >= k - 2.
// Removed edges get state `value`.  Updates ps->n_alive.
int peel_level(Graph* g, PeelState* ps, int32_t k, int32_t value, cudaStream_t s) {
    const int32_t thr = k - 2;
    unsigned h[3];
    TC_CUDA_TRY(cudaMemsetAsync(ps->counters, 0, sizeof(unsigned) * 3, s));
    const int32_t* in = ps->first ? nullptr : ps->alive[ps->cur];
    int32_t* out = ps->alive[ps->cur ^ 1];
    k_level_scan<<<blocks_for_items(ps->n_alive), PL_THREADS, 0, s>>>(
        in, ps->n_alive, ps->t, ps->s, thr, out, ps->counters + 0, ps->F, ps->counters + 1);
    TC_LAUNCH_CHECK("k_level_scan");
    TC_CUDA_TRY(cudaMemcpyAsync(h, ps->counters, sizeof(unsigned) * 2, cudaMemcpyDeviceToHost, s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    ps->first = false;
    ps->cur ^= 1;
    int64_t n_alive = h[0];
    unsigned nF = h[1];
    int32_t* F = ps->F;
    int32_t* Fn = ps->Fn;
    int64_t rounds = 0;
    while (nF > 0) {
        if (++rounds > g->m + 1) return fail(TC_ETIMEDOUT, "peel: round limit exceeded");
        TC_CUDA_TRY(cudaMemsetAsync(ps->counters + 2, 0, sizeof(unsigned), s));
        k_peel_round<<<blocks_for_warps(nF), PL_THREADS, 0, s>>>(
            F, nF, g->ends, g->rowptr, g->col, g->eid, ps->t, ps->s, thr, Fn, ps->counters + 2);
        TC_LAUNCH_CHECK("k_peel_round");
        k_finalize<<<blocks_for_items(std::max<int64_t>(nF, 1024)), PL_THREADS, 0, s>>>(
            F, nF, value, Fn, ps->counters + 2, ps->t);
        TC_LAUNCH_CHECK("k_finalize");
        TC_CUDA_TRY(
            cudaMemcpyAsync(&h[2], ps->counters + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
        n_alive -= nF;
        nF = h[2];
        std::swap(F, Fn);
    }
    ps->n_alive = n_alive;
    return TC_OK;
}

int ensure_support(Graph* g, cudaStream_t s) {
    if (g->support_valid) return TC_OK;
    if (!g->support) TC_TRY(dev_alloc_n(&g->support, g->m, s));
    int64_t T = 0;
    TC_TRY(compute_support(g, g->support, true, &T, s));
    g->triangles = T;
    g->support_valid = true;
    return TC_OK;
}

}  // namespace

int peel_ktruss(Graph* g, int32_t k, uint8_t* mask, int64_t* edges_left, cudaStream_t s) {
    const int64_t m = g->m;
    if (m == 0) {
        if (edges_left) *edges_left = 0;
        return TC_OK;
    }
    TC_TRY(ensure_support(g, s));
    Scratch sc(s);
    PeelState ps;
    TC_TRY(sc.alloc(&ps.t, m));
    TC_TRY(alloc_state(sc, g, &ps, s));
    TC_TRY(peel_level(g, &ps, k, 1, s));
    k_mask_from_state<<<blocks_for_items(m), PL_THREADS, 0, s>>>(ps.t, m, mask);
    TC_LAUNCH_CHECK("k_mask_from_state");
    if (edges_left) *edges_left = ps.n_alive;
    return TC_OK;
}

int peel_decompose(Graph* g, int32_t* truss, int32_t* kmax, cudaStream_t s) {
    const int64_t m = g->m;
    if (m == 0) {
        *kmax = 0;
        return TC_OK;
    }
    TC_TRY(ensure_support(g, s));
    Scratch sc(s);
    PeelState ps;
    ps.t = truss;
    TC_TRY(alloc_state(sc, g, &ps, s));
    int32_t k = 3;
    int32_t best = 2;
    for (;;) {
        TC_TRY(peel_level(g, &ps, k, k - 1, s));
        if (ps.n_alive == 0) break;
        best = k;
        ++k;
    }
    *kmax = best;
    return TC_OK;
}

}  // namespace tc
