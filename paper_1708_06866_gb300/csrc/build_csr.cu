// build_csr.cu — device graph construction (Section II cleaning rules plus the
// degree-ordered adjacency the triangle kernels use).
//
//   1. keys:   each input pair (u, v) -> packed (min << b | max); a self-loop
//              gets a sentinel key that sorts last; ids outside [0, n) flag
//              DEV_ERR_RANGE.                                    (Section II)
//   2. sort + dedupe -> the canonical edge list lo[e] < hi[e].
//   3. degrees, and the degree order rank(v) = position of (deg(v), v).
//   4. every edge as (lower rank, higher rank), sorted -> the out-lists
//      N+(u) of the degree-oriented adjacency L (Algorithm 3's L with a
//      degree order in place of the index order), numbering the edges; the
//      same pairs stably re-sorted by their higher end -> the in-lists.
//      Together: a symmetric CSR whose rows ascend, each row's in-entries
//      (below u) followed by N+(u).
#include <algorithm>

#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int CB_THREADS = 256;
constexpr int CB_ITEMS = 8;
constexpr int CB_CHUNK = CB_THREADS * CB_ITEMS;

__global__ void k_make_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                            int64_t m_in, int32_t n, int bits, uint64_t sentinel,
                            uint64_t* __restrict__ keys, int* __restrict__ err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_in; i += stride) {
        const int32_t u = src[i], v = dst[i];
        uint64_t key = sentinel;
        if (u < 0 || u >= n || v < 0 || v >= n) {
            bad = true;
        } else if (u != v) {
            const uint64_t a = (uint64_t)min(u, v), b = (uint64_t)max(u, v);
            key = (a << bits) | b;
        }
        keys[i] = key;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, DEV_ERR_RANGE);
}

// Stream compaction in index order: count per chunk, scan, write.
struct DedupeOp {
    const uint64_t* keys;
    uint64_t sentinel;
    int bits;
    int32_t* lo;
    int32_t* hi;
    __device__ bool flag(int64_t i) const {
        const uint64_t k = keys[i];
        return k != sentinel && (i == 0 || keys[i - 1] != k);
    }
    __device__ void emit(int64_t i, int64_t pos) const {
        const uint64_t k = keys[i];
        lo[pos] = (int32_t)(k >> bits);
        hi[pos] = (int32_t)(k & ((1ull << bits) - 1));
    }
};


template <typename Op>
__global__ void __launch_bounds__(CB_THREADS) k_compact_count(Op op, int64_t n,
                                                              uint32_t* __restrict__ totals) {
    const int64_t base = (int64_t)blockIdx.x * CB_CHUNK;
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < CB_ITEMS; ++i) {
        const int64_t idx = base + i * CB_THREADS + threadIdx.x;
        if (idx < n && op.flag(idx)) ++c;
    }
    c = warp_sum(c);
    __shared__ uint32_t s[CB_THREADS / 32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < CB_THREADS / 32; ++w) t += s[w];
        totals[blockIdx.x] = t;
    }
}

template <typename Op>
__global__ void __launch_bounds__(CB_THREADS) k_compact_write(Op op, int64_t n,
                                                              const uint32_t* __restrict__ offs) {
    __shared__ uint32_t s_scan[33];
    const int64_t base = (int64_t)blockIdx.x * CB_CHUNK;
    int64_t run = offs[blockIdx.x];
#pragma unroll 1
    for (int i = 0; i < CB_ITEMS; ++i) {
        const int64_t idx = base + i * CB_THREADS + threadIdx.x;
        const bool f = idx < n && op.flag(idx);
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(f ? 1u : 0u, s_scan, &tot);
        if (f) op.emit(idx, run + ex);
        run += tot;
    }
}

// Degrees of the canonical list.  The list is sorted by its lower endpoint,
// so a warp's 32 consecutive edges mostly share it: lanes with the same
// lower endpoint add their count with one atomic (the higher endpoints are
// scattered and take one each).
__global__ void k_degree(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                         int64_t m, int32_t* __restrict__ deg) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps iterate together (the match needs every lane)
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; b < m; b += stride) {
        const int64_t e = b + lane;
        const bool ok = e < m;
        const int32_t a = ok ? lo[e] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, a);
        if (ok && lane == __ffs(peers) - 1) atomicAdd(&deg[a], __popc(peers));
        if (ok) atomicAdd(&deg[hi[e]], 1);
    }
}

__global__ void k_vertex_keys(const int32_t* __restrict__ deg, int32_t n, int bits,
                              uint64_t* __restrict__ keys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        keys[v] = ((uint64_t)deg[v] << bits) | (uint64_t)v;
}

__global__ void k_rank(const uint64_t* __restrict__ sorted, int32_t n, int bits,
                       int32_t* __restrict__ rank) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t mask = (1ull << bits) - 1;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
        rank[sorted[p] & mask] = (int32_t)p;
}

// One key per edge, oriented by rank: (lower rank u) << bits | (higher rank
// v), with the edge's canonical id as its value.  Sorted, these are the
// out-lists N+(u) in CSR order, and an edge's position in that order is its
// internal id.
__global__ void k_out_pairs(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                            int64_t m, const int32_t* __restrict__ rank, int bits,
                            uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t a = rank[lo[e]], c = rank[hi[e]];
        keys[e] = ((uint64_t)min(a, c) << bits) | (uint64_t)max(a, c);
        vals[e] = (uint32_t)e;
    }
}

// obase[r] = the first position of the sorted out-pairs whose row is >= r
// (r = 0 .. n; obase[n] = m): the out-degrees' exclusive scan, read off the
// sorted keys.  Entry i sets the rows from its predecessor's row + 1 to its
// own; the rows before the first entry (the degree-0 vertices, which the
// degree order puts first) are set by a grid-stride loop.
__global__ void k_out_starts(const uint64_t* __restrict__ keys, int64_t m, int32_t n, int bits,
                             unsigned long long* __restrict__ obase) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = m > 0 ? (int64_t)(keys[0] >> bits) : (int64_t)n;
    for (int64_t r = tid; r <= first; r += stride) obase[r] = 0;
    for (int64_t i = tid + 1; i <= m; i += stride) {
        const int64_t r_prev = (int64_t)(keys[i - 1] >> bits);
        const int64_t r_cur = i == m ? (int64_t)n : (int64_t)(keys[i] >> bits);
        for (int64_t r = r_prev + 1; r <= r_cur; ++r) obase[r] = (unsigned long long)i;
    }
}

// Degrees by rank (the symmetric CSR's row lengths).
__global__ void k_rank_degrees(const int32_t* __restrict__ deg, const int32_t* __restrict__ rank,
                               int32_t n, int32_t* __restrict__ deg_rank) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride)
        deg_rank[rank[x]] = deg[x];
}

// Row r of the symmetric CSR holds its in-entries (neighbours below r) and
// then its out-entries: upper[r] = rowptr[r] + in-degree; out-entry p of row
// r is internal edge p - oshift[r] with oshift[r] = upper[r] - obase[r];
// oend[r] = obase[r + 1] is the end of r's out-edge ids (int32: edge ids are
// below 2^31; a small array, so the scattered reads of it mostly hit L2).
__global__ void k_row_bounds(const int64_t* __restrict__ rowptr,
                             const unsigned long long* __restrict__ obase,
                             const int32_t* __restrict__ deg_rank, int32_t n,
                             int64_t* __restrict__ upper, int64_t* __restrict__ oshift,
                             int32_t* __restrict__ oend, int* __restrict__ err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const int64_t dout = (int64_t)(obase[r + 1] - obase[r]);
        const int64_t din = (int64_t)deg_rank[r] - dout;
        if (din < 0) atomicOr(err, DEV_ERR_BOUNDS);  // degrees and pairs disagree
        upper[r] = rowptr[r] + din;
        oshift[r] = upper[r] - (int64_t)obase[r];
        oend[r] = (int32_t)obase[r + 1];
    }
}

// Out-entries from the sorted out-pairs: internal edge j = (u, v) records
// its ends, its head v, the inverse map inv[canonical id] = j, and its entry
// at position j + oshift[u] of row u; vals[j] becomes j, the value the
// in-entry sort carries.
__global__ void k_out_part(const uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                           int64_t m, int bits, const int64_t* __restrict__ oshift,
                           int32_t* __restrict__ inv, int2* __restrict__ ends,
                           int32_t* __restrict__ head, int32_t* __restrict__ col,
                           int32_t* __restrict__ eid, int* __restrict__ err) {
    const uint64_t mask = (1ull << bits) - 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const uint64_t k = keys[j];
        const int32_t u = (int32_t)(k >> bits), v = (int32_t)(k & mask);
        inv[vals[j]] = (int32_t)j;
        vals[j] = (uint32_t)j;
        ends[j] = make_int2(u, v);
        head[j] = v;
        const int64_t p = j + oshift[u];
        if (p < 0 || p >= 2 * m) {  // only if degrees and pairs disagree
            atomicOr(err, DEV_ERR_BOUNDS);
            continue;
        }
        col[p] = v;
        eid[p] = (int32_t)j;
    }
}

// In-entries from the out-pairs stably re-sorted by their higher end v: the
// q-th of them is u's entry in row v (rows ascend by v, and within a row by
// u, since the first order was by (u, v)), at position q + obase[v] (the
// in-entries before row v number rowptr[v] - obase[v]); it records edge j,
// and iend[q], the end of u's out-edge ids (the column kernel streams u's
// out-list above v up to it).
__global__ void k_in_part(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                          int64_t m, int bits, const unsigned long long* __restrict__ obase,
                          const int32_t* __restrict__ oend, int32_t* __restrict__ col,
                          int32_t* __restrict__ eid, int32_t* __restrict__ iend,
                          int* __restrict__ err) {
    const uint64_t mask = (1ull << bits) - 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += stride) {
        const uint64_t k = keys[q];
        const int32_t u = (int32_t)(k >> bits), v = (int32_t)(k & mask);
        const int64_t p = q + (int64_t)obase[v];
        iend[q] = oend[u];
        if (p >= 2 * m) {  // only if degrees and pairs disagree
            atomicOr(err, DEV_ERR_BOUNDS);
            continue;
        }
        col[p] = u;
        eid[p] = (int32_t)vals[q];
    }
}

// [0] = largest degree, [1] = largest out-list, [2 + i] = rows of degree
// at most 16 << i, i < 4 (rows ascend by degree, so these are the rows below
// that count: the column kernel's light columns for that bound).
__global__ void k_row_stats(const int64_t* __restrict__ rowptr, const int64_t* __restrict__ upper,
                            int32_t n, unsigned long long* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long md = 0, mo = 0, nl[4] = {0, 0, 0, 0};
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const int64_t d = rowptr[r + 1] - rowptr[r];
        md = max(md, (unsigned long long)d);
        mo = max(mo, (unsigned long long)(rowptr[r + 1] - upper[r]));
#pragma unroll
        for (int i = 0; i < 4; ++i) nl[i] += d <= (16 << i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        md = max(md, __shfl_xor_sync(0xffffffffu, md, o));
        mo = max(mo, __shfl_xor_sync(0xffffffffu, mo, o));
#pragma unroll
        for (int i = 0; i < 4; ++i) nl[i] += __shfl_xor_sync(0xffffffffu, nl[i], o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], md);
        atomicMax(&out[1], mo);
#pragma unroll
        for (int i = 0; i < 4; ++i) atomicAdd(&out[2 + i], nl[i]);
    }
}

inline unsigned grid_for(int64_t n, int threads = 256) {
    const int64_t cap = (int64_t)num_sms() * 32;
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (unsigned)std::min(b, cap);
}

}  // namespace

int build_graph(Graph* g, const int32_t* src, const int32_t* dst, cudaStream_t s) {
    const int64_t m_in = g->m_in;
    const int32_t n = g->n;
    const int bits = bits_for((uint64_t)(n > 1 ? n - 1 : 1));
    g->bits = bits;
    const uint64_t id_mask = (1ull << bits) - 1;
    const uint64_t sentinel = (id_mask << bits) | id_mask;
    uint64_t* scalar = reinterpret_cast<uint64_t*>(g->dev_scalars);

    TC_CUDA_TRY(cudaMemsetAsync(g->dev_err, 0, sizeof(int), s));
    int64_t m = 0;
    {
        // 1-2. canonical edge list
        Scratch sc(s);
        uint64_t *keys = nullptr, *keys_alt = nullptr;
        TC_TRY(sc.alloc(&keys, m_in));
        if (m_in > 0) {
            k_make_keys<<<grid_for(m_in), 256, 0, s>>>(src, dst, m_in, n, bits, sentinel, keys,
                                                      g->dev_err);
            TC_LAUNCH_CHECK("k_make_keys");
            TC_TRY(check_dev_err(g->dev_err, s));
            TC_TRY(sc.alloc(&keys_alt, m_in));
            TC_TRY(radix_sort_u64(keys, keys_alt, nullptr, nullptr, m_in, 2 * bits, g->dev_err, s));
        }
        // upper bound for the unique count is m_in; allocate after counting
        DedupeOp op{keys, sentinel, bits, nullptr, nullptr};
        const int64_t chunks = (m_in + CB_CHUNK - 1) / CB_CHUNK;
        if (m_in > 0) {
            uint32_t* totals;
            TC_TRY(sc.alloc(&totals, chunks));
            k_compact_count<DedupeOp><<<(unsigned)chunks, CB_THREADS, 0, s>>>(op, m_in, totals);
            TC_LAUNCH_CHECK("k_compact_count");
            TC_TRY(scan_block_totals(totals, chunks, scalar, s));
            uint64_t cnt = 0;
            TC_CUDA_TRY(cudaMemcpyAsync(&cnt, scalar, 8, cudaMemcpyDeviceToHost, s));
            TC_CUDA_TRY(cudaStreamSynchronize(s));
            TC_TRY(check_dev_err(g->dev_err, s));
            m = (int64_t)cnt;
            if (m > 0x7fffffffLL) return fail(TC_EOVERFLOW, "more than 2^31-1 edges after cleaning");
            TC_TRY(dev_alloc_n(&g->lo, m, s));
            TC_TRY(dev_alloc_n(&g->hi, m, s));
            op.lo = g->lo;
            op.hi = g->hi;
            k_compact_write<DedupeOp><<<(unsigned)chunks, CB_THREADS, 0, s>>>(op, m_in, totals);
            TC_LAUNCH_CHECK("k_compact_write");
        } else {
            TC_TRY(dev_alloc_n(&g->lo, 0, s));
            TC_TRY(dev_alloc_n(&g->hi, 0, s));
        }
    }
    g->m = m;

    // 3-4. degree order and the symmetric CSR in rank ids
    TC_TRY(dev_alloc_n(&g->rowptr, (int64_t)n + 1, s));
    TC_TRY(dev_alloc_n(&g->upper, (int64_t)n, s));
    TC_TRY(dev_alloc_n(&g->ends, m, s));
    TC_TRY(dev_alloc_n(&g->col, 2 * m, s));
    TC_TRY(dev_alloc_n(&g->eid, 2 * m, s));
    TC_TRY(dev_alloc_n(&g->inv, m, s));
    {
        Scratch sc(s);
        int32_t *deg, *rank;
        uint64_t *vkeys, *vkeys_alt;
        TC_TRY(sc.alloc(&deg, n));
        TC_TRY(sc.alloc(&rank, n));
        TC_TRY(sc.alloc(&vkeys, n));
        TC_TRY(sc.alloc(&vkeys_alt, n));
        TC_CUDA_TRY(cudaMemsetAsync(deg, 0, sizeof(int32_t) * n, s));
        if (m > 0) {
            k_degree<<<grid_for(m), 256, 0, s>>>(g->lo, g->hi, m, deg);
            TC_LAUNCH_CHECK("k_degree");
        }
        k_vertex_keys<<<grid_for(n), 256, 0, s>>>(deg, n, bits, vkeys);
        TC_LAUNCH_CHECK("k_vertex_keys");
        TC_TRY(radix_sort_u64(vkeys, vkeys_alt, nullptr, nullptr, n, 2 * bits, g->dev_err, s));
        k_rank<<<grid_for(n), 256, 0, s>>>(vkeys, n, bits, rank);
        TC_LAUNCH_CHECK("k_rank");

        // 4. the symmetric CSR in rank ids.  The out-pairs (u < v, one per
        // edge) sorted by (u, v) are the out-lists, and their order numbers
        // the edges; re-sorted stably by v alone (its digits only) they are
        // the in-lists, already in row order.  Row lengths come from the
        // degrees, so rows are laid out before either sort finishes.
        uint64_t *pkeys, *pkeys_alt;
        uint32_t *pvals, *pvals_alt;
        int32_t *deg_rank, *oend;
        unsigned long long* obase;
        TC_TRY(sc.alloc(&pkeys, m));
        TC_TRY(sc.alloc(&pkeys_alt, m));
        TC_TRY(sc.alloc(&pvals, m));
        TC_TRY(sc.alloc(&pvals_alt, m));
        TC_TRY(sc.alloc(&deg_rank, n));
        TC_TRY(sc.alloc(&obase, (int64_t)n + 1));
        TC_TRY(sc.alloc(&oend, n));
        TC_TRY(dev_alloc_n(&g->oshift, n, s));
        TC_TRY(dev_alloc_n(&g->head, m, s));
        TC_TRY(dev_alloc_n(&g->iend, m, s));
        if (m > 0) {
            k_out_pairs<<<grid_for(m), 256, 0, s>>>(g->lo, g->hi, m, rank, bits, pkeys, pvals);
            TC_LAUNCH_CHECK("k_out_pairs");
            TC_TRY(radix_sort_u64(pkeys, pkeys_alt, pvals, pvals_alt, m, 2 * bits, g->dev_err, s));
        }
        k_out_starts<<<grid_for(m + 1), 256, 0, s>>>(pkeys, m, n, bits, obase);
        TC_LAUNCH_CHECK("k_out_starts");
        k_rank_degrees<<<grid_for(n), 256, 0, s>>>(deg, rank, n, deg_rank);
        TC_LAUNCH_CHECK("k_rank_degrees");
        TC_TRY(exclusive_scan_i32(deg_rank, n, reinterpret_cast<unsigned long long*>(g->rowptr),
                                  sc, s));
        k_row_bounds<<<grid_for(n), 256, 0, s>>>(g->rowptr, obase, deg_rank, n, g->upper,
                                                 g->oshift, oend, g->dev_err);
        TC_LAUNCH_CHECK("k_row_bounds");
        if (m > 0) {
            k_out_part<<<grid_for(m), 256, 0, s>>>(pkeys, pvals, m, bits, g->oshift, g->inv,
                                                   g->ends, g->head, g->col, g->eid, g->dev_err);
            TC_LAUNCH_CHECK("k_out_part");
            TC_TRY(radix_sort_u64(pkeys, pkeys_alt, pvals, pvals_alt, m, bits, g->dev_err, s));
            k_in_part<<<grid_for(m), 256, 0, s>>>(pkeys, pvals, m, bits, obase, oend, g->col,
                                                  g->eid, g->iend, g->dev_err);
            TC_LAUNCH_CHECK("k_in_part");
        }
        TC_CUDA_TRY(cudaMemsetAsync(g->dev_scalars, 0, 6 * sizeof(unsigned long long), s));
        k_row_stats<<<grid_for(n), 256, 0, s>>>(g->rowptr, g->upper, n, g->dev_scalars);
        TC_LAUNCH_CHECK("k_row_stats");
        // the degrees must sum to 2m (rowptr[n]), as the pairs do
        TC_CUDA_TRY(cudaMemcpyAsync(g->dev_scalars + 6, g->rowptr + n, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToDevice, s));
        unsigned long long st[7];
        TC_CUDA_TRY(cudaMemcpyAsync(st, g->dev_scalars, sizeof(st), cudaMemcpyDeviceToHost, s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
        if ((int64_t)st[6] != 2 * m) return fail(TC_ECUDA, "internal: degree sum mismatch");
        g->max_deg = (int32_t)st[0];
        g->max_out = (int32_t)st[1];
        for (int i = 0; i < 4; ++i) g->light_rows[i] = (int32_t)st[2 + i];
        TC_TRY(check_dev_err(g->dev_err, s));
    }
    return TC_OK;
}

}  // namespace tc
