// intersect.cu — triangle count and per-edge support by the masked product
// (L L^T) ∘ L over the degree-oriented adjacency (Section III-A, Algorithm 3,
// with a degree order in place of the index order so that every triangle is
// found exactly once), and the support credit of Algorithm 4 (s = (R == 2) 1).
//
// For an oriented edge (u, v), (L L^T)(u, v) = |N+(u) ∩ N+(v)|: each common
// out-neighbour w closes the triangle u < v < w (in rank order), found only
// at its lowest edge (u, v).  The support pass credits all three edges of
// each triangle found: (u, v) and (v, w) by global atomics, (u, w) through a
// per-row shared-memory counter flushed once per row.
//
// Main kernel (k_rows): one block per row u, rows handed out dynamically from
// the highest rank down.  N+(u) goes into a shared-memory hash table (key =
// neighbour, value = its position in the row); each warp takes one v of
// N+(u) at a time and its lanes stream N+(v) with coalesced loads, probing
// the table for every w.  A third mode writes each edge's triangle list (the
// ids of the two other edges of every triangle through it) for the peel.
// Each edge's list fills from both ends: triangles found in the edge's own
// source row (where the edge is (u, v) or (u, w) of a triangle u < v < w)
// from the bottom through shared-memory cursors of that row, so those writes
// stay within one block's lifetime; the rest (the edge is (v, w)) from the
// top through one global cursor per edge.
// The default kernel (k_cols) takes the same product by columns: one
// column v of the mask at a time, N+(v) in the table, and for each
// in-neighbour u the part of N+(u) above v streamed against it (fewer
// entries read: see k_cols); k_rows stays as a selectable form.
// Graphs whose largest out-list exceeds the table capacity use k_edges_warp
// (one warp per oriented edge, binary search in global memory).
#include <algorithm>
#include <atomic>
#include <climits>

#include "tc_internal.cuh"

namespace tc {
namespace {

#ifndef TC_RX_THREADS
#define TC_RX_THREADS 256
#endif
#ifndef TC_RX_UNROLL
#define TC_RX_UNROLL 8     // 32-wide chunks of N+(v) in flight per warp pass
#endif
#ifndef TC_RX_SPARSE_LIMIT
#define TC_RX_SPARSE_LIMIT 1024  // rows up to this size get the sparser table
#endif
#ifndef TC_RX_SPARSE_FACTOR
#define TC_RX_SPARSE_FACTOR 4    // table slots per entry for those rows
#endif
constexpr int RX_THREADS = TC_RX_THREADS;
constexpr int RX_WARPS = RX_THREADS / 32;
constexpr int RX_MAX_OUT = 8192;  // largest |N+(u)| the shared table holds (load <= 1/2)
constexpr int IX_THREADS = 256;
constexpr int THREAD_MAX_OUT = 16;  // largest out-list for which a thread per edge is used

enum Mode { COUNT = 0, SUPPORT = 1, LISTS = 2 };

__device__ __forceinline__ uint32_t slot_of(int32_t w, int log_cap) {
    return ((uint32_t)w * 0x9E3779B1u) >> (32 - log_cap);
}

// Table size for an out-list of du entries: load <= 1/4 up to 1024 entries
// (short probe runs: a warp waits for its slowest lane), <= 1/2 above.
__host__ __device__ __forceinline__ int table_log_cap(int du) {
    const int want = du <= TC_RX_SPARSE_LIMIT ? TC_RX_SPARSE_FACTOR * du : 2 * du;
    int lc = 6;
    while ((1 << lc) < want) ++lc;
    return lc;
}

// Slot of w in the table, or -1.
__device__ __forceinline__ int table_find(const int32_t* keys, int log_cap, int32_t w) {
    const uint32_t mask = (1u << log_cap) - 1;
    uint32_t h = slot_of(w, log_cap);
    int32_t k = keys[h];
    while (k != w) {
        if (k == -1) return -1;
        h = (h + 1) & mask;
        k = keys[h];
    }
    return (int)h;
}

// LISTS with bound > 0 writes only the lists of edges whose support (sup,
// read-only in that mode) is below bound.
__device__ __forceinline__ bool gets_list(const int32_t* sup, int32_t bound, int32_t e) {
    return bound == 0 || sup[e] < bound;
}

template <int MODE>
__global__ void __launch_bounds__(RX_THREADS) k_rows(
    const int64_t* __restrict__ rowptr, const int64_t* __restrict__ upper,
    const int32_t* __restrict__ col, const int64_t* __restrict__ oshift, int32_t n,
    int32_t* __restrict__ sup, const unsigned long long* __restrict__ off,
    unsigned int* __restrict__ top, int2* __restrict__ pairs, unsigned int* __restrict__ next_row,
    unsigned long long* __restrict__ partials, int max_log_cap, int max_pos, int32_t bound) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int max_cap = 1 << max_log_cap;
    int32_t* keys = reinterpret_cast<int32_t*>(smem);
    uint16_t* pos = reinterpret_cast<uint16_t*>(keys + max_cap);
    // per position i of N+(u): SUPPORT: triangles credited to (u, N+(u)[i]);
    // LISTS: entries written at the bottom of that edge's list, the list's
    // start and the edge id
    int32_t* cnt = reinterpret_cast<int32_t*>(pos + max_cap);
    unsigned int* sbase = reinterpret_cast<unsigned int*>(cnt + max_pos);
    int32_t* seid = reinterpret_cast<int32_t*>(sbase + max_pos);
    __shared__ int s_row;
    __shared__ unsigned long long s_acc[RX_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long acc = 0;

    for (;;) {
        if (threadIdx.x == 0) s_row = (int)atomicAdd(next_row, 1u);
        __syncthreads();
        const int r = s_row;
        __syncthreads();
        if (r >= n) break;
        const int32_t u = n - 1 - r;
        const int64_t a0 = upper[u];
        // the out-edges of a row have consecutive ids: id of entry p = p - oshift[row]
        const int64_t eu = a0 - (MODE == COUNT ? 0 : oshift[u]);
        const int du = (int)(rowptr[u + 1] - a0);
        if (du < 2) continue;
        // clamped to the block's table (never binding when sized as the host
        // sizes it; a clamped table still has load <= 1/2 since du <= max_out)
        const int log_cap = min(table_log_cap(du), max_log_cap);
        const int cap = 1 << log_cap;
        for (int i = threadIdx.x; i < cap; i += RX_THREADS) keys[i] = -1;
        if (MODE == SUPPORT)
            for (int i = threadIdx.x; i < du; i += RX_THREADS) cnt[i] = 0;
        if (MODE == LISTS)
            for (int i = threadIdx.x; i < du; i += RX_THREADS) {
                const int32_t e = (int32_t)(eu + i);
                cnt[i] = 0;
                seid[i] = e;
                sbase[i] = gets_list(sup, bound, e) ? (unsigned int)off[e] : 0xffffffffu;
            }
        __syncthreads();
        for (int i = threadIdx.x; i < du; i += RX_THREADS) {
            const int32_t w = col[a0 + i];
            uint32_t h = slot_of(w, log_cap);
            while (atomicCAS(&keys[h], -1, w) != -1) h = (h + 1) & (cap - 1);
            pos[h] = (uint16_t)i;
        }
        __syncthreads();
        const int32_t umax = col[a0 + du - 1];
        // the largest v of N+(u) cannot close a triangle: nothing in N+(u) is above it
        for (int j = warp; j < du - 1; j += RX_WARPS) {
            const int32_t v = col[a0 + j];
            const int64_t b0 = upper[v], b1 = rowptr[v + 1];
            const int64_t ov = MODE == COUNT ? 0 : oshift[v];
            const int32_t e_uv = MODE == COUNT ? 0 : (int32_t)(eu + j);
            const unsigned int base_uv = MODE == LISTS ? sbase[j] : 0u;  // ~0u: no list
            uint32_t c = 0;
            // one hit: credit the triangle (u, v, w) found at N+(v) position p,
            // table slot h
            auto hit = [&](int h, int64_t p) {
                ++c;
                if (MODE == SUPPORT) {
                    atomicAdd(&cnt[pos[h]], 1);
                    atomicAdd(&sup[p - ov], 1);
                }
            };
            // the triangles of a chunk share edge (u, v): one append for all;
            // (u, v) and (u, w) fill from the bottom (this row's cursors),
            // (v, w) from the top
            auto lists = [&](int h, int64_t p) {
                const unsigned msk = __ballot_sync(0xffffffffu, h >= 0);
                if (!msk) return;
                const int ldr = __ffs(msk) - 1;
                unsigned base = 0;
                if (lane == ldr && base_uv != 0xffffffffu)
                    base = atomicAdd((unsigned int*)&cnt[j], (unsigned)__popc(msk));
                base = __shfl_sync(0xffffffffu, base, ldr);
                if (h >= 0) {
                    const int iw = pos[h];
                    const int32_t e_uw = seid[iw], e_vw = (int32_t)(p - ov);
                    if (base_uv != 0xffffffffu)
                        pairs[base_uv + base + __popc(msk & lanemask_lt())] = make_int2(e_uw, e_vw);
                    if (sbase[iw] != 0xffffffffu)
                        pairs[sbase[iw] + atomicAdd((unsigned int*)&cnt[iw], 1u)] =
                            make_int2(e_uv, e_vw);
                    if (gets_list(sup, bound, e_vw))
                        pairs[atomicSub(&top[e_vw], 1u) - 1u] = make_int2(e_uv, e_uw);
                }
            };
            // TC_RX_UNROLL 32-wide chunks per pass: their loads are in flight
            // before any probe
            for (int64_t cb = b0; cb < b1; cb += 32 * TC_RX_UNROLL) {
                int32_t w[TC_RX_UNROLL];
#pragma unroll
                for (int q = 0; q < TC_RX_UNROLL; ++q) {
                    const int64_t p = cb + 32 * q + lane;
                    w[q] = p < b1 ? col[p] : INT_MAX;
                }
                // rows ascend: once a chunk starts above max N+(u), nothing later matches
                if (__shfl_sync(0xffffffffu, w[0], 0) > umax) break;
                int h[TC_RX_UNROLL];
#pragma unroll
                for (int q = 0; q < TC_RX_UNROLL; ++q)
                    h[q] = w[q] <= umax ? table_find(keys, log_cap, w[q]) : -1;
#pragma unroll
                for (int q = 0; q < TC_RX_UNROLL; ++q) {
                    const int64_t p = cb + 32 * q + lane;
                    if (MODE == LISTS) lists(h[q], p);
                    if (h[q] >= 0) hit(h[q], p);
                }
            }
            c = warp_sum(c);
            if (lane == 0) {
                acc += c;
                if (MODE == SUPPORT && c) atomicAdd(&sup[e_uv], (int)c);
            }
        }
        __syncthreads();
        if (MODE == SUPPORT)
            for (int i = threadIdx.x; i < du; i += RX_THREADS)
                if (cnt[i]) atomicAdd(&sup[eu + i], cnt[i]);
        __syncthreads();
    }
    if (lane == 0) s_acc[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < RX_WARPS; ++w) t += s_acc[w];
        partials[blockIdx.x] = t;
    }
}

// Small out-lists (the largest at most THREAD_MAX_OUT entries): one thread
// per oriented edge (u, v) merges N+(u) and N+(v).  Each common w closes the
// triangle u < v < w.  SUPPORT credits its three edges by atomics; LISTS
// writes the triangle's pair into the three lists, each filled from its top
// by a per-edge cursor.
template <int MODE>
__global__ void __launch_bounds__(IX_THREADS) k_edges_thread(
    const int2* __restrict__ ends, const int64_t* __restrict__ rowptr,
    const int64_t* __restrict__ upper, const int32_t* __restrict__ col,
    const int64_t* __restrict__ oshift, int64_t m, int32_t* __restrict__ sup,
    unsigned int* __restrict__ top, int2* __restrict__ pairs,
    unsigned long long* __restrict__ partials, int32_t bound) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long acc = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const int2 uv = ends[j];
        int64_t a = upper[uv.x], b = upper[uv.y];
        const int64_t a1 = rowptr[uv.x + 1], b1 = rowptr[uv.y + 1];
        const int64_t ou = MODE == COUNT ? 0 : oshift[uv.x];
        const int64_t ov = MODE == COUNT ? 0 : oshift[uv.y];
        uint32_t c = 0;
        while (a < a1 && b < b1) {
            const int32_t x = col[a], y = col[b];
            if (x < y) {
                ++a;
            } else if (x > y) {
                ++b;
            } else {
                ++c;
                if (MODE == SUPPORT) {
                    atomicAdd(&sup[a - ou], 1);
                    atomicAdd(&sup[b - ov], 1);
                }
                if (MODE == LISTS) {
                    const int32_t e_uw = (int32_t)(a - ou), e_vw = (int32_t)(b - ov);
                    const int32_t e_uv = (int32_t)j;
                    if (gets_list(sup, bound, e_uv))
                        pairs[atomicSub(&top[e_uv], 1u) - 1u] = make_int2(e_uw, e_vw);
                    if (gets_list(sup, bound, e_uw))
                        pairs[atomicSub(&top[e_uw], 1u) - 1u] = make_int2(e_uv, e_vw);
                    if (gets_list(sup, bound, e_vw))
                        pairs[atomicSub(&top[e_vw], 1u) - 1u] = make_int2(e_uv, e_uw);
                }
                ++a;
                ++b;
            }
        }
        if (MODE == SUPPORT && c) atomicAdd(&sup[j], (int)c);
        acc += c;
    }
    __shared__ unsigned long long s_acc[IX_THREADS / 32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_acc[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < IX_THREADS / 32; ++w) t += s_acc[w];
        partials[blockIdx.x] = t;
    }
}

// Fallback: one warp per oriented edge; lanes take the shorter out-list's
// elements and look each up in the longer list by binary search.
template <bool SUPPORT>
__global__ void __launch_bounds__(IX_THREADS) k_edges_warp(
    const int2* __restrict__ ends,
    const int64_t* __restrict__ rowptr, const int64_t* __restrict__ upper,
    const int32_t* __restrict__ col, const int64_t* __restrict__ oshift, int64_t m,
    int32_t* __restrict__ sup, unsigned long long* __restrict__ partials) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long acc = 0;
    for (int64_t j = wid; j < m; j += nw) {
        const int32_t e = (int32_t)j;
        const int2 uv = ends[e];
        int64_t s0 = upper[uv.x], s1 = rowptr[uv.x + 1];
        int64_t l0 = upper[uv.y], l1 = rowptr[uv.y + 1];
        int64_t os = SUPPORT ? oshift[uv.x] : 0, ol = SUPPORT ? oshift[uv.y] : 0;
        if (s1 - s0 > l1 - l0) {
            const int64_t t0 = s0, t1 = s1, t2 = os;
            s0 = l0;
            s1 = l1;
            os = ol;
            l0 = t0;
            l1 = t1;
            ol = t2;
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
                    atomicAdd(&sup[p - os], 1);
                    atomicAdd(&sup[lo - ol], 1);
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

// ---- column kernel: the masked product organised by the middle vertex
//
// Every triangle u < v < w (rank order) has exactly one middle vertex v.
// The column kernel takes each column v of the mask L (its in-neighbours u,
// the entries [rowptr[v], upper[v]) of row v), puts N+(v) into a
// shared-memory hash table and, for every in-neighbour u, streams the part
// of N+(u) above v against it: (L L^T)(u, v) = |N+(u) ∩ N+(v)| and only
// w > v can lie in N+(v).  Per oriented edge that reads |N+(u) above v|
// entries instead of the row kernel's |N+(v)|; on R-MAT graphs the total is
// 3-4x smaller (the sum over u of |N+(u)|^2 / 2 against the sum over edges
// of |N+(v)|), because degree ordering makes the lower vertex's out-list the
// short one.
//
// Columns of vertices of degree > LIGHT_DEG (the highest ranks) get one block
// each, its warps sharing the in-neighbours; the rest (most of the vertices)
// get one warp each with a warp-private table, so light columns pay no block
// barrier.  The out-lists are read by edge id (head[e] = the higher end of
// edge e; a row's out-edges have consecutive ids), so in-neighbour u's
// segment of N+(u) after v is head[eid(u, v) + 1 .. iend), iend (the end of
// u's out-edge ids) stored with the in-entry by the build: both come from
// coalesced loads, with no per-neighbour lookups.  Segments longer than
// CX_SHORT are streamed by the whole warp (coalesced, CX_UNROLL chunks in
// flight), shorter ones by one lane each.
//
// Credits of a triangle (u, v, w) found at edge id q of u's out-edges, table
// slot h: (v, w) is the column's own edge (position pos[h] of N+(v)): a
// shared counter, flushed once per column; (u, w) is edge q: a global
// atomic; (u, v): one add per segment.  LISTS writes the pair into the three
// lists: (v, w) from the bottom through the column's shared cursors (its
// bottom entries come only from this column), (u, v) and (u, w) from the top
// through the global per-edge cursors.
//
// Lists for only the edges of support below a bound (LISTS, bound > 0): a
// triangle needs an entry only if one of its edges has a list.  A segment
// is streamed in full only when (u, v) has a list or some edge (v, w) of the
// column does; otherwise only u's low out-entries above v (a compacted list
// per row, lowptr / lowlist) are probed, each hit filling the (u, w) list.

#ifndef TC_CX_SHORT
#define TC_CX_SHORT 16    // in-neighbour segments up to this length: one lane each
#endif
#ifndef TC_CX_UNROLL
#define TC_CX_UNROLL 4    // 32-wide chunks of a long segment in flight per warp pass
#endif
#ifndef TC_CX_SPLIT
#define TC_CX_SPLIT 64    // long segments up to this length: two chunks per pass (0: off)
#endif
#ifndef TC_CX_MIN_BLOCKS
#define TC_CX_MIN_BLOCKS 7  // resident blocks per SM the register allocation must allow (latency-bound: occupancy pays)
#endif
#ifndef TC_CX_LISTS_MIN_BLOCKS
// the list build keeps more live state per entry; its shared-memory use caps it
// at 6 blocks per SM anyway, so it takes the registers of 6 (no spills)
#define TC_CX_LISTS_MIN_BLOCKS 6
#endif
#ifndef TC_CX_FULL_TABLE
#define TC_CX_FULL_TABLE 1  // heavy columns: the whole table, whatever the column's size
#endif
#ifndef TC_CX_BITS
#define TC_CX_BITS 1  // heavy columns spanning <= 32 x table slots of ranks: a bitmap
#endif
#ifndef TC_CX_DYNAMIC
#define TC_CX_DYNAMIC 1     // heavy columns: in-neighbour batches handed out dynamically
#endif
// warp table: 4 slots per entry for <= LIGHT_DEG entries (load <= 1/4)
constexpr int CX_LIGHT_LOG_CAP = LIGHT_DEG <= 64 ? 8 : LIGHT_DEG <= 128 ? 9 : 10;
constexpr int CX_LIGHT_CAP = 1 << CX_LIGHT_LOG_CAP;

struct ColArgs {
    const int64_t* rowptr;
    const int64_t* upper;
    const int32_t* head;   // head[e]: the higher end of edge e
    const int32_t* eid;
    const int32_t* iend;   // per in-entry: end of its neighbour's out-edge ids
    const int64_t* oshift;
    int32_t n;
    int32_t n_light;   // ranks [0, n_light) are light columns
    int32_t* sup;
    const unsigned long long* off;
    unsigned int* top;
    int2* pairs;
    unsigned int* next;  // [0] heavy columns taken, [1] light columns taken
    unsigned long long* partials;
    int max_log_cap;
    int max_pos;
    int* err;
    int32_t bound;                 // LISTS: lists only for supports below it (0: all)
    const unsigned int* lowbits;   // ... one bit per edge: it gets a list
    const unsigned int* lowpos;    // ... low edges with a smaller id (m + 1 entries)
    const int2* lowlist;           // ... {w, edge id} of every low edge, in edge-id order
};

__device__ __forceinline__ bool low_bit(const unsigned int* bits, int32_t e) {
    return (bits[e >> 5] >> (e & 31)) & 1u;
}

// The list build's table: buckets of 4 slots (16 bytes, one shared-memory
// load), linear probing by bucket.  A bucket fills from its first slot on
// (an insert tries slot j only after slot j - 1 is taken), so a lookup ends
// at the first bucket that holds w or has a free last slot.  At a load of
// at most 1/4 (1/2 above 1024 entries) a bucket is rarely full: nearly every
// lookup is one load, and a warp seldom waits on a lane's longer probe run.
// (The support and count passes keep one slot per probe: there the 16-byte
// loads' extra shared-memory wavefronts cost more than the probe runs.)
__device__ __forceinline__ uint32_t bucket_of(int32_t w, int log_nb) {
    return ((uint32_t)w * 0x9E3779B1u) >> (32 - log_nb);
}

__device__ __forceinline__ int table4_find(const int32_t* keys, int log_cap, int32_t w) {
    const int log_nb = log_cap - 2;
    const uint32_t bmask = (1u << log_nb) - 1;
    uint32_t b = bucket_of(w, log_nb);
    for (;;) {
        const int4 k = reinterpret_cast<const int4*>(keys)[b];
        const int j = k.x == w ? 0 : k.y == w ? 1 : k.z == w ? 2 : k.w == w ? 3 : -1;
        if (j >= 0) return (int)(4 * b) + j;
        if (k.w == -1) return -1;
        b = (b + 1) & bmask;
    }
}

// Inserts w (not yet present) and returns its slot.
__device__ __forceinline__ int table4_insert(int32_t* keys, int log_cap, int32_t w) {
    const int log_nb = log_cap - 2;
    const uint32_t bmask = (1u << log_nb) - 1;
    uint32_t b = bucket_of(w, log_nb);
    for (;;) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (atomicCAS(&keys[4 * b + j], -1, w) == -1) return (int)(4 * b) + j;
        b = (b + 1) & bmask;
    }
}

// The column kernel's table by mode: LISTS buckets, the others single slots.
template <int MODE>
__device__ __forceinline__ int col_find(const int32_t* keys, int log_cap, int32_t w) {
    return MODE == LISTS ? table4_find(keys, log_cap, w) : table_find(keys, log_cap, w);
}

template <int MODE>
__device__ __forceinline__ int col_insert(int32_t* keys, int log_cap, int32_t w) {
    if (MODE == LISTS) return table4_insert(keys, log_cap, w);
    const uint32_t mask = (1u << log_cap) - 1;
    uint32_t h = slot_of(w, log_cap);
    while (atomicCAS(&keys[h], -1, w) != -1) h = (h + 1) & mask;
    return (int)h;
}

// Column v's out-list N+(v) as the streaming loops see it: find(w) is w's
// position in N+(v), or -1.  Callers pass only w with v < w <= max N+(v).
// HashTab: the hash table above, with each slot's position beside it.
template <typename P>
struct HashTab {
    const int32_t* keys;
    const P* pos;
    int log_cap;
    template <int MODE>
    __device__ __forceinline__ int find(int32_t w) const {
        const int h = col_find<MODE>(keys, log_cap, w);
        return h >= 0 ? (int)pos[h] : -1;
    }
};

// BitTab: one bit per rank in (v, max N+(v)] (bit w - v - 1), for columns
// whose out-list spans few enough ranks (the bits fit where the hash table's
// keys would be).  A probe is one 4-byte shared-memory load with no probe
// run.  pre[j] is the position in N+(v) of the first entry in word j (set
// only for words that hold one), so a set bit's position is pre[j] plus the
// set bits below it in its word.
struct BitTab {
    const uint32_t* bits;
    const uint16_t* pre;
    int32_t v;
    template <int MODE>
    __device__ __forceinline__ int find(int32_t w) const {
        const uint32_t b = (uint32_t)(w - v - 1);
        const uint32_t word = bits[b >> 5], bit = 1u << (b & 31);
        return (word & bit) ? (int)pre[b >> 5] + __popc(word & (bit - 1u)) : -1;
    }
};

// One long segment of an in-neighbour u (edge ids [ss, se) of u's out-edges,
// above v) streamed by the whole warp against column v's table, U chunks of
// 32 entries in flight; returns this lane's hits (LISTS: entries read).
template <int MODE, int U, typename Tab>
__device__ __forceinline__ uint32_t stream_segment(const ColArgs& a, const Tab& t, int32_t* cnt,
                                                   const unsigned int* sbase, int64_t ev,
                                                   int32_t vmax, bool partial, int32_t ss,
                                                   int32_t se, int32_t suv, bool sluv) {
    // edge ids (below 2^31) index the segment: 32-bit arithmetic throughout
    const int lane = threadIdx.x & 31;
    uint32_t c = 0;
    for (int32_t cb = ss; cb < se; cb += 32 * U) {
        int32_t w[U];
        if (cb + 32 * U <= se) {  // a full pass: no bounds checks
#pragma unroll
            for (int q = 0; q < U; ++q) w[q] = a.head[cb + 32 * q + lane];
            if (MODE == LISTS) c += U;  // LISTS counts the entries read (this lane's)
        } else {
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int32_t p = cb + 32 * q + lane;
                w[q] = p < se ? a.head[p] : INT_MAX;
                if (MODE == LISTS) c += p < se;
            }
        }
        // segments ascend: once a chunk starts above max N+(v), nothing later matches
        if (__shfl_sync(0xffffffffu, w[0], 0) > vmax) break;
        int h[U];
#pragma unroll
        for (int q = 0; q < U; ++q)
            h[q] = w[q] <= vmax ? t.template find<MODE>(w[q]) : -1;  // position in N+(v)
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int32_t p = cb + 32 * q + lane;
            if (MODE == LISTS) {
                // the chunk's triangles share (u, v): one top append for all
                const unsigned msk = __ballot_sync(0xffffffffu, h[q] >= 0);
                if (msk) {
                    const int ldr = __ffs(msk) - 1;
                    unsigned base = 0;
                    if (lane == ldr && sluv)
                        base = atomicSub(&a.top[suv], (unsigned)__popc(msk));
                    base = __shfl_sync(0xffffffffu, base, ldr) - (unsigned)__popc(msk);
                    if (h[q] >= 0) {
                        const int iw = h[q];
                        const int32_t e_vw = (int32_t)(ev + iw), e_uw = (int32_t)p;
                        if (sluv)
                            a.pairs[base + __popc(msk & lanemask_lt())] =
                                make_int2(e_uw, e_vw);
                        if (!partial || low_bit(a.lowbits, e_uw))
                            a.pairs[atomicSub(&a.top[e_uw], 1u) - 1u] = make_int2(suv, e_vw);
                        if (sbase[iw] != 0xffffffffu)
                            a.pairs[sbase[iw] + atomicAdd((unsigned int*)&cnt[iw], 1u)] =
                                make_int2(suv, e_uw);
                    }
                }
            }
            if (h[q] >= 0) {
                if (MODE != LISTS) ++c;
                if (MODE == SUPPORT) {  // (v, w) on the column's counter, (u, w) = edge p
                    atomicAdd(&cnt[h[q]], 1);
                    atomicAdd(&a.sup[p], 1);
                }
            }
        }
    }
    return c;
}

// One column's in-neighbours [i0, i1), in batches of 32 per warp; returns
// the triangles found (LISTS: the 4-byte words of out-lists read instead).
// Tab: column v's out-list (HashTab or BitTab).
template <int MODE, typename Tab>
__device__ __forceinline__ unsigned long long col_walk(const ColArgs& a, const Tab& t, int32_t* cnt,
                                                       const unsigned int* sbase, int64_t ev,
                                                       int32_t vmax, bool col_low, int64_t i0,
                                                       int64_t i1, unsigned int* next,
                                                       int64_t stride = 32) {
    const int lane = threadIdx.x & 31;
    const bool partial = MODE == LISTS && a.bound > 0;
    unsigned long long acc = 0;
    // batches of in-neighbours: handed out by the shared counter (a block's
    // warps sharing a column take them as they finish), or all to this warp.
    // A shared column with few in-neighbours uses smaller batches (down to
    // 4, about two per warp) so that every warp gets some; lanes past the
    // batch take none, long segments are still streamed by the whole warp.
    int bsz = 32;
    if (next) {
        const int64_t want = (i1 - i0 + 2 * RX_WARPS - 1) / (2 * RX_WARPS);
        bsz = (int)max((int64_t)4, min((int64_t)32, want));
    }
    auto take = [&](int64_t done) -> int64_t {
        if (!next) return done;  // static: i0, i0 + stride, ...
        unsigned b = 0;
        if (lane == 0) b = atomicAdd(next, (unsigned)bsz);
        return i0 + (int64_t)__shfl_sync(0xffffffffu, b, 0);
    };
    for (int64_t ib = take(i0); ib < i1; ib = take(ib + stride)) {
        const int64_t i = lane < bsz ? ib + lane : i1;  // lanes past the batch: none
        int32_t s = 0, end = 0;  // edge ids: below 2^31
        int32_t e_uv = 0;
        bool luv = true;   // (u, v) has a list
        bool full = true;  // the whole segment is streamed
        if (i < i1) {
            e_uv = a.eid[i];
            s = e_uv + 1;                 // u's out-edges after (u, v), by edge id
            end = a.iend[i - ev];         // in-entries of column v start at index rowptr[v] - ev
            if (partial) {
                luv = low_bit(a.lowbits, e_uv);
                full = luv || col_low;
            }
        }
        const int32_t len = full ? end - s : 0;
        // a triangle (u, v, w): w at edge id q of u's out-edges, position h of N+(v)
        auto hit_support = [&](int h, int32_t q) {
            atomicAdd(&cnt[h], 1);
            atomicAdd(&a.sup[q], 1);
        };
        // long segments: the whole warp, one after another
        unsigned lng = __ballot_sync(0xffffffffu, len > TC_CX_SHORT);
        while (lng) {
            const int src = __ffs(lng) - 1;
            lng &= lng - 1;
            const int32_t ss = __shfl_sync(0xffffffffu, s, src);
            const int32_t se = __shfl_sync(0xffffffffu, end, src);
            const int32_t suv = __shfl_sync(0xffffffffu, e_uv, src);
            const bool sluv = __shfl_sync(0xffffffffu, luv, src);
            // segments up to TC_CX_SPLIT entries: two chunks per pass (fewer idle
            // lanes in their one pass); longer ones TC_CX_UNROLL (more loads in flight)
            uint32_t c = (TC_CX_SPLIT > 0 && se - ss <= TC_CX_SPLIT)
                             ? stream_segment<MODE, 2>(a, t, cnt, sbase, ev, vmax, partial, ss,
                                                       se, suv, sluv)
                             : stream_segment<MODE, TC_CX_UNROLL>(a, t, cnt, sbase, ev, vmax,
                                                                   partial, ss, se, suv, sluv);
            c = __reduce_add_sync(0xffffffffu, c);
            if (lane == 0) {
                acc += c;
                if (MODE == SUPPORT && c) atomicAdd(&a.sup[suv], (int)c);
            }
        }
        // short segments: one lane each, four entries in flight
        if (len > 0 && len <= TC_CX_SHORT) {
            uint32_t c = 0;
            for (int32_t p = s; p < end; p += 4) {
                int32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) w[q] = p + q < end ? a.head[p + q] : INT_MAX;
                if (MODE == LISTS) c += (uint32_t)min(4, end - p);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (w[q] > vmax) continue;
                    const int h = t.template find<MODE>(w[q]);  // position in N+(v)
                    if (h < 0) continue;
                    if (MODE != LISTS) ++c;
                    if (MODE == SUPPORT) hit_support(h, p + q);
                    if (MODE == LISTS) {
                        const int iw = h;
                        const int32_t e_vw = (int32_t)(ev + iw), e_uw = (int32_t)(p + q);
                        if (luv) a.pairs[atomicSub(&a.top[e_uv], 1u) - 1u] = make_int2(e_uw, e_vw);
                        if (!partial || low_bit(a.lowbits, e_uw))
                            a.pairs[atomicSub(&a.top[e_uw], 1u) - 1u] = make_int2(e_uv, e_vw);
                        if (sbase[iw] != 0xffffffffu)
                            a.pairs[sbase[iw] + atomicAdd((unsigned int*)&cnt[iw], 1u)] =
                                make_int2(e_uv, e_uw);
                    }
                }
                if (w[3] > vmax) break;
            }
            acc += c;
            if (MODE == SUPPORT && c) atomicAdd(&a.sup[e_uv], (int)c);
        }
        // lists below a bound, segment not streamed: only u's low out-entries
        // above v can close a triangle that needs an entry, in the (u, w) list
        if (partial && i < i1 && !full && s < end) {
            // u's low out-entries after v: edge ids e_uv + 1 .. end - 1
            const unsigned int l1 = a.lowpos[end];
            for (unsigned int q = a.lowpos[e_uv + 1]; q < l1; ++q) {
                const int2 we = a.lowlist[q];  // {w, edge id of (u, w)}
                acc += 2;                      // an 8-byte entry read
                if (we.x > vmax) break;
                const int h = t.template find<MODE>(we.x);
                if (h < 0) continue;
                const int32_t e_vw = (int32_t)(ev + h);
                a.pairs[atomicSub(&a.top[we.y], 1u) - 1u] = make_int2(e_uv, e_vw);
            }
        }
    }
    return acc;
}

template <int MODE>
__global__ void __launch_bounds__(RX_THREADS, MODE == LISTS ? TC_CX_LISTS_MIN_BLOCKS : TC_CX_MIN_BLOCKS)
    k_cols(ColArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_col;
    __shared__ unsigned int s_next;  // heavy column: next in-neighbour batch (offset)
    __shared__ unsigned long long s_acc[RX_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long acc = 0;
    const int32_t n_heavy = a.n - a.n_light;

    // heavy columns, highest rank first: one block each
    {
        const int max_cap = 1 << a.max_log_cap;
        int32_t* keys = reinterpret_cast<int32_t*>(smem);
        uint16_t* pos = reinterpret_cast<uint16_t*>(keys + max_cap);
        int32_t* cnt = reinterpret_cast<int32_t*>(pos + max_cap);
        unsigned int* sbase = reinterpret_cast<unsigned int*>(cnt + a.max_pos);
        for (;;) {
            if (threadIdx.x == 0) {
                s_col = (int)atomicAdd(&a.next[0], 1u);
                s_next = 0;
            }
            __syncthreads();
            const int c = s_col;
            __syncthreads();
            if (c >= n_heavy) break;
            const int32_t v = a.n - 1 - c;
            const int64_t i0 = a.rowptr[v], b0 = a.upper[v], b1 = a.rowptr[v + 1];
            const int dv = (int)(b1 - b0);
            if (dv < 1 || b0 == i0) continue;  // no out-list or no in-neighbour: no triangle
            const int64_t ev = b0 - a.oshift[v];  // first out-edge id of v
            // the block's table is sized for the largest column: a smaller
            // column may use all of it (lower load, shorter probe runs)
            const int log_cap = TC_CX_FULL_TABLE ? a.max_log_cap
                                                 : min(table_log_cap(dv), a.max_log_cap);
            const int cap = 1 << log_cap;
            for (int i = threadIdx.x; i < cap; i += RX_THREADS) keys[i] = -1;
            bool low = false;  // some edge (v, w) of the column has a list
            if (MODE != COUNT)
                for (int i = threadIdx.x; i < dv; i += RX_THREADS) {
                    cnt[i] = 0;
                    if (MODE == LISTS) {
                        const bool has = a.bound == 0 || low_bit(a.lowbits, (int32_t)(ev + i));
                        sbase[i] = has ? (unsigned int)a.off[ev + i] : 0xffffffffu;
                        low |= has && a.bound > 0;
                    }
                }
            const bool col_low = __syncthreads_or(low) != 0;
            const int32_t vmax = a.head[ev + dv - 1];
            // an out-list within 32 x cap ranks above v: a bitmap of those
            // ranks in the keys' space, first positions per word in pos's
            const int64_t span = (int64_t)vmax - v;  // bits 0 .. span - 1
            if (TC_CX_BITS && span <= 32 * (int64_t)max_cap) {
                uint32_t* bits = reinterpret_cast<uint32_t*>(keys);
                const int nw = (int)((span + 31) >> 5);
                for (int i = threadIdx.x; i < nw; i += RX_THREADS) bits[i] = 0u;
                __syncthreads();
                for (int i = threadIdx.x; i < dv; i += RX_THREADS) {
                    const uint32_t b = (uint32_t)(a.head[ev + i] - v - 1);
                    atomicOr(&bits[b >> 5], 1u << (b & 31));
                    if (i == 0 || (uint32_t)(a.head[ev + i - 1] - v - 1) >> 5 != b >> 5)
                        pos[b >> 5] = (uint16_t)i;  // N+(v) ascends: i is the word's first
                }
                __syncthreads();
                const BitTab t{bits, pos, v};
                if (TC_CX_DYNAMIC)
                    acc += col_walk<MODE>(a, t, cnt, sbase, ev, vmax, col_low, i0, b0, &s_next);
                else
                    acc += col_walk<MODE>(a, t, cnt, sbase, ev, vmax, col_low, i0 + 32 * warp, b0,
                                          nullptr, 32 * RX_WARPS);
            } else {
                for (int i = threadIdx.x; i < dv; i += RX_THREADS)
                    pos[col_insert<MODE>(keys, log_cap, a.head[ev + i])] = (uint16_t)i;
                __syncthreads();
                const HashTab<uint16_t> t{keys, pos, log_cap};
                if (TC_CX_DYNAMIC)
                    acc += col_walk<MODE>(a, t, cnt, sbase, ev, vmax, col_low, i0, b0, &s_next);
                else
                    acc += col_walk<MODE>(a, t, cnt, sbase, ev, vmax, col_low, i0 + 32 * warp, b0,
                                          nullptr, 32 * RX_WARPS);
            }
            __syncthreads();
            if (MODE == SUPPORT)
                for (int i = threadIdx.x; i < dv; i += RX_THREADS)
                    if (cnt[i]) atomicAdd(&a.sup[ev + i], cnt[i]);
            __syncthreads();
        }
    }

    // light columns: one warp each, warp-private table; each warp takes 32
    // columns at a time (one counter update per 32 columns)
    {
        constexpr int per_warp = CX_LIGHT_CAP * 4 + CX_LIGHT_CAP + LIGHT_DEG * 8;
        unsigned char* base = smem + (size_t)warp * per_warp;
        int32_t* keys = reinterpret_cast<int32_t*>(base);
        uint8_t* pos = reinterpret_cast<uint8_t*>(keys + CX_LIGHT_CAP);
        int32_t* cnt = reinterpret_cast<int32_t*>(pos + CX_LIGHT_CAP);
        unsigned int* sbase = reinterpret_cast<unsigned int*>(cnt + LIGHT_DEG);
        for (;;) {
            unsigned c0 = 0;
            if (lane == 0) c0 = atomicAdd(&a.next[1], 32u);
            c0 = __shfl_sync(0xffffffffu, c0, 0);
            if (c0 >= (unsigned)a.n_light) break;
            const int cend = (int)min((unsigned)a.n_light, c0 + 32u);
            for (int c = (int)c0; c < cend; ++c) {
                const int32_t v = a.n_light - 1 - c;
                const int64_t i0 = a.rowptr[v], b0 = a.upper[v], b1 = a.rowptr[v + 1];
                const int dv = (int)(b1 - b0);
                if (dv < 1 || b0 == i0) continue;
                // the warp table is sized for LIGHT_DEG entries; a light
                // column's out-list is at most its degree (never taken)
                if (dv > LIGHT_DEG) {
                    if (lane == 0) atomicOr(a.err, DEV_ERR_BOUNDS);
                    continue;
                }
                const int64_t ev = b0 - a.oshift[v];  // first out-edge id of v
                for (int i = lane; i < CX_LIGHT_CAP; i += 32) keys[i] = -1;
                bool low = false;
                if (MODE != COUNT)
                    for (int i = lane; i < dv; i += 32) {
                        cnt[i] = 0;
                        if (MODE == LISTS) {
                            const bool has = a.bound == 0 || low_bit(a.lowbits, (int32_t)(ev + i));
                            sbase[i] = has ? (unsigned int)a.off[ev + i] : 0xffffffffu;
                            low |= has && a.bound > 0;
                        }
                    }
                const bool col_low = __any_sync(0xffffffffu, low);
                __syncwarp();
                for (int i = lane; i < dv; i += 32)
                    pos[col_insert<MODE>(keys, CX_LIGHT_LOG_CAP, a.head[ev + i])] = (uint8_t)i;
                __syncwarp();
                const int32_t vmax = a.head[ev + dv - 1];
                const HashTab<uint8_t> t{keys, pos, CX_LIGHT_LOG_CAP};
                acc += col_walk<MODE>(a, t, cnt, sbase, ev, vmax, col_low, i0, b0, nullptr, 32);
                __syncwarp();
                if (MODE == SUPPORT)
                    for (int i = lane; i < dv; i += 32)
                        if (cnt[i]) atomicAdd(&a.sup[ev + i], cnt[i]);
                __syncwarp();
            }
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) s_acc[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < RX_WARPS; ++w) t += s_acc[w];
        a.partials[blockIdx.x] = t;
    }
}

// Dynamic shared memory of the column kernel: the heavy columns' table and
// per-position arrays (as the row kernel's), or the warps' light tables,
// whichever is larger (the two phases reuse the same memory).
size_t cols_smem(int log_cap, int mode, int max_pos) {
    const size_t cap = (size_t)1 << log_cap;
    const size_t per = mode == SUPPORT ? 4 : mode == LISTS ? 8 : 0;
    const size_t heavy = cap * 4 + cap * 2 + per * (size_t)std::max(max_pos, 1) + 16;
    const size_t light = (size_t)RX_WARPS * (CX_LIGHT_CAP * 4 + CX_LIGHT_CAP + LIGHT_DEG * 8);
    return std::max(heavy, light);
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

// out[0] = sum over oriented edges of |N+(u)| + |N+(v)|; out[1] = sum over
// rows u of |N+(u)| (|N+(u)| - 1) / 2.
__global__ void k_wedge_work(const int2* __restrict__ ends,
                             const int64_t* __restrict__ rowptr, const int64_t* __restrict__ upper,
                             int64_t m, int32_t n, unsigned long long* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long acc = 0, cw = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const int2 uv = ends[j];
        acc += (unsigned long long)(rowptr[uv.x + 1] - upper[uv.x]) +
               (unsigned long long)(rowptr[uv.y + 1] - upper[uv.y]);
    }
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const unsigned long long d = (unsigned long long)(rowptr[r + 1] - upper[r]);
        cw += d * (d - (d > 0)) / 2;
    }
    acc = warp_sum(acc);
    cw = warp_sum(cw);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], acc);
        atomicAdd(&out[1], cw);
    }
}

// ---- 64-bit exclusive scan of int32 values (offsets of the triangle lists)

constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 8;
constexpr int SC_CHUNK = SC_THREADS * SC_ITEMS;

__device__ unsigned long long block_sum64(unsigned long long v, unsigned long long* sh) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        sh[32] = t;
    }
    __syncthreads();
    t = sh[32];
    __syncthreads();
    return t;
}

// Values at or above `bound` (when bound > 0) count as 0: the offsets of
// lists kept only for the edges whose support is below it.
__device__ __forceinline__ unsigned long long bounded(int32_t x, int32_t bound) {
    return (bound > 0 && x >= bound) ? 0ull : (unsigned long long)x;
}

__global__ void __launch_bounds__(SC_THREADS) k_chunk_sums(const int32_t* __restrict__ x,
                                                           int64_t n, int32_t bound,
                                                           unsigned long long* __restrict__ sums) {
    __shared__ unsigned long long sh[33];
    const int64_t base = (int64_t)blockIdx.x * SC_CHUNK;
    unsigned long long v = 0;
    for (int i = threadIdx.x; i < SC_CHUNK; i += SC_THREADS)
        if (base + i < n) v += bounded(x[base + i], bound);
    const unsigned long long t = block_sum64(v, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
}

__global__ void __launch_bounds__(1024) k_scan_sums64(unsigned long long* __restrict__ v,
                                                      int64_t count) {
    __shared__ unsigned long long sh[1024];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < count; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const unsigned long long x = i < count ? v[i] : 0ull;
        sh[threadIdx.x] = x;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
            const unsigned long long y = threadIdx.x >= o ? sh[threadIdx.x - o] : 0ull;
            __syncthreads();
            sh[threadIdx.x] += y;
            __syncthreads();
        }
        if (i < count) v[i] = carry + sh[threadIdx.x] - x;
        __syncthreads();
        if (threadIdx.x == 0) carry += sh[1023];
        __syncthreads();
    }
}

// off[i] = sum of x[0..i); off[n] = total.
__global__ void __launch_bounds__(SC_THREADS) k_chunk_scan(const int32_t* __restrict__ x, int64_t n,
                                                           int32_t bound,
                                                           const unsigned long long* __restrict__ sums,
                                                           unsigned long long* __restrict__ off) {
    __shared__ unsigned long long sh[SC_THREADS];
    const int64_t base = (int64_t)blockIdx.x * SC_CHUNK;
    // each thread owns SC_ITEMS consecutive values
    unsigned long long loc[SC_ITEMS];
    unsigned long long tsum = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        const int64_t i = base + (int64_t)threadIdx.x * SC_ITEMS + k;
        loc[k] = i < n ? bounded(x[i], bound) : 0ull;
        tsum += loc[k];
    }
    sh[threadIdx.x] = tsum;
    __syncthreads();
    for (int o = 1; o < SC_THREADS; o <<= 1) {
        const unsigned long long y = threadIdx.x >= o ? sh[threadIdx.x - o] : 0ull;
        __syncthreads();
        sh[threadIdx.x] += y;
        __syncthreads();
    }
    unsigned long long run = sums[blockIdx.x] + sh[threadIdx.x] - tsum;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        const int64_t i = base + (int64_t)threadIdx.x * SC_ITEMS + k;
        if (i < n) off[i] = run;
        if (i == n - 1) off[n] = run + loc[k];
        run += loc[k];
    }
}

__global__ void k_u32_from_u64(const unsigned long long* __restrict__ in, int64_t n,
                               unsigned int* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = (unsigned int)in[i];
}

// Sum of the supports in (0, bound) and the number of such edges.
__global__ void k_low_sums(const int32_t* __restrict__ sup, int64_t m, int32_t bound,
                           unsigned long long* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long e = 0, c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int32_t x = sup[i];
        const bool low = x > 0 && x < bound;
        e += low ? (unsigned long long)x : 0ull;
        c += low;
    }
    e = warp_sum(e);
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], e);
        atomicAdd(&out[1], c);
    }
}

// Edges with a support in (0, bound) ("low": the edges that get lists):
// lowbits holds one bit per edge; lowpos[e] counts the low edges with id
// below e (m + 1 entries, an exclusive scan); lowlist[lowpos[e]] = {head
// w of e, e} for every low e.  Edge ids follow the out-lists, so the low
// out-entries of u after its out-neighbour v (edge e_uv) are lowlist
// [lowpos[e_uv + 1], lowpos[end of u's out-edges]).
__device__ __forceinline__ bool is_low(int32_t x, int32_t bound) { return x > 0 && x < bound; }

__global__ void __launch_bounds__(SC_THREADS) k_low_chunk_counts(const int32_t* __restrict__ sup,
                                                                 int64_t m, int32_t bound,
                                                                 unsigned int* __restrict__ lowbits,
                                                                 unsigned long long* __restrict__ sums) {
    __shared__ unsigned long long sh[33];
    const int64_t base = (int64_t)blockIdx.x * SC_CHUNK;
    unsigned long long c = 0;
    for (int i = threadIdx.x; i < SC_CHUNK; i += SC_THREADS) {
        const int64_t e = base + i;
        const bool low = e < m && is_low(sup[e], bound);
        const unsigned bits = __ballot_sync(0xffffffffu, low);
        if ((threadIdx.x & 31) == 0 && e < m) lowbits[e >> 5] = bits;
        c += low;
    }
    const unsigned long long t = block_sum64(c, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
}

__global__ void __launch_bounds__(SC_THREADS) k_low_scan(const int32_t* __restrict__ sup,
                                                         const int2* __restrict__ ends, int64_t m,
                                                         int32_t bound,
                                                         const unsigned long long* __restrict__ sums,
                                                         unsigned int* __restrict__ lowpos,
                                                         int2* __restrict__ lowlist) {
    __shared__ unsigned int sh[SC_THREADS];
    const int64_t base = (int64_t)blockIdx.x * SC_CHUNK;
    bool low[SC_ITEMS];
    unsigned int tsum = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        const int64_t e = base + (int64_t)threadIdx.x * SC_ITEMS + k;
        low[k] = e < m && is_low(sup[e], bound);
        tsum += low[k];
    }
    sh[threadIdx.x] = tsum;
    __syncthreads();
    for (int o = 1; o < SC_THREADS; o <<= 1) {
        const unsigned int y = threadIdx.x >= o ? sh[threadIdx.x - o] : 0u;
        __syncthreads();
        sh[threadIdx.x] += y;
        __syncthreads();
    }
    unsigned int run = (unsigned int)sums[blockIdx.x] + sh[threadIdx.x] - tsum;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        const int64_t e = base + (int64_t)threadIdx.x * SC_ITEMS + k;
        if (e < m) {
            lowpos[e] = run;
            if (low[k]) lowlist[run] = make_int2(ends[e].y, (int32_t)e);
        }
        if (e == m - 1) lowpos[m] = run + low[k];
        run += low[k];
    }
}

// The block's table must hold the largest table any row up to max_out
// entries asks for; table_log_cap is not monotone across the sparse limit,
// so take both regimes' largest.
int max_table_log_cap(int max_out) {
    return std::max(table_log_cap(std::min(max_out, (int)TC_RX_SPARSE_LIMIT)),
                    table_log_cap(max_out));
}

int rows_log_cap(const Graph* g) { return max_table_log_cap(g->max_out); }

// Table (keys + positions) and the per-position arrays of SUPPORT (4 B) and
// LISTS (12 B) for out-lists of up to max_pos entries.
size_t rows_smem(int log_cap, int mode, int max_pos) {
    const size_t cap = (size_t)1 << log_cap;
    const size_t per = mode == SUPPORT ? 4 : mode == LISTS ? 12 : 0;
    return cap * 4 + cap * 2 + per * (size_t)std::max(max_pos, 1) + 16;
}

// The row kernel's dynamic shared memory depends on the graph.  The
// function attribute that allows it is process-wide, so it is raised once
// per device to the largest size any graph can need and never lowered:
// concurrent calls on graphs of different sizes must not undercut each other.
int ensure_rows_smem_limit() {
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    TC_CUDA_TRY(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return TC_OK;
    const int sm_max = (int)rows_smem(max_table_log_cap(RX_MAX_OUT), LISTS, RX_MAX_OUT);
    TC_CUDA_TRY(cudaFuncSetAttribute(k_rows<COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_max));
    TC_CUDA_TRY(cudaFuncSetAttribute(k_rows<SUPPORT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_max));
    TC_CUDA_TRY(cudaFuncSetAttribute(k_rows<LISTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_max));
    done.fetch_or(bit);
    return TC_OK;
}

template <int MODE>
int launch_rows(Graph* g, int32_t* sup, const unsigned long long* off, unsigned int* top,
                int2* pairs, unsigned long long* partials, int blocks, cudaStream_t s,
                int32_t bound = 0) {
    TC_TRY(ensure_rows_smem_limit());
    if (g->max_out > RX_MAX_OUT) return fail(TC_EINVAL, "internal: row kernel above its table size");
    const int lc = rows_log_cap(g);
    const int max_pos = std::max(g->max_out, 1);
    const size_t sm = rows_smem(lc, MODE, max_pos);
    unsigned int* next_row = reinterpret_cast<unsigned int*>(g->dev_scalars + 4);
    TC_CUDA_TRY(cudaMemsetAsync(next_row, 0, sizeof(unsigned int), s));
    k_rows<MODE><<<blocks, RX_THREADS, sm, s>>>(g->rowptr, g->upper, g->col, g->oshift, g->n, sup,
                                                off, top, pairs, next_row, partials, lc,
                                                max_pos, bound);
    TC_LAUNCH_CHECK("k_rows");
    return TC_OK;
}

int ensure_cols_smem_limit() {
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    TC_CUDA_TRY(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return TC_OK;
    const int sm_max = (int)cols_smem(max_table_log_cap(RX_MAX_OUT), LISTS, RX_MAX_OUT);
    TC_CUDA_TRY(cudaFuncSetAttribute(k_cols<COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_max));
    TC_CUDA_TRY(cudaFuncSetAttribute(k_cols<SUPPORT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_max));
    TC_CUDA_TRY(cudaFuncSetAttribute(k_cols<LISTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_max));
    done.fetch_or(bit);
    return TC_OK;
}

template <int MODE>
int launch_cols(Graph* g, int32_t* sup, const unsigned long long* off, unsigned int* top,
                int2* pairs, unsigned long long* partials, int blocks, cudaStream_t s,
                int32_t bound = 0, const unsigned int* lowbits = nullptr,
                const unsigned int* lowpos = nullptr, const int2* lowlist = nullptr) {
    TC_TRY(ensure_cols_smem_limit());
    if (g->max_out > RX_MAX_OUT) return fail(TC_EINVAL, "internal: column kernel above its table size");
    const int lc = rows_log_cap(g);
    const int max_pos = std::max(g->max_out, 1);
    const size_t sm = cols_smem(lc, MODE, max_pos);
    unsigned int* next = reinterpret_cast<unsigned int*>(g->dev_scalars + 5);
    TC_CUDA_TRY(cudaMemsetAsync(next, 0, 2 * sizeof(unsigned int), s));
    // light columns: degree <= the graph's bound (16, 32, 64 or LIGHT_DEG)
    int li = 3;
    while (li > 0 && (16 << li) > g->col_light_deg) --li;
    ColArgs a{g->rowptr, g->upper, g->head, g->eid, g->iend, g->oshift, g->n, g->light_rows[li], sup,
              off, top, pairs, next, partials, lc, max_pos, g->dev_err, bound, lowbits, lowpos,
              lowlist};
    k_cols<MODE><<<blocks, RX_THREADS, sm, s>>>(a);
    TC_LAUNCH_CHECK("k_cols");
    return TC_OK;
}

int cols_blocks(Graph* g, int mode) {
    int per_sm = 0;
    const size_t sm = cols_smem(rows_log_cap(g), mode, std::max(g->max_out, 1));
    cudaError_t e = cudaSuccess;
    if (ensure_cols_smem_limit() != TC_OK) per_sm = 1;
    else if (mode == COUNT)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cols<COUNT>, RX_THREADS, sm);
    else if (mode == SUPPORT)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cols<SUPPORT>, RX_THREADS, sm);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cols<LISTS>, RX_THREADS, sm);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return num_sms() * per_sm;
}

int rows_blocks(Graph* g, int mode) {
    int per_sm = 0;
    const size_t sm = rows_smem(rows_log_cap(g), mode, std::max(g->max_out, 1));
    cudaError_t e = cudaSuccess;
    if (ensure_rows_smem_limit() != TC_OK) per_sm = 1;
    else if (mode == COUNT)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rows<COUNT>, RX_THREADS, sm);
    else if (mode == SUPPORT)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rows<SUPPORT>, RX_THREADS, sm);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rows<LISTS>, RX_THREADS, sm);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return num_sms() * per_sm;
}

}  // namespace

int graph_wedge_work(Graph* g, int64_t* out, cudaStream_t s) {
    if (g->wedge_work < 0) {
        unsigned long long h[2] = {0, 0};
        if (g->m > 0) {
            TC_CUDA_TRY(cudaMemsetAsync(g->dev_scalars + 2, 0, 2 * sizeof(unsigned long long), s));
            k_wedge_work<<<num_sms() * 8, 256, 0, s>>>(g->ends, g->rowptr, g->upper, g->m, g->n,
                                                       g->dev_scalars + 2);
            TC_LAUNCH_CHECK("k_wedge_work");
            TC_CUDA_TRY(cudaMemcpyAsync(h, g->dev_scalars + 2, sizeof(h), cudaMemcpyDeviceToHost, s));
            TC_CUDA_TRY(cudaStreamSynchronize(s));
        }
        g->wedge_work = (int64_t)h[0];
        g->column_work = (int64_t)h[1];
    }
    *out = g->wedge_work;
    return TC_OK;
}

// The intersection kernel a call uses: 1 = by columns (k_cols: hash table
// of N+(v), in-neighbours' segments streamed), 2 = one warp per oriented
// edge, 3 = one thread per oriented edge, 4 = by rows (k_rows: hash table of
// N+(u), out-neighbours' lists streamed).  form 0 (automatic, unless the
// test hook forces one): threads for small out-lists, columns while the
// largest out-list fits the table, else warps.
int concrete_form(const Graph* g, int form) {
    const int f = form != 0 ? form : intersect_mode();
    if (f == 3) return 3;
    if (f == 2) return 2;
    if (f == 1 || f == 4) return g->max_out <= RX_MAX_OUT ? f : 2;
    if (g->max_out <= THREAD_MAX_OUT) return 3;
    return g->max_out <= RX_MAX_OUT ? 1 : 2;
}

int product_blocks(Graph* g, int f, int mode) {
    return f == 1 ? cols_blocks(g, mode) : f == 4 ? rows_blocks(g, mode) : num_sms() * 8;
}

int compute_support(Graph* g, int32_t* sup, bool want_support, int64_t* triangles,
                    cudaStream_t s, int form) {
    const int64_t m = g->m;
    if (m == 0) {
        if (triangles) *triangles = 0;
        return TC_OK;
    }
    const int f = concrete_form(g, form);
    const int blocks = product_blocks(g, f, want_support ? SUPPORT : COUNT);
    g->stats.product_form = f;
    Scratch sc(s);
    unsigned long long* partials;
    TC_TRY(sc.alloc(&partials, blocks));
    if (want_support) TC_CUDA_TRY(cudaMemsetAsync(sup, 0, sizeof(int32_t) * m, s));
    KernelTimer timer;
    TC_TRY(timer.start(s));
    if (f == 1) {
        if (want_support)
            TC_TRY(launch_cols<SUPPORT>(g, sup, nullptr, nullptr, nullptr, partials, blocks, s));
        else TC_TRY(launch_cols<COUNT>(g, nullptr, nullptr, nullptr, nullptr, partials, blocks, s));
    } else if (f == 4) {
        if (want_support)
            TC_TRY(launch_rows<SUPPORT>(g, sup, nullptr, nullptr, nullptr, partials, blocks, s));
        else TC_TRY(launch_rows<COUNT>(g, nullptr, nullptr, nullptr, nullptr, partials, blocks, s));
    } else if (f == 3) {
        if (want_support)
            k_edges_thread<SUPPORT><<<blocks, IX_THREADS, 0, s>>>(
                g->ends, g->rowptr, g->upper, g->col, g->oshift, m, sup, nullptr, nullptr, partials,
                0);
        else
            k_edges_thread<COUNT><<<blocks, IX_THREADS, 0, s>>>(
                g->ends, g->rowptr, g->upper, g->col, g->oshift, m, nullptr, nullptr, nullptr,
                partials, 0);
        TC_LAUNCH_CHECK("k_edges_thread");
    } else if (want_support) {
        k_edges_warp<true><<<blocks, IX_THREADS, 0, s>>>(g->ends, g->rowptr, g->upper,
                                                         g->col, g->oshift, m, sup, partials);
        TC_LAUNCH_CHECK("k_edges_warp");
    } else {
        k_edges_warp<false><<<blocks, IX_THREADS, 0, s>>>(g->ends, g->rowptr, g->upper,
                                                          g->col, g->oshift, m, nullptr, partials);
        TC_LAUNCH_CHECK("k_edges_warp");
    }
    TC_TRY(timer.stop(s));
    k_reduce_partials<<<1, 1024, 0, s>>>(partials, blocks, g->dev_scalars);
    TC_LAUNCH_CHECK("k_reduce_partials");
    if (triangles) {
        unsigned long long t = 0;
        TC_CUDA_TRY(cudaMemcpyAsync(&t, g->dev_scalars, sizeof(t), cudaMemcpyDeviceToHost, s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
        *triangles = (int64_t)t;
        (want_support ? g->stats.support_ns : g->stats.count_ns) = timer.elapsed_ns();
    }
    return TC_OK;
}

bool triangle_lists_supported(const Graph* g) { return g->max_out <= RX_MAX_OUT; }

namespace {
__global__ void k_gather_i32(const int32_t* __restrict__ in, const int32_t* __restrict__ inv,
                             int64_t m, int32_t* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < m; c += stride)
        out[c] = in[inv[c]];
}
}  // namespace

int to_canonical_i32(const int32_t* in, const int32_t* inv, int64_t m, int32_t* out,
                     cudaStream_t s) {
    if (m == 0) return TC_OK;
    k_gather_i32<<<(unsigned)std::min<int64_t>((m + 255) / 256, (int64_t)num_sms() * 16), 256, 0,
                   s>>>(in, inv, m, out);
    TC_LAUNCH_CHECK("k_gather_i32");
    return TC_OK;
}

int exclusive_scan_i32(const int32_t* x, int64_t n, unsigned long long* out, Scratch& sc,
                       cudaStream_t s) {
    if (n <= 0) {
        TC_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(unsigned long long), s));
        return TC_OK;
    }
    const int64_t chunks = (n + SC_CHUNK - 1) / SC_CHUNK;
    unsigned long long* sums;
    TC_TRY(sc.alloc(&sums, chunks));
    k_chunk_sums<<<(unsigned)chunks, SC_THREADS, 0, s>>>(x, n, 0, sums);
    TC_LAUNCH_CHECK("k_chunk_sums");
    k_scan_sums64<<<1, 1024, 0, s>>>(sums, chunks);
    TC_LAUNCH_CHECK("k_scan_sums64");
    k_chunk_scan<<<(unsigned)chunks, SC_THREADS, 0, s>>>(x, n, 0, sums, out);
    TC_LAUNCH_CHECK("k_chunk_scan");
    return TC_OK;
}

int partial_list_entries(Graph* g, int32_t bound, int64_t* entries, int64_t* low_edges,
                         cudaStream_t s) {
    unsigned long long h[2] = {0, 0};
    if (g->m > 0) {
        unsigned long long* d = g->dev_scalars + 6;
        TC_CUDA_TRY(cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), s));
        k_low_sums<<<(unsigned)std::min<int64_t>((g->m + 255) / 256, (int64_t)num_sms() * 8), 256, 0,
                     s>>>(g->support, g->m, bound, d);
        TC_LAUNCH_CHECK("k_low_sums");
        TC_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
    }
    *entries = (int64_t)h[0];
    if (low_edges) *low_edges = (int64_t)h[1];
    return TC_OK;
}

int plan_triangle_lists(Graph* g, Scratch& sc, ListsPlan* lp) {
    const int64_t m = g->m;
    lp->chunks = (m + SC_CHUNK - 1) / SC_CHUNK;
    TC_TRY(sc.alloc(&lp->sums, lp->chunks));
    TC_TRY(sc.alloc(&lp->top, m));
    if (lp->bound > 0) {
        // the column kernel's low edges: bits, positions, compacted list
        TC_TRY(sc.alloc(&lp->lowbits, m / 32 + 1));
        TC_TRY(sc.alloc(&lp->lowpos, m + 1));
        TC_TRY(sc.alloc(&lp->lowsums, lp->chunks));
        TC_TRY(sc.alloc(&lp->lowlist, std::max<int64_t>(1, lp->low_edges)));
    }
    lp->form = concrete_form(g, 0);
    if (lp->form == 2) lp->form = 1;  // lists need a table kernel (the caller checked the size)
    // every edge's list: the row kernel fills two of a triangle's three lists
    // through its shared cursors (the column kernel only one), measured
    // faster; lists below a bound: the column kernel, which skips segments
    if (lp->form == 1 && lp->bound == 0 && intersect_mode() == 0) lp->form = 4;
    lp->thread = lp->form == 3;
    lp->blocks = product_blocks(g, lp->form, LISTS);
    TC_TRY(sc.alloc(&lp->partials, lp->blocks));
    return TC_OK;
}

// Offsets = exclusive scan of the supports; then every triangle writes its
// pair into the lists of its three edges.  List positions fit in 32 bits
// (the caller keeps 3T below 2^32), so a 4-byte top cursor per edge
// (starting at the end of its list) keeps the cursor array small enough for L2.
int enqueue_triangle_lists(Graph* g, const int32_t* sup, unsigned long long* off, int2* pairs,
                           ListsPlan* lp, cudaStream_t s) {
    const int64_t m = g->m;
    k_chunk_sums<<<(unsigned)lp->chunks, SC_THREADS, 0, s>>>(sup, m, lp->bound, lp->sums);
    TC_LAUNCH_CHECK("k_chunk_sums");
    k_scan_sums64<<<1, 1024, 0, s>>>(lp->sums, lp->chunks);
    TC_LAUNCH_CHECK("k_scan_sums64");
    k_chunk_scan<<<(unsigned)lp->chunks, SC_THREADS, 0, s>>>(sup, m, lp->bound, lp->sums, off);
    TC_LAUNCH_CHECK("k_chunk_scan");
    if (lp->bound > 0 && lp->form == 1) {
        k_low_chunk_counts<<<(unsigned)lp->chunks, SC_THREADS, 0, s>>>(sup, m, lp->bound,
                                                                      lp->lowbits, lp->lowsums);
        TC_LAUNCH_CHECK("k_low_chunk_counts");
        k_scan_sums64<<<1, 1024, 0, s>>>(lp->lowsums, lp->chunks);
        TC_LAUNCH_CHECK("k_scan_sums64");
        k_low_scan<<<(unsigned)lp->chunks, SC_THREADS, 0, s>>>(sup, g->ends, m, lp->bound,
                                                              lp->lowsums, lp->lowpos, lp->lowlist);
        TC_LAUNCH_CHECK("k_low_scan");
    }
    k_u32_from_u64<<<(unsigned)std::min<int64_t>((m + 255) / 256, (int64_t)num_sms() * 16), 256, 0,
                     s>>>(off + 1, m, lp->top);
    TC_LAUNCH_CHECK("k_u32_from_u64");
    TC_TRY(lp->timer.start(s));
    int32_t* sup_rw = const_cast<int32_t*>(sup);  // read-only in LISTS mode
    if (lp->thread) {
        k_edges_thread<LISTS><<<lp->blocks, IX_THREADS, 0, s>>>(
            g->ends, g->rowptr, g->upper, g->col, g->oshift, m, sup_rw, lp->top, pairs,
            lp->partials, lp->bound);
        TC_LAUNCH_CHECK("k_edges_thread");
    } else if (lp->form == 4) {
        TC_TRY(launch_rows<LISTS>(g, sup_rw, off, lp->top, pairs, lp->partials, lp->blocks, s,
                                  lp->bound));
    } else {
        TC_TRY(launch_cols<LISTS>(g, sup_rw, off, lp->top, pairs, lp->partials, lp->blocks, s,
                                  lp->bound, lp->lowbits, lp->lowpos, lp->lowlist));
    }
    TC_TRY(lp->timer.stop(s));
    if (lp->form == 1) {  // the column kernel's words read, for its algorithmic bytes
        k_reduce_partials<<<1, 1024, 0, s>>>(lp->partials, lp->blocks, g->dev_scalars + 7);
        TC_LAUNCH_CHECK("k_reduce_partials");
    }
    return TC_OK;
}

}  // namespace tc
