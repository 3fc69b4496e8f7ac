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
//   then the dying edges are removed (state = k - 1, their truss number).
// The decomposition runs k = 3, 4, ... on the survivors of the previous level
// until no edge is left.
//
// All levels and rounds run inside one persistent cooperative kernel whose
// blocks meet at grid barriers between phases; every barrier wait is bounded
// in time (on expiry the kernel sets an abort flag and every block returns).
// When at least half of the adjacency entries belong to removed edges, the
// rows are compacted in place so later rounds scan only live entries.
//
// Edge state t[e]: 0 = alive, -1 = in the current frontier, > 0 = removed.
#include <algorithm>
#include <climits>
#include <new>

#include "tc_internal.cuh"

namespace tc {
namespace {

#ifndef TC_PK_THREADS
#define TC_PK_THREADS 1024
#endif
constexpr int PK_THREADS = TC_PK_THREADS;
constexpr int PK_WARPS = PK_THREADS / 32;
#ifndef TC_PK_WINDOW
#define TC_PK_WINDOW 16
#endif
constexpr int WINDOW = TC_PK_WINDOW;  // support values one full scan covers (see k_peel)
#ifndef TC_PK_HEAVY
#define TC_PK_HEAVY 4096             // triangle-list length above which an edge is "heavy"
#endif
constexpr int64_t HEAVY = TC_PK_HEAVY;

#ifndef TC_PK_LANE_EDGES
#define TC_PK_LANE_EDGES 32          // frontier edges per warp from which lanes take one each
#endif
#ifndef TC_PK_SHORT_LIST
#define TC_PK_SHORT_LIST 32          // ... and walk lists up to this length alone
#endif
constexpr int64_t LANE_EDGES = TC_PK_LANE_EDGES;
constexpr int64_t SHORT_LIST = TC_PK_SHORT_LIST;
#ifndef TC_PK_MAX_BLOCKS
#define TC_PK_MAX_BLOCKS (1 << 20)   // cap on the peel's grid
#endif
#ifndef TC_PK_UNROLL
#define TC_PK_UNROLL 3               // triangle-list entries per lane in flight
#endif
#ifndef TC_PK_SCAN_UNROLL
#define TC_PK_SCAN_UNROLL 4          // level scan: 32-edge chunks per warp iteration
#endif

struct PeelCtl {
    unsigned long long bar;      // grid-barrier arrivals (monotonic)
    unsigned long long cntA[2];  // alive-list appends, by full-scan parity (monotonic)
    unsigned long long cntW[2];  // window-list appends, by level parity
    unsigned long long cntF[2];  // light-frontier appends, by round parity
    unsigned long long cntH[2];  // heavy-frontier appends, by round parity
    unsigned long long cntZ;     // edges of support 0 removed by a level scan (monotonic)
    int minenc[3];               // per level (mod 3): INT_MAX - smallest alive support scanned
    int abort;                   // 1 = a barrier wait ran out of time
    int kmax;                    // decomposition result
    int overflow;                // 1 = the round table ran out (not expected)
    int pad;
    long long n_alive;           // edges left after the last level
    long long rounds;            // non-empty rounds
    long long compactions;
    long long full_scans;
    unsigned long long scanned;   // level-scan entries read
    unsigned long long entries;   // triangle-list entries (TL) or shorter-list entries (IX) read
    unsigned long long searches;  // binary-search loads (IX)
    unsigned long long lookups;   // edge-state loads while processing frontiers
    unsigned long long lowered;   // support decrements
};

// Per-thread work counters, summed into PeelCtl at the end.
struct Tally {
    unsigned long long scanned = 0, entries = 0, searches = 0, lookups = 0, lowered = 0;
};

struct PeelArgs {
    int64_t m;
    int32_t n;
    const int2* ends;
    const int64_t* rowptr;
    int32_t* rowlen;  // live length of each row (rows compact in place)
    int32_t* col;     // working copies of the adjacency
    int32_t* eid;
    int32_t* t;       // edge state (see below)
    int32_t* s;
    int32_t* A[2];    // alive lists
    int32_t* W[2];    // window lists
    int32_t* F[2];    // light frontiers
    int32_t* H[2];    // heavy frontiers
    uint2* FR[2];     // list form: triangle-list range {q0, q1} of each F entry
    uint2* HR[2];     // ... and of each H entry
    int32_t* level_of;  // level k of each round number
    int64_t max_round;  // entries of level_of
    PeelCtl* ctl;
    const unsigned long long* off;  // triangle-list mode: list of edge e = pairs[off[e]..off[e+1])
    const int2* pairs;              // the two other edges of each triangle through e
    int32_t k_first;
    int32_t r_first;  // first round number (2 when resuming: state -1 = removed before)
    int32_t single;  // 1: peel level k_first only
    int32_t no_compact;  // 1: col / eid are the graph's own (read only): never compact
    int32_t k_last;      // decomposition: stop after level k_last (0: until empty)
    long long* level_left;  // ... and record the k-truss size of levels k_first..k_last
    int64_t spin_ns;
};

// Loads of data that other blocks write during the kernel go through L2.
__device__ __forceinline__ int ld_cg(const int32_t* p) { return __ldcg(p); }

// Binary-search probes of a live neighbour list go through L1: the upper
// levels of a search are shared by the lanes and warps searching the same
// list (9% faster at R-MAT scale 24).  The lists change only while rows are
// compacted, a phase that ends at a grid barrier, whose acquire (the fence
// after the poll, then the block barrier) orders every later load after the
// compaction's writes.
__device__ __forceinline__ int ld_search(const int32_t* p) { return __ldca(p); }

__device__ __forceinline__ unsigned long long ld_vol(const unsigned long long* p) {
    return *(const volatile unsigned long long*)p;
}

// Grid barrier: monotonic arrival counter; bounded wait.  Returns false on
// abort (every caller then returns from the kernel).
__device__ bool grid_sync(PeelCtl* ctl, unsigned long long* epoch, int64_t spin_ns, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        *epoch += 1;
        const unsigned long long target = *epoch * (unsigned long long)gridDim.x;
        __threadfence();
        atomicAdd(&ctl->bar, 1ull);
        uint64_t t0 = 0;
        // relaxed polls (one round trip each; the fence after the loop gives
        // the acquire), the abort flag read every 16th poll
        for (unsigned polls = 0;
             ld_relaxed_u64(reinterpret_cast<const uint64_t*>(&ctl->bar)) < target; ++polls) {
            if ((polls & 15) == 15 && *(volatile int*)&ctl->abort) {
                ok = 0;
                break;
            }
            const uint64_t now = global_timer_ns();
            if (t0 == 0) {
                t0 = now;
            } else if ((int64_t)(now - t0) > spin_ns) {
                atomicExch(&ctl->abort, 1);
                ok = 0;
                break;
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Edge states during round r: 0 = alive; -r = in round r's frontier (dying);
// -(r + 1) = alive, already in the next frontier; -q with q < r = removed in
// round q.  Stamping states with round numbers needs no pass that retires a
// frontier: the next round reads the round number instead.
struct Round {
    int32_t r;
    __device__ bool removed(int32_t st) const { return st < 0 && st > -r; }
    __device__ bool dying(int32_t st) const { return st == -r; }
    __device__ bool alive(int32_t st) const { return st == 0 || st == -(r + 1); }
};

// Where a round's appends go (counters and bases are uniform per phase).
struct Sinks {
    int32_t* Fn;
    int32_t* Hn;
    uint2* FRn;  // list form: the entries' list ranges
    uint2* HRn;
    int32_t* Wc;
    unsigned long long* cntF;
    unsigned long long* cntH;
    unsigned long long* cntW;
    unsigned long long baseF, baseH, baseW;
    int32_t thr;    // frontier threshold k - 2
    int32_t bound;  // window bound: the window list holds alive edges with s < bound
};

// List form: edge e's triangle list is pairs[q0, q1).  Positions are below
// 2^32 (the list form needs 3T < 2^32).  Frontier entries carry this range,
// so processing an entry does not wait for an offset load.
__device__ __forceinline__ uint2 list_range(const PeelArgs& a, int32_t e) {
    return make_uint2((unsigned)a.off[e], (unsigned)a.off[e + 1]);
}

__device__ __forceinline__ bool is_heavy(uint2 rg) { return (int64_t)(rg.y - rg.x) > HEAVY; }

// The crossing checks after a decrement of alive edge x returned old: x
// joins the next frontier when its support falls from k - 2 to k - 3 and the
// window list when it falls to just below the window bound (exactly one
// decrement sees each crossing).  x < 0: no decrement.  The list length
// (heavy or not) is read only for a crossing edge: reading it for every
// decrement costs more than the extra latency of the few crossings.
// One atomic per append: warp-aggregating these appends measured slower.
template <bool TL>
__device__ __forceinline__ void after_lower(const PeelArgs& a, Round rd, int32_t x, int old,
                                            const Sinks& k) {
    if (x < 0) return;
    if (old == k.thr) {
        a.t[x] = -(rd.r + 1);
        if (TL) {
            const uint2 rg = list_range(a, x);
            if (is_heavy(rg)) {
                const unsigned long long q = atomicAdd(k.cntH, 1ull) - k.baseH;
                k.Hn[q] = x;
                k.HRn[q] = rg;
            } else {
                const unsigned long long q = atomicAdd(k.cntF, 1ull) - k.baseF;
                k.Fn[q] = x;
                k.FRn[q] = rg;
            }
        } else {
            k.Fn[atomicAdd(k.cntF, 1ull) - k.baseF] = x;
        }
    }
    if (old == k.bound) k.Wc[atomicAdd(k.cntW, 1ull) - k.baseW] = x;
}

// Lowers the support of alive edge x by one.
template <bool TL>
__device__ __forceinline__ void lower(const PeelArgs& a, Round rd, int32_t x, const Sinks& k,
                                      Tally& tl) {
    ++tl.lowered;
    after_lower<TL>(a, rd, x, atomicSub(a.s + x, 1), k);
}

// A frontier edge's triangle {e, f, g} whose other two edges are not yet
// removed is destroyed this round; the smallest dying edge of the triangle
// owns it and lowers the support of each of f, g that is not dying.
template <bool TL>
__device__ __forceinline__ void destroy(const PeelArgs& a, Round rd, int32_t e, int32_t f,
                                        int32_t tf, int32_t g, int32_t tg, const Sinks& k,
                                        Tally& tl) {
    if ((rd.dying(tf) && f < e) || (rd.dying(tg) && g < e)) return;
    if (rd.alive(tf)) lower<TL>(a, rd, f, k, tl);
    if (rd.alive(tg)) lower<TL>(a, rd, g, k, tl);
}

// All triangles through frontier edge e, by a group of gsize lanes (rg: its
// triangle-list range, when lists exist).  The edge's current support is
// exactly its number of live triangles (those whose other two edges are not
// removed): support 0 means nothing to do, and a single-warp group stops
// once it has seen them all.  TL: edges have triangle lists (with IX, only
// some do: an edge with live triangles and an empty range has none);
// IX: the live neighbour lists are kept for intersecting.
template <bool TL, bool IX>
__device__ __forceinline__ void process_edge(const PeelArgs& a, Round rd, int32_t e, uint2 rg,
                                             int64_t glane, int64_t gsize, const Sinks& k,
                                             Tally& tl) {
    const bool one_warp = gsize == 32;
    int32_t seen = 0;  // live triangles met so far (one_warp only; warp-uniform)
    if (TL && (!IX || rg.y > rg.x)) {
        const int64_t q0 = rg.x, q1 = rg.y;
        const int32_t live = ld_cg(a.s + e);
        if (live <= 0) return;
        // PU entries per lane in flight: the pair loads, then both state
        // loads of each pair, then every decrement, then their checks
        constexpr int PU = TC_PK_UNROLL;
        for (int64_t b = q0; b < q1; b += gsize * PU) {  // b is uniform in the group
            int2 fg[PU];
            bool v[PU];
#pragma unroll
            for (int u = 0; u < PU; ++u) {
                const int64_t q = b + glane + (int64_t)u * gsize;
                v[u] = q < q1;
                fg[u] = v[u] ? a.pairs[q] : make_int2(0, 0);
            }
            int32_t tf[PU], tg[PU];
#pragma unroll
            for (int u = 0; u < PU; ++u) {
                tf[u] = v[u] ? ld_cg(a.t + fg[u].x) : 1;
                tg[u] = v[u] ? ld_cg(a.t + fg[u].y) : 1;
            }
            int32_t xf[PU], xg[PU];
            int of[PU] = {}, og[PU] = {};
            int found = 0;
#pragma unroll
            for (int u = 0; u < PU; ++u) {
                xf[u] = -1;
                xg[u] = -1;
                if (v[u]) {
                    ++tl.entries;
                    tl.lookups += 2;
                }
                if (v[u] && !rd.removed(tf[u]) && !rd.removed(tg[u])) {
                    ++found;
                    // the smallest dying edge of the triangle owns it
                    const bool own = !((rd.dying(tf[u]) && fg[u].x < e) ||
                                       (rd.dying(tg[u]) && fg[u].y < e));
                    if (own && rd.alive(tf[u])) xf[u] = fg[u].x;
                    if (own && rd.alive(tg[u])) xg[u] = fg[u].y;
                }
            }
#pragma unroll
            for (int u = 0; u < PU; ++u) {
                if (xf[u] >= 0) of[u] = atomicSub(a.s + xf[u], 1);
                if (xg[u] >= 0) og[u] = atomicSub(a.s + xg[u], 1);
            }
#pragma unroll
            for (int u = 0; u < PU; ++u) {
                tl.lowered += (xf[u] >= 0) + (xg[u] >= 0);
                after_lower<TL>(a, rd, xf[u], of[u], k);
                after_lower<TL>(a, rd, xg[u], og[u], k);
            }
            if (one_warp) {
                seen += __reduce_add_sync(0xffffffffu, (unsigned)found);
                if (seen >= live) break;
            } else if (gsize == 1) {  // one lane alone
                seen += found;
                if (seen >= live) break;
            }
        }
        return;
    }
    if (!IX) return;
    const int32_t live = ld_cg(a.s + e);
    if (live <= 0) return;
    const int2 ab = a.ends[e];
    int64_t s0 = a.rowptr[ab.x], l0 = a.rowptr[ab.y];
    int32_t sl = ld_cg(a.rowlen + ab.x), ll = ld_cg(a.rowlen + ab.y);
    if (sl > ll) {
        const int64_t t0 = s0;
        s0 = l0;
        l0 = t0;
        const int32_t t1 = sl;
        sl = ll;
        ll = t1;
    }
    for (int64_t cb = (glane & ~31ll); cb < sl; cb += gsize) {
        const int64_t p = cb + (glane & 31);
        bool found = false;
        if (p < sl) {
            ++tl.entries;
            const int32_t f = ld_cg(a.eid + s0 + p);
            const int32_t tf = ld_cg(a.t + f);
            ++tl.lookups;
            if (!rd.removed(tf)) {
                const int32_t w = ld_cg(a.col + s0 + p);
                int32_t lo = 0, hi = ll;
                while (lo < hi) {
                    const int32_t mid = (lo + hi) >> 1;
                    ++tl.searches;
                    if (ld_search(a.col + l0 + mid) < w) lo = mid + 1;
                    else hi = mid;
                }
                if (lo < ll && ld_search(a.col + l0 + lo) == w) {
                    const int32_t g = ld_cg(a.eid + l0 + lo);
                    const int32_t tg = ld_cg(a.t + g);
                    ++tl.lookups;
                    if (!rd.removed(tg)) {
                        found = true;
                        destroy<TL>(a, rd, e, f, tf, g, tg, k, tl);
                    }
                }
            }
        }
        if (one_warp) {
            seen += __popc(__ballot_sync(0xffffffffu, found));
            if (seen >= live) break;
        }
    }
}

// Groups of W warps per edge (W a power of two, as wide as the list count
// allows, spanning blocks when the list is short); each group takes edges
// round-robin.
template <bool TL, bool IX>
__device__ __forceinline__ void process_list(const PeelArgs& a, Round rd, const int32_t* L,
                                             const uint2* LR, int64_t nL, int64_t gwarp,
                                             int64_t nwarps, const Sinks& k, Tally& tl) {
    if (nL == 0) return;
    if (TL && nL >= nwarps * LANE_EDGES) {
        // many edges per warp: each lane takes one; lists of up to
        // SHORT_LIST entries are walked by their lane alone, longer ones (and,
        // with IX, edges without a list, whose neighbour lists are
        // intersected) by the whole warp, one after another
        const int lane = threadIdx.x & 31;
        for (int64_t base = gwarp * 32; base < nL; base += nwarps * 32) {
            const int64_t j = base + lane;
            const int32_t e = j < nL ? ld_cg(L + j) : -1;
            const uint2 rg = j < nL ? __ldcg(LR + j) : make_uint2(0, 0);
            const bool longer =
                e >= 0 && ((int64_t)(rg.y - rg.x) > SHORT_LIST || (IX && rg.y == rg.x));
            if (e >= 0 && !longer) process_edge<TL, IX>(a, rd, e, rg, 0, 1, k, tl);
            unsigned rest = __ballot_sync(0xffffffffu, longer);
            while (rest) {
                const int src = __ffs(rest) - 1;
                rest &= rest - 1;
                const uint2 rs = make_uint2(__shfl_sync(0xffffffffu, rg.x, src),
                                            __shfl_sync(0xffffffffu, rg.y, src));
                process_edge<TL, IX>(a, rd, __shfl_sync(0xffffffffu, e, src), rs, lane, 32, k, tl);
            }
        }
        return;
    }
    int64_t W = 1;
    while (nL * (W * 2) <= nwarps) W *= 2;
    const int64_t ngroups = nwarps / W;
    const int64_t group = gwarp / W;
    if (group >= ngroups) return;
    const int64_t glane = (gwarp % W) * 32 + (threadIdx.x & 31);
    for (int64_t j = group; j < nL; j += ngroups)
        process_edge<TL, IX>(a, rd, ld_cg(L + j), TL ? __ldcg(LR + j) : make_uint2(0, 0), glane,
                             32 * W, k, tl);
}

// The peel.  Levels k = k_first, k_first + 1, ...; each level starts with a
// scan that collects the edges below the threshold (the first frontier) and
// then runs rounds until no frontier is left.  A full scan (of every alive
// edge) also collects the "window": alive edges with support below
// thr + WINDOW.  The next levels scan only the window, because every edge
// that can join their frontiers is in it: supports only fall, and an edge
// whose support falls below the window bound during a round is appended to
// the window at that moment.  Once the threshold passes the bound, the next
// level makes a full scan again.
//
// TL: an edge's triangles come from its precomputed triangle list; IX:
// from the intersection of its endpoints' live neighbour lists.  Both: the
// list when the edge has one (lists were built only for edges whose support
// was below a bound), else the intersection.
template <bool TL, bool IX>
__global__ void __launch_bounds__(PK_THREADS) k_peel(PeelArgs a) {
    __shared__ int s_ok;
    unsigned long long epoch = 0;
    PeelCtl* ctl = a.ctl;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t gwarp = (int64_t)blockIdx.x * PK_WARPS + wib;
    const int64_t nwarps = (int64_t)gridDim.x * PK_WARPS;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;

    unsigned long long baseA[2] = {0, 0}, baseW[2] = {0, 0}, baseF[2] = {0, 0},
                       baseH[2] = {0, 0}, baseZ = 0;
    int ai = 0, wi = 0, fi = 0;  // which buffer of each pair is the current one
    bool first = true;           // the first full scan reads every edge id
    int64_t nA = a.m;            // entries of the current alive list
    int64_t nW = 0;              // entries of the current window list
    int64_t n_alive = a.m;
    int64_t nnz = 2 * a.m;
    int64_t rounds = 0, compactions = 0, fulls = 0;
    int32_t k = a.k_first;
    int32_t kmax = 2;
    int32_t r = a.r_first;  // round whose frontier the next level scan collects
    int32_t bound = INT_MIN;
    int level = 0;
    Tally tl;

    for (;;) {
        if (r + 2 >= a.max_round) {  // uniform: every block sees the same r
            if (leader) ctl->overflow = 1;
            return;
        }
        const int32_t thr = k - 2;
        const bool full = thr > bound;
        if (full) bound = thr + WINDOW;
        const int wp = level & 1, pf = r & 1, pa = (int)(fulls & 1);
        if (leader) a.level_of[r] = k;
        int32_t* Wout = a.W[wi ^ 1];
        {
            const int32_t* in = full ? (first ? nullptr : a.A[ai]) : a.W[wi];
            const int64_t n_in = full ? nA : nW;
            int32_t* Aout = a.A[ai ^ 1];
            const int ms = level % 3;
            // the slot the level after next uses: clear it for that level
            if (leader) ctl->minenc[(level + 1) % 3] = 0;
            int smin = INT_MAX;  // smallest support among the alive edges scanned
            // Two passes over the warp's share: the first classifies every
            // scanned edge (marking the frontier) and counts what each list
            // receives; one atomic per warp and list then reserves the
            // ranges, and the second pass writes the entries.  (An append per
            // 32 edges serialised millions of atomics on one counter in a
            // full scan.)  A call that peels one level never scans again: it
            // needs neither the alive list (only its length) nor the window.
            const bool wantA = full && !a.single, wantW = !a.single;
            // SU chunks of 32 edges per warp iteration, all loads in flight
            // before any is used (the scan is bound by load latency)
            constexpr int SU = TC_PK_SCAN_UNROLL;
            const int64_t wstep = nwarps * 32 * SU;
            // An edge below the threshold with support 0 is in no live
            // triangle: removing it lowers no other support, so it is stamped
            // with the round number (removed in round r, as the frontier is)
            // but joins no frontier list (counted in cZ instead).
            unsigned long long cA = 0, cW = 0, cF = 0, cH = 0, cZ = 0;
            for (int64_t base = gwarp * 32 * SU; base < n_in; base += wstep) {
                int32_t e[SU], te[SU], se[SU];
#pragma unroll
                for (int u = 0; u < SU; ++u) {
                    const int64_t i = base + 32 * u + lane;
                    e[u] = i < n_in ? (in ? ld_cg(in + i) : (int32_t)i) : -1;
                }
#pragma unroll
                for (int u = 0; u < SU; ++u) {
                    // state and support loaded together (scanned edges are
                    // mostly alive)
                    te[u] = e[u] >= 0 ? ld_cg(a.t + e[u]) : 1;
                    se[u] = e[u] >= 0 ? ld_cg(a.s + e[u]) : 0;
                }
#pragma unroll
                for (int u = 0; u < SU; ++u) {
                    bool alive = false, win = false, light = false, heavy = false, zero = false;
                    if (e[u] >= 0) {
                        ++tl.scanned;
                        alive = te[u] == 0;
                        if (alive) {
                            smin = min(smin, se[u]);
                            win = se[u] < bound;
                            if (se[u] < thr) {
                                a.t[e[u]] = -r;
                                zero = se[u] == 0;
                                heavy = !zero && TL && is_heavy(list_range(a, e[u]));
                                light = !zero && !heavy;
                            }
                        }
                    }
                    cA += __popc(__ballot_sync(0xffffffffu, alive));
                    cW += __popc(__ballot_sync(0xffffffffu, win));
                    cF += __popc(__ballot_sync(0xffffffffu, light));
                    cH += __popc(__ballot_sync(0xffffffffu, heavy));
                    cZ += __popc(__ballot_sync(0xffffffffu, zero));
                }
            }
            smin = __reduce_min_sync(0xffffffffu, smin);
            if (lane == 0 && smin != INT_MAX) atomicMax(&ctl->minenc[ms], INT_MAX - smin);
            unsigned long long rA = 0, rW = 0, rF = 0, rH = 0;
            if (lane == 0) {
                if (full && cA) rA = atomicAdd(&ctl->cntA[pa], cA);
                if (wantW && cW) rW = atomicAdd(&ctl->cntW[wp], cW);
                if (cF) rF = atomicAdd(&ctl->cntF[pf], cF);
                if (cH) rH = atomicAdd(&ctl->cntH[pf], cH);
                if (cZ) atomicAdd(&ctl->cntZ, cZ);
            }
            rA = __shfl_sync(0xffffffffu, rA, 0) - baseA[pa];
            rW = __shfl_sync(0xffffffffu, rW, 0) - baseW[wp];
            rF = __shfl_sync(0xffffffffu, rF, 0) - baseF[pf];
            rH = __shfl_sync(0xffffffffu, rH, 0) - baseH[pf];
            if ((wantA && cA) || (wantW && cW) || cF || cH) {
                for (int64_t base = gwarp * 32 * SU; base < n_in; base += wstep) {
                    int32_t e[SU], te[SU];
#pragma unroll
                    for (int u = 0; u < SU; ++u) {
                        const int64_t i = base + 32 * u + lane;
                        e[u] = i < n_in ? (in ? ld_cg(in + i) : (int32_t)i) : -1;
                    }
#pragma unroll
                    for (int u = 0; u < SU; ++u) te[u] = e[u] >= 0 ? ld_cg(a.t + e[u]) : 1;
#pragma unroll
                    for (int u = 0; u < SU; ++u) {
                        bool alive = false, win = false, light = false, heavy = false;
                        uint2 rg = make_uint2(0, 0);
                        if (e[u] >= 0) {
                            // this scan's frontier carries the (fresh) round number
                            const bool front = te[u] == -r;
                            alive = te[u] == 0 || front;
                            if (alive && wantW) win = ld_cg(a.s + e[u]) < bound;
                            // (the frontier leaves out edges of support 0)
                            if (front && ld_cg(a.s + e[u]) > 0) {
                                if (TL) rg = list_range(a, e[u]);
                                heavy = TL && is_heavy(rg);
                                light = !heavy;
                            }
                        }
                        const unsigned lt = lanemask_lt();
                        if (wantA) {
                            const unsigned mk = __ballot_sync(0xffffffffu, alive);
                            if (alive) Aout[rA + __popc(mk & lt)] = e[u];
                            rA += __popc(mk);
                        }
                        if (wantW) {
                            const unsigned mk = __ballot_sync(0xffffffffu, win);
                            if (win) Wout[rW + __popc(mk & lt)] = e[u];
                            rW += __popc(mk);
                        }
                        {
                            const unsigned mk = __ballot_sync(0xffffffffu, light);
                            if (light) {
                                const unsigned long long q = rF + __popc(mk & lt);
                                a.F[fi][q] = e[u];
                                if (TL) a.FR[fi][q] = rg;
                            }
                            rF += __popc(mk);
                        }
                        {
                            const unsigned mk = __ballot_sync(0xffffffffu, heavy);
                            if (heavy) {
                                const unsigned long long q = rH + __popc(mk & lt);
                                a.H[fi][q] = e[u];
                                if (TL) a.HR[fi][q] = rg;
                            }
                            rH += __popc(mk);
                        }
                    }
                }
            }
        }
        if (!grid_sync(ctl, &epoch, a.spin_ns, &s_ok)) return;
        if (full) {
            const unsigned long long endA = ld_vol(&ctl->cntA[pa]);
            nA = (int64_t)(endA - baseA[pa]);
            baseA[pa] = endA;
            n_alive = nA;
            ai ^= 1;
            first = false;
            ++fulls;
        }
        int64_t nF, nH;
        {
            const unsigned long long eF = ld_vol(&ctl->cntF[pf]), eH = ld_vol(&ctl->cntH[pf]);
            nF = (int64_t)(eF - baseF[pf]);
            nH = (int64_t)(eH - baseH[pf]);
            baseF[pf] = eF;
            baseH[pf] = eH;
            const unsigned long long eZ = ld_vol(&ctl->cntZ);
            n_alive -= (int64_t)(eZ - baseZ);  // support-0 edges: removed now
            baseZ = eZ;
        }
        // no edge below the threshold: levels up to the smallest alive
        // support + 2 remove nothing either (their k-trusses are all alive
        // edges), so the next level to peel is that support + 3
        int32_t k_next = k + 1;
        if (nF + nH == 0) {
            int32_t m0 = INT_MAX - *(volatile int*)&ctl->minenc[level % 3];
            if (!full) m0 = min(m0, bound);  // edges outside the window have s >= bound
            if (m0 != INT_MAX && m0 + 3 > k_next) k_next = m0 + 3;
        }
        ++level;

        while (nF + nH > 0) {
            if (r + 2 >= a.max_round) {
                if (leader) ctl->overflow = 1;
                return;
            }
            ++rounds;
            const Round rd{r};
            const int pn = (r + 1) & 1;
            if (leader) a.level_of[r + 1] = k;
            const Sinks sk{a.F[fi ^ 1], a.H[fi ^ 1], a.FR[fi ^ 1], a.HR[fi ^ 1], Wout,
                           &ctl->cntF[pn], &ctl->cntH[pn], &ctl->cntW[wp], baseF[pn],
                           baseH[pn], baseW[wp], thr, a.single ? INT_MIN : bound};
            process_list<TL, IX>(a, rd, a.F[fi], a.FR[fi], nF, gwarp, nwarps, sk, tl);
            process_list<TL, IX>(a, rd, a.H[fi], a.HR[fi], nH, gwarp, nwarps, sk, tl);
            if (!grid_sync(ctl, &epoch, a.spin_ns, &s_ok)) return;
            const unsigned long long eF = ld_vol(&ctl->cntF[pn]), eH = ld_vol(&ctl->cntH[pn]);
            n_alive -= nF + nH;
            nF = (int64_t)(eF - baseF[pn]);
            nH = (int64_t)(eH - baseH[pn]);
            baseF[pn] = eF;
            baseH[pn] = eH;
            fi ^= 1;
            ++r;
            // compact the rows once half of their entries are removed edges
            if (IX && !a.no_compact && 4 * n_alive < nnz) {
                ++compactions;
                const Round now{r};
                for (int64_t row = gwarp; row < a.n; row += nwarps) {
                    const int64_t b = a.rowptr[row];
                    const int32_t len = ld_cg(a.rowlen + row);
                    int32_t wpos = 0;
                    for (int32_t c = 0; c < len; c += 32) {
                        const int32_t i = c + lane;
                        bool keep = false;
                        int32_t cv = 0, ev = 0;
                        if (i < len) {
                            ev = ld_cg(a.eid + b + i);
                            cv = ld_cg(a.col + b + i);
                            keep = !now.removed(ld_cg(a.t + ev));
                        }
                        const unsigned msk = __ballot_sync(0xffffffffu, keep);
                        if (keep) {
                            const int32_t q = wpos + __popc(msk & lanemask_lt());
                            a.col[b + q] = cv;
                            a.eid[b + q] = ev;
                        }
                        wpos += __popc(msk);
                    }
                    if (lane == 0) a.rowlen[row] = wpos;
                }
                if (!grid_sync(ctl, &epoch, a.spin_ns, &s_ok)) return;
                nnz = 2 * n_alive;
            }
        }
        // every append to this level's window list happened before the last
        // barrier; the next level appends to the other counter
        {
            const unsigned long long eW = ld_vol(&ctl->cntW[wp]);
            nW = (int64_t)(eW - baseW[wp]);
            baseW[wp] = eW;
            wi ^= 1;
        }
        // round r's frontier was empty; the next scan takes a fresh round number
        ++r;
        if (a.single) break;
        if (leader && a.level_left)  // levels up to k_next - 1 remove nothing more
            for (int32_t kk = k; kk < k_next && kk <= a.k_last; ++kk)
                a.level_left[kk - a.k_first] = n_alive;
        if (n_alive == 0) break;
        if (a.k_last > 0 && k_next > a.k_last) break;
        kmax = k_next - 1;
        k = k_next;
    }
    atomicAdd(&ctl->scanned, tl.scanned);
    atomicAdd(&ctl->entries, tl.entries);
    atomicAdd(&ctl->searches, tl.searches);
    atomicAdd(&ctl->lookups, tl.lookups);
    atomicAdd(&ctl->lowered, tl.lowered);
    if (leader) {
        ctl->kmax = kmax;
        ctl->n_alive = n_alive;
        ctl->rounds = rounds;
        ctl->compactions = compactions;
        ctl->full_scans = fulls;
    }
}

__global__ void k_peel_init(const int64_t* __restrict__ rowptr, int32_t n,
                            int32_t* __restrict__ rowlen) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride)
        rowlen[r] = (int32_t)(rowptr[r + 1] - rowptr[r]);
}

// Final states -> canonical-order outputs: the k-truss mask (alive = 0) or
// truss numbers (an edge removed in a round of level k has truss number k - 1).
__global__ void k_mask_from_state(const int32_t* __restrict__ t,
                                  const int32_t* __restrict__ inv, int64_t m,
                                  uint8_t* __restrict__ mask) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < m; c += stride)
        mask[c] = t[inv[c]] == 0 ? 1 : 0;
}

// The same mask in two passes: one bit per internal edge (coalesced over the
// states; the bitmap, 1/32 of them, stays in L2), then a gather of bits in
// canonical order, four edges per thread in flight (a gather of the states
// themselves reads a 32-byte sector per edge).
__global__ void k_alive_bits(const int32_t* __restrict__ t, int64_t m,
                             unsigned int* __restrict__ bits) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < m;
         base += nw * 32) {
        const int64_t j = base + lane;
        const unsigned b = __ballot_sync(0xffffffffu, j < m && t[j] == 0);
        if (lane == 0) bits[base >> 5] = b;
    }
}

__global__ void k_mask_from_bits(const unsigned int* __restrict__ bits,
                                 const int32_t* __restrict__ inv, int64_t m,
                                 uint8_t* __restrict__ mask) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c0 < m; c0 += 4 * stride) {
        int32_t j[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) j[u] = c0 + u * stride < m ? inv[c0 + u * stride] : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (j[u] >= 0) mask[c0 + u * stride] = (bits[j[u] >> 5] >> (j[u] & 31)) & 1u;
    }
}

__global__ void k_resume_states(int32_t* __restrict__ t, int64_t m) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride)
        if (t[j] != 0) t[j] = -1;
}

__global__ void k_truss_from_state(const int32_t* __restrict__ t,
                                   const int32_t* __restrict__ inv, int64_t m,
                                   const int32_t* __restrict__ level_of,
                                   int32_t* __restrict__ truss) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < m; c += stride) {
        const int32_t st = t[inv[c]];
        truss[c] = st < 0 ? level_of[-st] - 1 : 0;
    }
}

int ensure_support_impl(Graph* g, cudaStream_t s) {
    // the peel needs the supports and T (it sizes the triangle lists by T)
    if (g->support_valid && g->triangles >= 0) return TC_OK;
    if (!g->support) TC_TRY(dev_alloc_n(&g->support, g->m, s));
    int64_t T = 0;
    TC_TRY(compute_support(g, g->support, true, &T, s));
    g->triangles = T;
    g->support_valid = true;
    return TC_OK;
}

inline unsigned small_grid(int64_t items) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * 8,
                                                            (items + 255) / 256));
}

}  // namespace

// A peel split into host planning (decisions and every allocation), stream
// work (capturable in a CUDA graph: no host synchronisation) and completion
// (reads the control block back).  The triangle-list form is used when the
// lists (3T pairs of edge ids) fit comfortably in free device memory, unless
// the caller or a test hook forces a form.
struct PeelPlan {
    Graph* g = nullptr;
    PeelArgs a{};
    bool tl = false;           // triangle lists (all edges, or with ix those below bound)
    bool ix = true;            // live neighbour lists kept for intersections
    int32_t bound = 0;         // lists only for edges whose support is below it (0: all)
    bool single = false;
    const void* fn = nullptr;
    int blocks = 0;
    unsigned long long* off = nullptr;
    int2* pairs = nullptr;
    ListsPlan lists;
    bool resume = false;       // start from the graph's cached k-truss
    bool cache = false;        // state/support (and adjacency) are the graph's cache
    bool fresh_adj = true;     // the working adjacency must be copied from the graph
    bool readonly_adj = false; // ... or the graph's own is read in place (one level)
    uint8_t* out_mask = nullptr;    // single level: canonical k-truss mask
    int32_t* out_truss = nullptr;   // decomposition: canonical truss numbers
    bool build_lists = false;  // the lists are built by this peel (else cached)
    bool keep_lists = false;   // ... and stay with the graph afterwards
    KernelTimer timer;
    PeelCtl result{};
};

PeelPlan* peel_plan_new() { return new (std::nothrow) PeelPlan(); }

namespace {
// Optional memory the graph keeps now: triangle lists, the compacted
// adjacency of the latest k-truss, truss numbers.
double lists_bytes(const Graph* g, int64_t entries) {
    return 8.0 * (double)std::max<int64_t>(entries, 0) + 8.0 * (double)(g->m + 1);
}
double lists_bytes(const Graph* g) { return lists_bytes(g, g->tri_entries); }
double adj_bytes(const Graph* g) { return 16.0 * (double)g->m + 4.0 * (double)g->n; }
double kept_optional_bytes(const Graph* g) {
    return (g->tri_off ? lists_bytes(g) : 0.0) + (g->kt_col ? adj_bytes(g) : 0.0) +
           (g->truss_cache ? 4.0 * (double)g->m : 0.0);
}
// Whether a structure of `bytes` (counted in `kept_optional_bytes` when
// `held`) may be kept: with a bound, everything kept stays within it; without
// one, the structure fits a share of the free device memory.
bool may_keep(const Graph* g, double bytes, bool held, double free_share) {
    if (g->mem_limit >= 0)
        return kept_optional_bytes(g) - (held ? bytes : 0.0) + bytes <= (double)g->mem_limit;
    return held || bytes <= free_share;
}
}  // namespace
void peel_plan_delete(PeelPlan* p) { delete p; }

int peel_plan(PeelPlan* pp, Scratch& sc, Graph* g, int32_t k_first, bool single, int32_t* t,
              int form, bool keep_lists, bool use_cache, int max_blocks) {
    PeelPlan& p = *pp;
    const int64_t m = g->m;
    if (!g->support_valid) return fail(TC_EINVAL, "internal: peel planned without supports");
    p.g = g;
    p.single = single;
    p.readonly_adj = false;
    p.fresh_adj = true;
    PeelArgs& a = p.a;
    a = PeelArgs{};
    a.m = m;
    a.n = g->n;
    a.ends = g->ends;
    a.rowptr = g->rowptr;
    a.t = t;
    a.k_first = k_first;
    a.r_first = 1;
    a.single = single ? 1 : 0;
    a.spin_ns = spin_limit_ns();
    p.cache = single && use_cache;
    p.resume = p.cache && g->kt_k > 0 && k_first >= g->kt_k;
    if (p.cache) {
        if (!g->kt_state) TC_TRY(dev_alloc_n(&g->kt_state, m, g->last_stream));
        if (!g->kt_support) TC_TRY(dev_alloc_n(&g->kt_support, m, g->last_stream));
        a.t = g->kt_state;
        if (!p.resume) g->kt_k = 0;  // rebuilt below; valid again only if this peel completes
    }
    const int forced = form != PEEL_AUTO ? form : peel_mode();
    p.tl = false;
    p.ix = true;
    p.bound = 0;
    size_t free_b = 0, total_b = 0;
    TC_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    // optional memory (lists, caches) stays within the graph's bound, all of
    // it together, or a share of the free memory when the caller set none.
    // List positions are 32-bit: full lists need 3T < 2^32, partial lists
    // (edges whose support is below LIST_BOUND) fewer than 2^32 entries.
    int64_t entries = 0;
    if (triangle_lists_supported(g) && forced != PEEL_INTERSECT) {
        const int64_t full = 3 * std::max<int64_t>(g->triangles, 0);
        const bool held_full = g->tri_off && g->tri_bound == 0;
        if (full < 0xffffffffLL && forced != PEEL_HYBRID &&
            (forced == PEEL_LISTS ||
             may_keep(g, lists_bytes(g, full), held_full, 0.6 * (double)free_b))) {
            p.tl = true;
            p.ix = false;
            entries = full;
        } else if (forced != PEEL_LISTS || full >= 0xffffffffLL) {
            if (g->tri_valid && g->tri_bound == LIST_BOUND)
                entries = g->tri_entries;  // the graph keeps these lists: nothing to count
            else
                TC_TRY(partial_list_entries(g, LIST_BOUND, &entries, &p.lists.low_edges,
                                            g->last_stream));
            const bool held = g->tri_off && g->tri_bound == LIST_BOUND;
            if (entries < 0xffffffffLL &&
                (forced == PEEL_HYBRID ||
                 may_keep(g, lists_bytes(g, entries), held, 0.6 * (double)free_b))) {
                p.tl = true;
                p.bound = LIST_BOUND;
            }
        }
    }
    if (g->tri_off && (!p.tl || g->tri_bound != p.bound)) {
        // cached lists above a lowered limit, or of the other kind, are dropped
        dev_free(g->tri_off, g->last_stream);
        dev_free(g->tri_pairs, g->last_stream);
        g->tri_off = nullptr;
        g->tri_pairs = nullptr;
        g->tri_valid = false;
        g->tri_entries = 0;
    }
    if (p.tl && g->tri_valid) {
        p.off = g->tri_off;  // built by an earlier peel of this graph
        p.pairs = g->tri_pairs;
        p.build_lists = false;
        a.off = p.off;
        a.pairs = p.pairs;
    } else if (p.tl) {
        p.build_lists = true;
        p.keep_lists = keep_lists;
        if (keep_lists) {
            if (!g->tri_off) TC_TRY(dev_alloc_n(&g->tri_off, m + 1, g->last_stream));
            if (!g->tri_pairs) {
                TC_TRY(dev_alloc_n(&g->tri_pairs, std::max<int64_t>(1, entries), g->last_stream));
                g->tri_entries = entries;
                g->tri_bound = p.bound;
            }
            p.off = g->tri_off;
            p.pairs = g->tri_pairs;
        } else {
            TC_TRY(sc.alloc(&p.off, m + 1));
            TC_TRY(sc.alloc(&p.pairs, std::max<int64_t>(1, entries)));
        }
        p.lists.bound = p.bound;
        p.lists.entries = entries;
        TC_TRY(plan_triangle_lists(g, sc, &p.lists));
        a.off = p.off;
        a.pairs = p.pairs;
    }
    if (!p.ix) {
        // list form only: no adjacency
    } else if (p.cache) {
        // the compacted adjacency stays with the graph when it fits
        p.fresh_adj = !(p.resume && g->kt_adj);
        const bool adj_ok = may_keep(g, adj_bytes(g), g->kt_col != nullptr, 0.4 * (double)free_b);
        if (g->kt_col && !adj_ok) {
            dev_free(g->kt_col, g->last_stream);  // above a lowered limit
            dev_free(g->kt_eid, g->last_stream);
            dev_free(g->kt_rowlen, g->last_stream);
            g->kt_col = g->kt_eid = nullptr;
            g->kt_rowlen = nullptr;
            g->kt_adj = false;
            p.fresh_adj = true;
        }
        if (adj_ok) {
            if (!g->kt_col) {
                TC_TRY(dev_alloc_n(&g->kt_col, 2 * m, g->last_stream));
                TC_TRY(dev_alloc_n(&g->kt_eid, 2 * m, g->last_stream));
                TC_TRY(dev_alloc_n(&g->kt_rowlen, g->n, g->last_stream));
            }
            a.col = g->kt_col;
            a.eid = g->kt_eid;
            a.rowlen = g->kt_rowlen;
        } else {
            p.readonly_adj = true;
        }
        g->kt_adj = false;  // valid again only if this peel completes in the graph's buffers
    } else if (single) {
        p.readonly_adj = true;
    } else {
        TC_TRY(sc.alloc(&a.rowlen, g->n));
        TC_TRY(sc.alloc(&a.col, 2 * m));
        TC_TRY(sc.alloc(&a.eid, 2 * m));
    }
    if (p.readonly_adj) {
        // one level: the intersections read the graph's own adjacency, with
        // dead entries left in place (no compaction), instead of a copy
        p.fresh_adj = false;
        a.no_compact = 1;
        a.col = g->col;
        a.eid = g->eid;
        TC_TRY(sc.alloc(&a.rowlen, g->n));
    }
    if (p.cache) a.s = g->kt_support;
    else TC_TRY(sc.alloc(&a.s, m));
    // a heavy edge has more than HEAVY of the list entries (the
    // intersection form has none)
    const int64_t heavy_cap = p.tl ? std::min<int64_t>(m, entries / HEAVY + 1) : 1;
    for (int i = 0; i < 2; ++i) {
        // one level: no alive list or window is written; A[0] only holds
        // the mask's bitmap afterwards (one bit per edge)
        if (!single) {
            TC_TRY(sc.alloc(&a.A[i], m));
            TC_TRY(sc.alloc(&a.W[i], m));
        } else if (i == 0) {
            TC_TRY(sc.alloc(&a.A[0], m / 32 + 1));
        }
        TC_TRY(sc.alloc(&a.F[i], m));
        TC_TRY(sc.alloc(&a.H[i], heavy_cap));
        if (p.tl) {
            TC_TRY(sc.alloc(&a.FR[i], m));
            TC_TRY(sc.alloc(&a.HR[i], heavy_cap));
        }
    }
    TC_TRY(sc.alloc(&a.ctl, 1));
    // round numbers live in int32 edge states: at most 2^31 - 16 rounds.  A
    // non-empty round removes at least one edge (at most m of them) and a
    // level takes one more number for its scan; levels end at k <= the
    // largest support + 3 <= max degree + 2, so there are at most max degree
    // + 1 of them.  The kernel stops with an overflow status if the table
    // ever runs out.
    a.max_round = std::min<int64_t>(m + 2 * (int64_t)g->max_deg + 64, 0x7fffffffLL - 16);
    TC_TRY(sc.alloc(&a.level_of, a.max_round));
    p.fn = !p.tl ? (const void*)k_peel<false, true>
           : p.ix ? (const void*)k_peel<true, true> : (const void*)k_peel<true, false>;
    int per_sm = 0;
    TC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p.fn, PK_THREADS, 0));
    if (per_sm < 1) return fail(TC_ECUDA, "k_peel cannot be resident");
    // one block per ~24K edges up to one per SM: the peel is latency-bound,
    // so below about 4M edges a partial grid is as fast (cheaper barriers)
    // and leaves SMs to other streams' work (concurrent requests)
    const int64_t want = std::min<int64_t>(std::max<int64_t>(1, (m + 24575) / 24576),
                                           TC_PK_MAX_BLOCKS);
    p.blocks = (int)std::min<int64_t>(want, (int64_t)num_sms() * std::min(per_sm, 1024 / PK_THREADS));
    if (max_blocks > 0) p.blocks = std::min(p.blocks, max_blocks);
    g->last_peel_lists = p.tl ? (p.ix ? 2 : 1) : 0;
    return TC_OK;
}

int peel_enqueue(PeelPlan* pp, cudaStream_t s) {
    PeelPlan& p = *pp;
    Graph* g = p.g;
    PeelArgs& a = p.a;
    const int64_t m = g->m;
    if (p.tl && p.build_lists)
        TC_TRY(enqueue_triangle_lists(g, g->support, p.off, p.pairs, &p.lists, s));
    if (p.ix && p.readonly_adj) {
        k_peel_init<<<small_grid(g->n), 256, 0, s>>>(g->rowptr, g->n, a.rowlen);
        TC_LAUNCH_CHECK("k_peel_init");
    } else if (p.ix && p.fresh_adj) {
        TC_CUDA_TRY(cudaMemcpyAsync(a.col, g->col, sizeof(int32_t) * 2 * m,
                                    cudaMemcpyDeviceToDevice, s));
        TC_CUDA_TRY(cudaMemcpyAsync(a.eid, g->eid, sizeof(int32_t) * 2 * m,
                                    cudaMemcpyDeviceToDevice, s));
        k_peel_init<<<small_grid(g->n), 256, 0, s>>>(g->rowptr, g->n, a.rowlen);
        TC_LAUNCH_CHECK("k_peel_init");
    }
    if (p.resume) {
        // edges outside the cached truss count as removed before round 2;
        // the cached supports are already those within the truss
        k_resume_states<<<small_grid(m), 256, 0, s>>>(a.t, m);
        TC_LAUNCH_CHECK("k_resume_states");
        a.r_first = 2;
    } else {
        TC_CUDA_TRY(cudaMemcpyAsync(a.s, g->support, sizeof(int32_t) * m,
                                    cudaMemcpyDeviceToDevice, s));
        TC_CUDA_TRY(cudaMemsetAsync(a.t, 0, sizeof(int32_t) * m, s));
    }
    TC_CUDA_TRY(cudaMemsetAsync(a.ctl, 0, sizeof(PeelCtl), s));
    void* params[] = {&a};
    TC_TRY(p.timer.start(s));
    // one block is always resident: its grid barrier needs no cooperative
    // launch, and a plain launch can run beside other streams' cooperative ones
    if (p.blocks == 1)
        TC_CUDA_TRY(cudaLaunchKernel(p.fn, dim3(1), dim3(PK_THREADS), params, 0, s));
    else
        TC_CUDA_TRY(cudaLaunchCooperativeKernel(p.fn, dim3(p.blocks), dim3(PK_THREADS), params, 0,
                                                s));
    count_launch();
    TC_TRY(p.timer.stop(s));
    if (!p.single && p.out_truss) {
        k_truss_from_state<<<small_grid(m), 256, 0, s>>>(a.t, g->inv, m, a.level_of, p.out_truss);
        TC_LAUNCH_CHECK("k_truss_from_state");
    }
    if (p.single && p.out_mask) {
        // the peel's alive lists are free now: the first holds the bitmap
        unsigned int* bits = reinterpret_cast<unsigned int*>(a.A[0]);
        k_alive_bits<<<small_grid(m), 256, 0, s>>>(a.t, m, bits);
        TC_LAUNCH_CHECK("k_alive_bits");
        k_mask_from_bits<<<small_grid(m), 256, 0, s>>>(bits, g->inv, m, p.out_mask);
        TC_LAUNCH_CHECK("k_mask_from_bits");
    }
    return TC_OK;
}

int peel_finish(PeelPlan* pp, cudaStream_t s, int64_t* n_alive, int32_t* kmax) {
    PeelPlan& p = *pp;
    Graph* g = p.g;
    PeelCtl& r = p.result;
    TC_CUDA_TRY(cudaMemcpyAsync(&r, p.a.ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, s));
    const bool col_lists = p.tl && p.build_lists && p.lists.form == 1;
    unsigned long long words = 0;
    if (col_lists)
        TC_CUDA_TRY(cudaMemcpyAsync(&words, g->dev_scalars + 7, sizeof(words),
                                    cudaMemcpyDeviceToHost, s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    // column-kernel list build: the out-list words it read, per in-neighbour
    // entry its id, edge id and the in-neighbour's row end and edge shift
    // (24 B), per column its bounds and shift (24 B), per list entry the
    // 8-byte pair and its 4-byte cursor read and written (16 B)
    g->stats.lists_bytes = col_lists ? 4 * (int64_t)words + 24 * g->m + 24 * (int64_t)g->n +
                                           16 * p.lists.entries
                                     : -1;
    g->last_peel_rounds = r.rounds;
    g->stats.peel_ns = p.timer.elapsed_ns();
    g->stats.lists_ns = p.tl && p.build_lists ? p.lists.timer.elapsed_ns() : -1;
    // algorithmic bytes: a scanned entry reads its id, state and support
    // (12 B); a triangle-list entry is an 8-B pair, a neighbour-list entry
    // an id and an edge id (8 B); binary-search steps and state lookups read
    // 4 B each; a decrement is a 4-B read-modify-write (8 B)
    g->stats.peel_scanned = (int64_t)r.scanned;
    g->stats.peel_entries = (int64_t)r.entries;
    g->stats.peel_searches = (int64_t)r.searches;
    g->stats.peel_lookups = (int64_t)r.lookups;
    g->stats.peel_lowered = (int64_t)r.lowered;
    g->stats.peel_bytes = 12 * (int64_t)r.scanned + 8 * (int64_t)r.entries +
                          4 * (int64_t)r.searches + 4 * (int64_t)r.lookups +
                          8 * (int64_t)r.lowered;
    if (r.abort) return fail(TC_ETIMEDOUT, "peel: a grid barrier wait ran out of time");
    if (r.overflow) return fail(TC_EOVERFLOW, "peel: round table exhausted");
    if (p.build_lists && p.keep_lists) g->tri_valid = true;
    if (p.cache) {
        g->kt_k = p.a.k_first;
        g->kt_adj = p.ix && p.a.col == g->kt_col && g->kt_col != nullptr;
    }
    if (n_alive) *n_alive = r.n_alive;
    if (kmax) *kmax = r.kmax;
    return TC_OK;
}

bool peel_uses_lists(const PeelPlan* p) { return p->tl && !p->ix; }
int peel_form_of(const PeelPlan* p) { return p->tl ? (p->ix ? PEEL_HYBRID : PEEL_LISTS) : PEEL_INTERSECT; }

namespace {

// Plan, run and complete one peel on the graph's stream; results go to the
// canonical-order output (mask for one level, truss numbers otherwise).
int run_peel(Graph* g, int32_t k_first, bool single, uint8_t* out_mask, int32_t* out_truss,
             PeelCtl* result, cudaStream_t s, int32_t k_last = 0,
             long long* level_left = nullptr) {
    TC_TRY(ensure_support_impl(g, s));
    Scratch sc(s);
    int32_t* t;
    TC_TRY(sc.alloc(&t, g->m));
    PeelPlan p;
    TC_TRY(peel_plan(&p, sc, g, k_first, single, t, PEEL_AUTO, /*keep_lists=*/true,
                     /*use_cache=*/single && g->keep_results, g->peel_max_blocks));
    p.out_mask = out_mask;
    p.out_truss = out_truss;
    p.a.k_last = k_last;
    p.a.level_left = level_left;
    TC_TRY(peel_enqueue(&p, s));
    TC_TRY(peel_finish(&p, s, nullptr, nullptr));
    *result = p.result;
    return TC_OK;
}

}  // namespace

int ensure_support(Graph* g, cudaStream_t s) { return ensure_support_impl(g, s); }

int mask_from_state(const int32_t* t, const int32_t* inv, int64_t m, uint8_t* mask,
                    cudaStream_t s) {
    k_mask_from_state<<<small_grid(m), 256, 0, s>>>(t, inv, m, mask);
    TC_LAUNCH_CHECK("k_mask_from_state");
    return TC_OK;
}

namespace {
// The k-truss from truss numbers: e is in it iff truss[e] >= k (the
// k-trusses nest, Section III-B); counts the edges in it.
__global__ void k_mask_from_truss(const int32_t* __restrict__ truss, int64_t m, int32_t k,
                                  uint8_t* __restrict__ mask,
                                  unsigned long long* __restrict__ count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const bool in = truss[e] >= k;
        mask[e] = in ? 1 : 0;
        c += in;
    }
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// A test hook forcing a peel form always peels.
bool truss_cache_usable(const Graph* g) {
    return g->keep_results && g->truss_valid && peel_mode() == PEEL_AUTO &&
           intersect_mode() == 0;
}
}  // namespace

int peel_ktruss(Graph* g, int32_t k, uint8_t* mask, int64_t* edges_left, cudaStream_t s) {
    const int64_t m = g->m;
    if (m == 0) {
        if (edges_left) *edges_left = 0;
        return TC_OK;
    }
    if (truss_cache_usable(g)) {
        unsigned long long* cnt = g->dev_scalars + 1;
        TC_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
        k_mask_from_truss<<<small_grid(m), 256, 0, s>>>(g->truss_cache, m, k, mask, cnt);
        TC_LAUNCH_CHECK("k_mask_from_truss");
        unsigned long long h = 0;
        TC_CUDA_TRY(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
        if (edges_left) *edges_left = (int64_t)h;
        return TC_OK;
    }
    PeelCtl r{};
    TC_TRY(run_peel(g, k, true, mask, nullptr, &r, s));
    if (edges_left) *edges_left = r.n_alive;
    return TC_OK;
}

namespace {
// Counts, per k in [k_lo, k_hi], the edges with truss number >= k.
__global__ void k_truss_counts(const int32_t* __restrict__ truss, int64_t m, int32_t k_lo,
                               int32_t k_hi, unsigned long long* __restrict__ counts) {
    __shared__ unsigned long long sh[64];
    const int nk = k_hi - k_lo + 1;
    for (int i = threadIdx.x; i < nk; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t t = truss[e];
        if (t >= k_lo) atomicAdd(&sh[min(t, k_hi) - k_lo], 1ull);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nk; i += blockDim.x)
        if (sh[i]) atomicAdd(&counts[i], sh[i]);
}
}  // namespace

int peel_sizes(Graph* g, int32_t k_lo, int32_t k_hi, int64_t* sizes, cudaStream_t s) {
    const int64_t m = g->m;
    const int nk = k_hi - k_lo + 1;
    int32_t k = k_lo;
    for (; k <= 2 && k <= k_hi; ++k) sizes[k - k_lo] = m;  // the 2-truss is every edge
    if (k > k_hi) return TC_OK;
    if (m == 0) {
        for (; k <= k_hi; ++k) sizes[k - k_lo] = 0;
        return TC_OK;
    }
    Scratch sc(s);
    if (truss_cache_usable(g)) {
        // the kept decomposition: count truss numbers >= k (suffix sums of a histogram)
        unsigned long long* cnt;
        TC_TRY(sc.alloc(&cnt, nk));
        TC_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * nk, s));
        k_truss_counts<<<small_grid(m), 256, 0, s>>>(g->truss_cache, m, k, k_hi, cnt + (k - k_lo));
        TC_LAUNCH_CHECK("k_truss_counts");
        unsigned long long h[64] = {};
        TC_CUDA_TRY(cudaMemcpyAsync(h, cnt, sizeof(unsigned long long) * nk,
                                    cudaMemcpyDeviceToHost, s));
        TC_CUDA_TRY(cudaStreamSynchronize(s));
        unsigned long long run = 0;
        for (int32_t kk = k_hi; kk >= k; --kk) {
            run += h[kk - k_lo];
            sizes[kk - k_lo] = (int64_t)run;
        }
        return TC_OK;
    }
    long long* left;
    TC_TRY(sc.alloc(&left, nk));
    TC_CUDA_TRY(cudaMemsetAsync(left, 0, sizeof(long long) * nk, s));  // emptied levels stay 0
    PeelCtl r{};
    TC_TRY(run_peel(g, k, false, nullptr, nullptr, &r, s, k_hi, left + (k - k_lo)));
    long long h[64] = {};
    TC_CUDA_TRY(cudaMemcpyAsync(h, left, sizeof(long long) * nk, cudaMemcpyDeviceToHost, s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    for (int32_t kk = k; kk <= k_hi; ++kk) sizes[kk - k_lo] = h[kk - k_lo];
    return TC_OK;
}

int peel_decompose(Graph* g, int32_t* truss, int32_t* kmax, cudaStream_t s) {
    const int64_t m = g->m;
    if (m == 0) {
        *kmax = 0;
        return TC_OK;
    }
    if (truss_cache_usable(g)) {
        TC_CUDA_TRY(cudaMemcpyAsync(truss, g->truss_cache, sizeof(int32_t) * m,
                                    cudaMemcpyDeviceToDevice, s));
        *kmax = g->truss_kmax;
        return TC_OK;
    }
    PeelCtl r{};
    TC_TRY(run_peel(g, 3, false, nullptr, truss, &r, s));
    *kmax = r.kmax;
    // keep the decomposition when it fits the graph's optional memory
    size_t free_b = 0, total_b = 0;
    TC_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    bool room = g->keep_results &&
                may_keep(g, 4.0 * (double)m, g->truss_cache != nullptr, 0.4 * (double)free_b);
    if (!room && g->truss_cache) {
        dev_free(g->truss_cache, s);
        g->truss_cache = nullptr;
        g->truss_valid = false;
    }
    if (room && !g->truss_cache) TC_TRY(dev_alloc_n(&g->truss_cache, m, s));
    if (room) {
        TC_CUDA_TRY(cudaMemcpyAsync(g->truss_cache, truss, sizeof(int32_t) * m,
                                    cudaMemcpyDeviceToDevice, s));
        g->truss_kmax = r.kmax;
        g->truss_valid = true;
    }
    return TC_OK;
}

}  // namespace tc
