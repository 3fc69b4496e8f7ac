/*
 * graphgen.c — seeded synthetic edge-list generators.
 *
 * These produce the raw inputs that both the CPU oracle (tests) and the GPU
 * library consume.  They hold none of the method's arithmetic: no cleaning,
 * no sorting, no triangle or truss logic.  Outputs may contain self-loops and
 * duplicate pairs; removing them is the job of the code under test.
 *
 * Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used in counter mode: draw i
 * of stream p is  mix64(key_p + (i + 1) * GAMMA)  with GAMMA the golden-ratio
 * increment and key_p = mix64(seed ^ (p * STREAM_SALT)).  Counter mode makes
 * every draw addressable, so the R-MAT generator parallelises with OpenMP and
 * still emits the same list on every machine and thread count.
 *
 * Generators (Graph500-style R-MAT with a seeded vertex relabelling, and
 * Erdős–Rényi G(n, m)) follow the synthetic data families the Graph
 * Challenge names for its inputs (Section II).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 0x9e3779b97f4a7c15ULL
#define STREAM_SALT 0xd1b54a32d192ed03ULL

enum { STREAM_RMAT = 1, STREAM_PERM = 2, STREAM_ER = 3, STREAM_REJECT = 4 };

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return mix64(seed ^ (stream * STREAM_SALT));
}

static inline uint64_t draw(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GAMMA); }

/* Uniform integer in [0, bound) by the multiply-shift map of a 64-bit draw
 * (Lemire 2019, without the rejection step; bias < bound / 2^64). */
static inline uint64_t bounded(uint64_t r, uint64_t bound) {
    return (uint64_t)(((unsigned __int128)r * bound) >> 64);
}

/* Seeded Fisher–Yates shuffle of the identity on [0, n). */
void gg_permutation(int32_t n, uint64_t seed, int32_t* perm) {
    uint64_t key = stream_key(seed, STREAM_PERM);
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {
        uint64_t j = bounded(draw(key, (uint64_t)(n - 1 - i)), (uint64_t)i + 1);
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
}

/* Quadrant thresholds at 32-bit resolution: a draw's 32-bit half h picks
 * quadrant (0,0) if h < ta, (0,1) if h < tb, (1,0) if h < tc, else (1,1). */
typedef struct { uint64_t ta, tb, tc; } rmat_thr;

static rmat_thr make_thr(double a, double b, double c) {
    rmat_thr t;
    const double s = 4294967296.0;
    t.ta = (uint64_t)(a * s);
    t.tb = (uint64_t)((a + b) * s);
    t.tc = (uint64_t)((a + b + c) * s);
    return t;
}

/* One R-MAT endpoint pair at `scale` levels from draw counter base `ctr`
 * (two levels per 64-bit draw). */
static inline void rmat_pair(uint64_t key, uint64_t ctr, int scale, rmat_thr t,
                             uint32_t* pu, uint32_t* pv) {
    uint32_t u = 0, v = 0;
    uint64_t r = 0;
    for (int l = 0; l < scale; ++l) {
        if ((l & 1) == 0) r = draw(key, ctr + (uint64_t)(l >> 1));
        uint64_t h = (l & 1) ? (r >> 32) : (r & 0xffffffffULL);
        uint32_t bu = 0, bv = 0;
        if (h < t.ta) {
        } else if (h < t.tb) {
            bv = 1;
        } else if (h < t.tc) {
            bu = 1;
        } else {
            bu = 1;
            bv = 1;
        }
        u = (u << 1) | bu;
        v = (v << 1) | bv;
    }
    *pu = u;
    *pv = v;
}

/* R-MAT on n = 2^scale vertices: m draws, each an independent recursive
 * quadrant descent with probabilities (a, b, c, 1-a-b-c).  If `permute`, the
 * vertex ids are relabelled by a seeded random permutation. */
int gg_rmat(int scale, int64_t m, double a, double b, double c, uint64_t seed, int permute,
            int32_t* src, int32_t* dst) {
    if (scale < 1 || scale > 30 || m < 0) return -1;
    const int32_t n = (int32_t)1 << scale;
    const rmat_thr t = make_thr(a, b, c);
    const uint64_t key = stream_key(seed, STREAM_RMAT);
    const uint64_t per = (uint64_t)((scale + 1) / 2);
    int32_t* perm = NULL;
    if (permute) {
        perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        if (!perm) return -2;
        gg_permutation(n, seed, perm);
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        uint32_t u, v;
        rmat_pair(key, (uint64_t)i * per, scale, t, &u, &v);
        src[i] = perm ? perm[u] : (int32_t)u;
        dst[i] = perm ? perm[v] : (int32_t)v;
    }
    free(perm);
    return 0;
}

/* R-MAT on an arbitrary n: run at scale = ceil(log2 n) and reject draws with
 * an endpoint >= n until m pairs are accepted (sequential; attempt j uses
 * the counters of draw j). */
int gg_rmat_n(int32_t n, int64_t m, double a, double b, double c, uint64_t seed, int permute,
              int32_t* src, int32_t* dst) {
    if (n < 1 || m < 0) return -1;
    int scale = 0;
    while (((int64_t)1 << scale) < (int64_t)n) ++scale;
    if (scale == 0) scale = 1;
    const rmat_thr t = make_thr(a, b, c);
    const uint64_t key = stream_key(seed, STREAM_RMAT);
    const uint64_t per = (uint64_t)((scale + 1) / 2);
    int32_t* perm = NULL;
    if (permute) {
        perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        if (!perm) return -2;
        gg_permutation(n, seed, perm);
    }
    int64_t got = 0;
    for (uint64_t j = 0; got < m; ++j) {
        uint32_t u, v;
        rmat_pair(key, j * per, scale, t, &u, &v);
        if ((int64_t)u >= n || (int64_t)v >= n) continue;
        src[got] = perm ? perm[u] : (int32_t)u;
        dst[got] = perm ? perm[v] : (int32_t)v;
        ++got;
    }
    free(perm);
    return 0;
}

/* Erdős–Rényi G(n, m): m distinct unordered pairs {u, v}, u != v, drawn
 * uniformly without replacement (rejection of loops and repeats).  Pairs are
 * emitted in draw order with the endpoints as drawn. */
int gg_er(int32_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst) {
    if (n < 2 || m < 0) return -1;
    if ((double)m > 0.5 * (double)n * (double)(n - 1)) return -1;
    /* open-addressing set of packed pairs, load factor <= 1/2 */
    uint64_t cap = 16;
    while (cap < (uint64_t)m * 2 + 16) cap <<= 1;
    uint64_t* set = (uint64_t*)malloc(sizeof(uint64_t) * cap);
    if (!set) return -2;
    memset(set, 0xff, sizeof(uint64_t) * cap);
    const uint64_t key = stream_key(seed, STREAM_ER);
    int64_t got = 0;
    for (uint64_t j = 0; got < m; ++j) {
        uint64_t r = draw(key, j);
        /* each 32-bit half, placed in the top bits, maps to [0, n) */
        uint32_t u = (uint32_t)bounded((r & 0xffffffffULL) << 32, (uint64_t)n);
        uint32_t v = (uint32_t)bounded(r & 0xffffffff00000000ULL, (uint64_t)n);
        if (u == v) continue;
        uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
        uint64_t pk = (lo << 32) | hi;
        uint64_t h = mix64(pk) & (cap - 1);
        int dup = 0;
        while (set[h] != ~0ULL) {
            if (set[h] == pk) {
                dup = 1;
                break;
            }
            h = (h + 1) & (cap - 1);
        }
        if (dup) continue;
        set[h] = pk;
        src[got] = (int32_t)u;
        dst[got] = (int32_t)v;
        ++got;
    }
    free(set);
    return 0;
}

/* A batch of independent graphs, generated in parallel (one graph per task):
 * kind[g] = 0: Erdős–Rényi G(n[g], m[g]); kind[g] = 1: R-MAT on n[g]
 * vertices with m[g] draws (rejection of endpoints >= n[g]), permuted.
 * Graph g's pairs go to src/dst[off[g] .. off[g] + m[g]); its stream seed is
 * derived from (seed, g). */
int gg_batch(int32_t G, const int32_t* kind, const int32_t* n, const int64_t* m,
             const int64_t* off, uint64_t seed, double a, double b, double c, int32_t* src,
             int32_t* dst) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : bad)
    for (int32_t g = 0; g < G; ++g) {
        const uint64_t sg = mix64(seed * 0x100000001b3ULL + (uint64_t)g + 1);
        int rc;
        if (kind[g] == 0) rc = gg_er(n[g], m[g], sg, src + off[g], dst + off[g]);
        else rc = gg_rmat_n(n[g], m[g], a, b, c, sg, 1, src + off[g], dst + off[g]);
        if (rc != 0) bad = 1;
    }
    return bad ? -1 : 0;
}

/* The M x M 8-neighbour image graph (Section IV-C): vertex r*M + c; each
 * undirected edge once, in four blocks by offset (0,+1), (+1,-1), (+1,0),
 * (+1,+1), row-major within a block; (M - 1)(4M - 2) pairs in all. */
int gg_king(int32_t M, int32_t* src, int32_t* dst) {
    if (M < 1 || (int64_t)M * M > 2147483647LL) return -1;
    const int64_t m1 = (int64_t)M - 1;
    const int64_t cnt[4] = {(int64_t)M * m1, m1 * m1, m1 * (int64_t)M, m1 * m1};
    const int dr[4] = {0, 1, 1, 1}, dc[4] = {1, -1, 0, 1};
    int64_t base = 0;
    for (int d = 0; d < 4; ++d) {
        const int c0 = dc[d] < 0 ? 1 : 0;                /* first column of a row */
        const int ncol = dc[d] == 0 ? M : M - 1;          /* columns per row */
        const int nrow = dr[d] == 0 ? M : M - 1;
#pragma omp parallel for schedule(static)
        for (int32_t r = 0; r < nrow; ++r) {
            int64_t i = base + (int64_t)r * ncol;
            for (int32_t k = 0; k < ncol; ++k, ++i) {
                const int32_t c = c0 + k;
                src[i] = r * M + c;
                dst[i] = (r + dr[d]) * M + (c + dc[d]);
            }
        }
        base += cnt[d];
    }
    return 0;
}
