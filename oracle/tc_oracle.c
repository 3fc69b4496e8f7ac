/*
 * tc_oracle.c — reference CPU statement of triangle counting, per-edge
 * triangle support and k-truss peeling (Static Graph Challenge, Section III).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the GPU library is
 * checked against.  Only the test suite, the smoke check and the bench's CPU
 * baseline load it; the library never does, and the two share no code.
 *
 * Input: the canonical edge list (lo[e] < hi[e], sorted by (lo, hi), no
 * repeats), i.e. the graph after the cleaning rules of Section II (self-loops
 * dropped, one undirected edge per pair, unit weights).  Edge e's index in
 * that list is its id for every per-edge output.
 *
 * Everything is written from the definitions, with no reordering beyond them:
 *   - a triangle is a set of three mutually adjacent vertices (Section III-A);
 *   - the support of edge (a, b) is the number of triangles that contain it,
 *     i.e. |N(a) ∩ N(b)|, which is the row sum of (R == 2) in Algorithm 4
 *     where R = E A;
 *   - the k-truss is the largest subgraph in which every edge lies in at
 *     least k - 2 triangles of that subgraph (Section III-B); it is obtained
 *     by removing edges whose support is below k - 2 and lowering the support
 *     of the edges that shared a triangle with them, until none is below
 *     (the loop of Algorithm 4).  This file removes one edge at a time; the
 *     k-truss is unique, so the order of removal does not change it;
 *   - the truss decomposition runs k = 3 on the graph, passes the surviving
 *     edges to k + 1, and stops when nothing survives (Section III-B).
 *
 * Set intersection N(a) ∩ N(b) is a merge of the two sorted lists (or binary
 * search of the shorter list's elements in the longer, for skewed pairs).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n;
    int64_t m;
    int32_t* lo;   /* canonical endpoints, copied */
    int32_t* hi;
    int64_t* off;  /* adjacency offsets, n + 1 */
    int32_t* nbr;  /* N(x), ascending, 2m entries */
    int32_t* eid;  /* canonical id of the edge {x, nbr} */
} oracle_graph;

void oracle_free(oracle_graph* g) {
    if (!g) return;
    free(g->lo);
    free(g->hi);
    free(g->off);
    free(g->nbr);
    free(g->eid);
    free(g);
}

typedef struct { int32_t v; int32_t e; } nbr_entry;

static int cmp_entry(const void* x, const void* y) {
    int32_t a = ((const nbr_entry*)x)->v, b = ((const nbr_entry*)y)->v;
    return (a > b) - (a < b);
}

/* Builds the full adjacency lists N(x), each sorted, each entry carrying the
 * canonical id of its edge.  Returns NULL (and *err) if the list is not a
 * canonical edge list on [0, n). */
oracle_graph* oracle_open(int32_t n, int64_t m, const int32_t* lo, const int32_t* hi, int* err) {
    *err = 0;
    if (n < 0 || m < 0) { *err = -1; return NULL; }
    for (int64_t e = 0; e < m; ++e) {
        if (lo[e] < 0 || hi[e] >= n || lo[e] >= hi[e]) { *err = -2; return NULL; }
        if (e > 0 && (lo[e] < lo[e - 1] || (lo[e] == lo[e - 1] && hi[e] <= hi[e - 1]))) {
            *err = -3;
            return NULL;
        }
    }
    oracle_graph* g = (oracle_graph*)calloc(1, sizeof(oracle_graph));
    g->n = n;
    g->m = m;
    g->lo = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    g->hi = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    g->off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    g->nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    g->eid = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    nbr_entry* tmp = (nbr_entry*)malloc(sizeof(nbr_entry) * (size_t)(2 * m + 1));
    int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!g->lo || !g->hi || !g->off || !g->nbr || !g->eid || !tmp || !fill) {
        free(tmp);
        free(fill);
        oracle_free(g);
        *err = -4;
        return NULL;
    }
    memcpy(g->lo, lo, sizeof(int32_t) * (size_t)m);
    memcpy(g->hi, hi, sizeof(int32_t) * (size_t)m);
    /* degree of each vertex, then prefix sums as list offsets */
    for (int64_t e = 0; e < m; ++e) {
        g->off[lo[e] + 1]++;
        g->off[hi[e] + 1]++;
    }
    for (int32_t x = 0; x < n; ++x) g->off[x + 1] += g->off[x];
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = lo[e], b = hi[e];
        tmp[g->off[a] + fill[a]++] = (nbr_entry){b, (int32_t)e};
        tmp[g->off[b] + fill[b]++] = (nbr_entry){a, (int32_t)e};
    }
    /* sort each list (skipped for a list that is already in order) */
    for (int32_t x = 0; x < n; ++x) {
        int sorted = 1;
        for (int64_t i = g->off[x] + 1; i < g->off[x + 1] && sorted; ++i)
            sorted = tmp[i - 1].v < tmp[i].v;
        if (!sorted)
            qsort(tmp + g->off[x], (size_t)(g->off[x + 1] - g->off[x]), sizeof(nbr_entry),
                  cmp_entry);
    }
    for (int64_t i = 0; i < 2 * m; ++i) {
        g->nbr[i] = tmp[i].v;
        g->eid[i] = tmp[i].e;
    }
    free(tmp);
    free(fill);
    return g;
}

int64_t oracle_num_edges(const oracle_graph* g) { return g->m; }

/* Position of w in N(x), or -1. */
static int64_t find(const oracle_graph* g, int32_t x, int32_t w) {
    int64_t lo = g->off[x], hi = g->off[x + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->nbr[mid] < w) lo = mid + 1;
        else hi = mid;
    }
    return (lo < g->off[x + 1] && g->nbr[lo] == w) ? lo : -1;
}

/* Common neighbours of a and b: for each w in N(a) ∩ N(b), writes the
 * positions of w in N(a) and in N(b).  Returns how many were found.
 * The two sorted lists are merged; when one is much shorter than the other
 * (|short| * log2|long| < |short| + |long|) each of its elements is looked
 * up in the longer list by binary search instead. */
static int64_t common(const oracle_graph* g, int32_t a, int32_t b, int64_t* pa, int64_t* pb) {
    int64_t da = g->off[a + 1] - g->off[a], db = g->off[b + 1] - g->off[b];
    int32_t s = a, l = b;
    int64_t ds = da, dl = db;
    if (da > db) { s = b; l = a; ds = db; dl = da; }
    int64_t lg = 1;
    while (((int64_t)1 << lg) < dl) ++lg;
    int64_t cnt = 0;
    if (ds * lg < ds + dl) {
        for (int64_t i = g->off[s]; i < g->off[s + 1]; ++i) {
            int64_t j = find(g, l, g->nbr[i]);
            if (j < 0) continue;
            if (s == a) { pa[cnt] = i; pb[cnt] = j; }
            else { pa[cnt] = j; pb[cnt] = i; }
            ++cnt;
        }
        return cnt;
    }
    int64_t i = g->off[a], j = g->off[b];
    const int64_t ie = g->off[a + 1], je = g->off[b + 1];
    while (i < ie && j < je) {
        if (g->nbr[i] < g->nbr[j]) ++i;
        else if (g->nbr[i] > g->nbr[j]) ++j;
        else {
            pa[cnt] = i++;
            pb[cnt] = j++;
            ++cnt;
        }
    }
    return cnt;
}

static int64_t max_degree(const oracle_graph* g) {
    int64_t d = 0;
    for (int32_t x = 0; x < g->n; ++x)
        if (g->off[x + 1] - g->off[x] > d) d = g->off[x + 1] - g->off[x];
    return d;
}

/* Number of triangles: every triangle {a < b < w} is counted once, at its
 * edge (a, b), as a common neighbour w of a and b with w > b. */
int64_t oracle_count(const oracle_graph* g) {
    const int64_t dmax = max_degree(g) + 1;
    int64_t total = 0;
#pragma omp parallel reduction(+ : total)
    {
        int64_t* pa = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
        int64_t* pb = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
#pragma omp for schedule(dynamic, 1024)
        for (int64_t e = 0; e < g->m; ++e) {
            int32_t a = g->lo[e], b = g->hi[e];
            int64_t c = common(g, a, b, pa, pb);
            for (int64_t i = 0; i < c; ++i)
                if (g->nbr[pa[i]] > b) ++total;
        }
        free(pa);
        free(pb);
    }
    return total;
}

/* Support of every edge: s[e] = |N(a) ∩ N(b)| for e = {a, b}. */
void oracle_support(const oracle_graph* g, int32_t* s) {
    const int64_t dmax = max_degree(g) + 1;
#pragma omp parallel
    {
        int64_t* pa = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
        int64_t* pb = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
#pragma omp for schedule(dynamic, 1024)
        for (int64_t e = 0; e < g->m; ++e) s[e] = (int32_t)common(g, g->lo[e], g->hi[e], pa, pb);
        free(pa);
        free(pb);
    }
}

/* Support of selected edges only (for sampled checks on large graphs). */
void oracle_support_of(const oracle_graph* g, const int64_t* edges, int64_t cnt, int32_t* s) {
    const int64_t dmax = max_degree(g) + 1;
    int64_t* pa = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
    int64_t* pb = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
    for (int64_t i = 0; i < cnt; ++i) {
        int64_t e = edges[i];
        s[i] = (e >= 0 && e < g->m) ? (int32_t)common(g, g->lo[e], g->hi[e], pa, pb) : -1;
    }
    free(pa);
    free(pb);
}

/* Support of edge e counted only over triangles whose three edges have
 * alive[] != 0 (used to check a truss on its own edges). */
void oracle_support_within(const oracle_graph* g, const uint8_t* alive, int32_t* s) {
    const int64_t dmax = max_degree(g) + 1;
#pragma omp parallel
    {
        int64_t* pa = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
        int64_t* pb = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
#pragma omp for schedule(dynamic, 1024)
        for (int64_t e = 0; e < g->m; ++e) {
            int32_t cnt = 0;
            if (alive[e]) {
                int64_t c = common(g, g->lo[e], g->hi[e], pa, pb);
                for (int64_t i = 0; i < c; ++i)
                    if (alive[g->eid[pa[i]]] && alive[g->eid[pb[i]]]) ++cnt;
            }
            s[e] = cnt;
        }
        free(pa);
        free(pb);
    }
}

/* For the listed edges only: the number of triangles through the edge whose
 * two other edges have alive[] != 0, whatever the edge's own flag.  For an
 * edge of a k-truss this is its support within the truss; for an edge
 * outside the (maximal) k-truss it must be below k - 2, or the truss plus
 * that edge would be a larger k-truss. */
void oracle_support_within_of(const oracle_graph* g, const uint8_t* alive, const int64_t* edges,
                              int64_t cnt, int32_t* s) {
    const int64_t dmax = max_degree(g) + 1;
    int64_t* pa = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
    int64_t* pb = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
    for (int64_t i = 0; i < cnt; ++i) {
        const int64_t e = edges[i];
        int32_t c = 0;
        if (e >= 0 && e < g->m) {
            const int64_t k = common(g, g->lo[e], g->hi[e], pa, pb);
            for (int64_t j = 0; j < k; ++j)
                if (alive[g->eid[pa[j]]] && alive[g->eid[pb[j]]]) ++c;
        }
        s[i] = c;
    }
    free(pa);
    free(pb);
}

/* One peeling level: starting from the edges with alive[e] != 0 and their
 * current supports s[], remove edges whose support is below k - 2 until
 * none is.  Removing e = {a, b} destroys each triangle {a, b, w} whose other
 * two edges are still present, and lowers their supports by one.  Edges
 * removed here get level[e] = k - 1 (if level is not NULL).  Returns the
 * number of edges left. */
static int64_t peel_level(const oracle_graph* g, int32_t k, uint8_t* alive, int32_t* s,
                          int32_t* level, int64_t* queue, uint8_t* queued, int64_t* pa,
                          int64_t* pb) {
    int64_t head = 0, tail = 0, left = 0;
    for (int64_t e = 0; e < g->m; ++e) {
        if (!alive[e]) continue;
        ++left;
        if (s[e] < k - 2 && !queued[e]) {
            queued[e] = 1;
            queue[tail++] = e;
        }
    }
    while (head < tail) {
        int64_t e = queue[head++];
        if (!alive[e]) continue;
        alive[e] = 0;
        --left;
        if (level) level[e] = k - 1;
        int64_t c = common(g, g->lo[e], g->hi[e], pa, pb);
        for (int64_t i = 0; i < c; ++i) {
            int32_t f = g->eid[pa[i]], h = g->eid[pb[i]];
            if (!alive[f] || !alive[h]) continue; /* triangle already destroyed */
            --s[f];
            --s[h];
            if (s[f] < k - 2 && !queued[f]) { queued[f] = 1; queue[tail++] = f; }
            if (s[h] < k - 2 && !queued[h]) { queued[h] = 1; queue[tail++] = h; }
        }
    }
    return left;
}

/* The k-truss (k >= 2) of the whole graph: mask[e] = 1 iff e survives.
 * If support_out is not NULL it receives each survivor's support within the
 * truss (0 for removed edges).  Returns the number of surviving edges, or -1
 * for k < 2. */
int64_t oracle_ktruss(const oracle_graph* g, int32_t k, uint8_t* mask, int32_t* support_out) {
    if (k < 2) return -1;
    const int64_t dmax = max_degree(g) + 1;
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->m + 1));
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(g->m + 1));
    uint8_t* queued = (uint8_t*)calloc((size_t)g->m + 1, 1);
    int64_t* pa = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
    int64_t* pb = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
    oracle_support(g, s);
    for (int64_t e = 0; e < g->m; ++e) mask[e] = 1;
    int64_t left = peel_level(g, k, mask, s, NULL, queue, queued, pa, pb);
    if (support_out)
        for (int64_t e = 0; e < g->m; ++e) support_out[e] = mask[e] ? s[e] : 0;
    free(s);
    free(queue);
    free(queued);
    free(pa);
    free(pb);
    return left;
}

/* Truss decomposition: k = 3, 4, ... each level continuing from the previous
 * level's survivors, until no edge is left.  truss[e] = the largest k whose
 * k-truss contains e (2 for an edge in no triangle).  Returns kmax, the
 * largest k with a non-empty k-truss (0 for a graph with no edges). */
int32_t oracle_truss_decomposition(const oracle_graph* g, int32_t* truss) {
    if (g->m == 0) return 0;
    const int64_t dmax = max_degree(g) + 1;
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)g->m);
    uint8_t* alive = (uint8_t*)malloc((size_t)g->m);
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->m);
    uint8_t* queued = (uint8_t*)calloc((size_t)g->m, 1);
    int64_t* pa = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
    int64_t* pb = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
    oracle_support(g, s);
    memset(alive, 1, (size_t)g->m);
    int32_t k = 3;
    int32_t kmax = 2;
    for (;;) {
        int64_t left = peel_level(g, k, alive, s, truss, queue, queued, pa, pb);
        if (left == 0) break;
        kmax = k;
        ++k;
    }
    free(s);
    free(alive);
    free(queue);
    free(queued);
    free(pa);
    free(pb);
    return kmax;
}

/* The first levels of the truss decomposition: k = 3 .. kmax, each level
 * continuing from the previous level's survivors (Section III-B), stopping
 * after kmax.  sizes[k - 3] = number of edges in the k-truss.  Returns 0, or
 * -1 for kmax < 3. */
int oracle_truss_levels(const oracle_graph* g, int32_t kmax, int64_t* sizes) {
    if (kmax < 3) return -1;
    const int64_t dmax = max_degree(g) + 1;
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->m + 1));
    uint8_t* alive = (uint8_t*)malloc((size_t)g->m + 1);
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(g->m + 1));
    uint8_t* queued = (uint8_t*)calloc((size_t)g->m + 1, 1);
    int64_t* pa = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
    int64_t* pb = (int64_t*)malloc(sizeof(int64_t) * (size_t)dmax);
    oracle_support(g, s);
    memset(alive, 1, (size_t)g->m);
    for (int32_t k = 3; k <= kmax; ++k)
        sizes[k - 3] = peel_level(g, k, alive, s, NULL, queue, queued, pa, pb);
    free(s);
    free(alive);
    free(queue);
    free(queued);
    free(pa);
    free(pb);
    return 0;
}

/* Connected components of the subgraph formed by the edges with alive[e] = 1
 * (the k-truss as a set of connected trusses, Section IV-A's enumeration of
 * k-trusses).  A component is the set of vertices reachable from one another
 * through alive edges, with the alive edges among them.  Vertices are
 * visited in increasing id and a search starts at each vertex with an alive
 * edge not yet reached, so the vertex that starts a component is its
 * smallest id; that id labels the component.
 *   edge_label[e]   = label of e's component, or -1 if e is not alive;
 *   vertex_label[v] = label of v's component, or -1 if v has no alive edge
 *                     (may be NULL).
 * Returns the number of components. */
int64_t oracle_truss_components(const oracle_graph* g, const uint8_t* alive,
                                int32_t* edge_label, int32_t* vertex_label) {
    int32_t* lab = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->n > 0 ? g->n : 1));
    int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->n > 0 ? g->n : 1));
    int64_t comps = 0;
    for (int32_t v = 0; v < g->n; ++v) lab[v] = -1;
    for (int32_t v = 0; v < g->n; ++v) {
        if (lab[v] >= 0) continue;
        int has = 0;
        for (int64_t p = g->off[v]; p < g->off[v + 1]; ++p)
            if (alive[g->eid[p]]) {
                has = 1;
                break;
            }
        if (!has) continue;
        ++comps;
        int64_t top = 0;
        lab[v] = v;
        stack[top++] = v;
        while (top > 0) {
            const int32_t x = stack[--top];
            for (int64_t p = g->off[x]; p < g->off[x + 1]; ++p) {
                const int32_t y = g->nbr[p];
                if (alive[g->eid[p]] && lab[y] < 0) {
                    lab[y] = v;
                    stack[top++] = y;
                }
            }
        }
    }
    for (int64_t e = 0; e < g->m; ++e) edge_label[e] = alive[e] ? lab[g->lo[e]] : -1;
    if (vertex_label)
        for (int32_t v = 0; v < g->n; ++v) vertex_label[v] = lab[v];
    free(lab);
    free(stack);
    return comps;
}
