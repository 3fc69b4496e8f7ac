/*
 * tc.h — C ABI of the GB300 triangle-counting / k-truss library.
 *
 * The library implements the kernels of the Static Graph Challenge
 * (Samsi et al., "Static Graph Challenge: Subgraph Isomorphism", 2017):
 * triangle counting (Section III-A), per-edge triangle support and k-truss
 * peeling with the truss decomposition (Section III-B, Algorithm 4).  All
 * computation runs in hand-written CUDA kernels on one GPU; there is no CPU
 * fallback.
 *
 * Conventions shared by every call
 *  - Vertex ids are 0-based int32 in [0, n).  (The Challenge's TSV files are
 *    1-based, Section II; a caller converts them.)
 *  - Edge ids: after cleaning, the graph's undirected edges are listed as
 *    pairs (lo, hi), lo < hi, in lexicographic order of the ORIGINAL ids
 *    (the "canonical edge list").  An edge's position in that list is its
 *    edge id, and every per-edge output is indexed by it.
 *  - Pointers: the caller owns every input and output buffer.  Array
 *    arguments may be device memory or host memory (pageable or pinned);
 *    the library inspects each pointer.  Pinned or registered host memory
 *    (mapped into the device's address space) is read or written in place
 *    by the kernels; pageable host memory is copied through the device.
 *    Scalar outputs (triangles_out, edges_out, kmax_out) are host pointers.
 *  - Streams: `cuda_stream` is a cudaStream_t (NULL = the legacy default
 *    stream).  Work is ordered on that stream.  A call that returns a host
 *    scalar, or writes a host array, synchronises that stream before
 *    returning; a call whose outputs are all device arrays returns without
 *    synchronising.
 *  - Memory: a tc_graph and the scratch of every call are allocated by the
 *    library from the device's stream-ordered pool (cudaMallocAsync) on the
 *    call's stream, on the device current at tc_build_csr.
 *  - Errors: every int-returning call returns TC_OK (0) or a negative
 *    TC_E* code; no exception crosses the ABI.  tc_strerror names a code and
 *    tc_last_error describes the calling thread's most recent failure.
 *  - Threads: distinct graphs may be used concurrently from distinct threads
 *    on distinct streams; one graph must not be used by two calls at once.
 */
#ifndef TC_GB300_H
#define TC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_graph tc_graph; /* opaque, device-resident, owned by the library */

enum {
    TC_OK = 0,
    TC_EINVAL = -1,     /* null pointer, n <= 0, m_in < 0, k < 2, bad flags */
    TC_ERANGE = -2,     /* a vertex id outside [0, n) */
    TC_ENOMEM = -3,     /* a device or host allocation failed */
    TC_ECUDA = -4,      /* a CUDA runtime call or kernel launch failed */
    TC_ETIMEDOUT = -5,  /* a bounded device-side wait gave up */
    TC_EOVERFLOW = -6   /* more than 2^31 - 1 edges after cleaning */
};

/* Flags of tc_build_csr: where src/dst live (AUTO inspects the pointers). */
enum { TC_INPUT_AUTO = 0, TC_INPUT_DEVICE = 1, TC_INPUT_HOST = 2 };

/*
 * tc_build_csr — clean an edge list and build the device graph.
 *
 * Follows Section II's input rules: vertex ids in [0, n), self-loops dropped,
 * a directed pair (u, v) stands for the undirected edge {u, v}, repeated
 * pairs collapse to one edge, weights are 1.  Builds on the device:
 *   - the canonical edge list (see above);
 *   - vertex degrees and a degree order rank(v) = position of (deg(v), v);
 *   - a symmetric CSR over rank ids whose rows are sorted, with the edge id
 *     of every entry; the part of row u above u is the out-list N+(u) of the
 *     degree-oriented adjacency L used by tc_count / tc_edge_support.
 * src, dst: m_in int32 endpoints each (device or host, see flags).
 * m_in >= 0 (0 gives an empty graph); n >= 1.
 * flags: TC_INPUT_AUTO / TC_INPUT_DEVICE / TC_INPUT_HOST.
 * out: receives the new graph (freed with tc_graph_free); untouched on error.
 * Inputs are not retained after the call returns.
 * Errors: TC_EINVAL (null pointers with m_in > 0, n < 1, m_in < 0),
 * TC_ERANGE (an id outside [0, n); no graph is returned), TC_EOVERFLOW,
 * TC_ENOMEM, TC_ECUDA, TC_ETIMEDOUT.
 */
int tc_build_csr(const int32_t* src, const int32_t* dst, int64_t m_in, int32_t n, int flags,
                 void* cuda_stream, tc_graph** out);

/*
 * tc_count — number of triangles (Section III-A).
 *
 * Computes the masked product (L L^T) ∘ L over the degree-oriented adjacency
 * L (the once-per-triangle form of Algorithm 3): for every oriented edge
 * (u, v), |N+(u) ∩ N+(v)|, summed.  Exact int64.  A graph is immutable, so
 * once T is known (an earlier tc_count, or tc_edge_support with
 * triangles_out) it is returned without a launch.
 * triangles_out: host int64.  Synchronises the stream.
 */
int tc_count(tc_graph* g, int64_t* triangles_out, void* cuda_stream);

/*
 * tc_edge_support — triangle support of every edge (Algorithm 4,
 * s = (R == 2) 1 with R = E A): s[e] = number of triangles containing e.
 * Every triangle found by the masked product credits its three edges; the
 * same pass gives T.  The supports are computed once per graph and kept
 * (later calls, and the peel, reuse them).
 * support_out: m int32 in edge-id order (device or host).
 * triangles_out: host int64, may be NULL (then, with a device support_out,
 * the call does not synchronise).
 */
int tc_edge_support(tc_graph* g, int32_t* support_out, int64_t* triangles_out,
                    void* cuda_stream);

/*
 * ktruss — the k-truss (Section III-B): the largest subgraph in which every
 * edge lies in at least k - 2 triangles of the subgraph.  Edges whose
 * support is below k - 2 are removed in bulk rounds and the supports of the
 * edges sharing their triangles are lowered, until no edge is below
 * (Algorithm 4's loop).  k >= 2 (k = 2 keeps every edge).
 * The graph keeps the supports, and the per-edge triangle lists when the
 * peel builds them and they fit, for later ktruss / ktruss_max calls, and
 * the result of the latest ktruss call: a later ktruss with a k at least as
 * large continues from that truss instead of the whole graph (Section
 * III-B's procedure of passing the k-truss on to the next k; the (k+1)-truss
 * lies inside the k-truss, so the result is the same).  tc_graph_info's
 * device_bytes counts what the graph keeps.
 * mask_out: m uint8 in edge-id order, 1 = in the k-truss (device or host).
 * edges_out: host int64, number of edges in the k-truss; may be NULL.
 * Errors: TC_EINVAL for k < 2.
 */
int ktruss(tc_graph* g, int32_t k, uint8_t* mask_out, int64_t* edges_out, void* cuda_stream);

/*
 * ktruss_sizes — the number of edges in the k-truss for every k in
 * [k_lo, k_hi] (Section III-B: the k-trusses nest, so the decomposition's
 * levels k_lo, k_lo + 1, ... each peel the previous level's survivors; one
 * peel from the supports answers the whole range, stopping after k_hi).
 * sizes_out: host int64, k_hi - k_lo + 1 entries (sizes_out[i] for
 * k = k_lo + i; k = 2 gives every edge).  Uses the kept truss numbers of an
 * earlier ktruss_max when the graph keeps results.  Synchronises the stream.
 * Errors: TC_EINVAL unless 2 <= k_lo <= k_hi < k_lo + 64.
 */
int ktruss_sizes(tc_graph* g, int32_t k_lo, int32_t k_hi, int64_t* sizes_out, void* cuda_stream);

/*
 * ktruss_max — truss decomposition (Section III-B): k = 3, 4, ... each level
 * peeling the previous level's survivors, until none is left.
 * kmax_out: host int32, the largest k with a non-empty k-truss (2 if the
 * graph has edges but no triangle, 0 if it has no edge).
 * truss_out: m int32 in edge-id order (device or host), the largest k whose
 * k-truss contains the edge (>= 2); may be NULL.
 * The decomposition stays with the graph when it fits its optional memory
 * (tc_graph_set_memory_limit; 4 bytes per edge): later ktruss_max calls copy
 * it, and ktruss(k) becomes the threshold truss >= k (the k-trusses nest).
 * Synchronises the stream.
 */
int ktruss_max(tc_graph* g, int32_t* kmax_out, int32_t* truss_out, void* cuda_stream);

/* Number of undirected edges after cleaning (m); -1 for a NULL graph. */
int64_t tc_num_edges(const tc_graph* g);

/* Number of vertices n given at build; -1 for a NULL graph. */
int32_t tc_num_vertices(const tc_graph* g);

/*
 * tc_edges — the canonical edge list: lo[e] < hi[e] in original ids, in
 * edge-id order.  lo, hi: m int32 each (device or host).
 */
int tc_edges(const tc_graph* g, int32_t* lo, int32_t* hi, void* cuda_stream);

/*
 * Sizes of a built graph, for reporting (the "edges" and "memory"
 * performance metrics of Section IV) and for work estimates.
 */
typedef struct {
    int64_t n;             /* vertices */
    int64_t m_in;          /* input pairs given to tc_build_csr */
    int64_t m;             /* undirected edges after cleaning */
    int64_t max_degree;    /* largest vertex degree */
    int64_t max_out;       /* largest out-degree |N+(u)| in the degree orientation */
    int64_t wedge_work;    /* sum over oriented edges (u, v) of |N+(u)| + |N+(v)|
                              (the list entries a merge-based masked product
                              reads), or -1 until tc_graph_wedge_work ran */
    int64_t device_bytes;  /* device memory held by the graph (CSR, edge arrays,
                              and what it keeps between calls: supports,
                              triangle lists, the latest k-truss, truss numbers) */
    int64_t peel_rounds;   /* bulk removal rounds of the most recent ktruss /
                              ktruss_max call on this graph (0 if none) */
    int64_t peel_lists;    /* 1 if that call read precomputed per-edge triangle
                              lists, 0 if it intersected neighbour lists, 2 if
                              it read lists kept only for the edges whose
                              support was below a bound and intersected for
                              the others */
    /* Device time (CUDA events on the call's stream, ns; -1 = not run or not
     * measured) of the latest launch on this graph of: the masked-product
     * kernel of tc_count, that of tc_edge_support (measured when the call
     * returns triangles), the triangle-list build and the peel kernel. */
    int64_t count_kernel_ns;
    int64_t support_kernel_ns;
    int64_t lists_kernel_ns;
    int64_t peel_kernel_ns;
    int64_t peel_bytes;    /* algorithmic bytes of that peel launch: 12 per
                              level-scan entry, 8 per triangle- or neighbour-list
                              entry read, 4 per binary-search step and per edge
                              state read, 8 per support decrement */
    /* that peel's work: level-scan entries, list entries read, binary-search
     * steps, edge-state reads, support decrements */
    int64_t peel_scanned;
    int64_t peel_entries;
    int64_t peel_searches;
    int64_t peel_lookups;
    int64_t peel_lowered;
    int64_t truss_cached;  /* 1 if the graph keeps the truss decomposition of
                              its latest ktruss_max (later ktruss calls then
                              threshold it instead of peeling) */
    int64_t column_work;   /* sum over vertices u of |N+(u)| (|N+(u)| - 1) / 2:
                              the out-list entries the column kernel streams
                              (for each oriented edge (u, v), the entries of
                              N+(u) above v), or -1 until tc_graph_wedge_work ran */
    int64_t product_form;  /* the masked-product kernel of the latest tc_count /
                              tc_edge_support launch: 1 columns, 2 warp per
                              edge, 3 thread per edge, 4 rows; 0 if none */
    int64_t lists_bytes;   /* algorithmic bytes of the latest triangle-list build
                              when the column kernel made it (4 per out-list
                              word read, 24 per edge, 24 per vertex, 16 per
                              list entry), else -1 */
} tc_graph_info_t;

/* Fills *info (host pointer) from values the library already holds; launches
 * nothing.  cuda_stream is unused. */
int tc_graph_info(const tc_graph* g, tc_graph_info_t* info, void* cuda_stream);

/* Computes (once per graph, one kernel) the sum over oriented edges (u, v)
 * of |N+(u)| + |N+(v)| into *out (host), and with it tc_graph_info's
 * column_work.  Synchronises the stream. */
int tc_graph_wedge_work(tc_graph* g, int64_t* out, void* cuda_stream);

/*
 * Chooses whether the graph keeps results between calls (keep != 0, the
 * default): the truss numbers of its latest ktruss_max (later ktruss calls
 * then threshold them, Section III-B: the k-trusses nest) and the state of
 * its latest ktruss (a later call with a k at least as large resumes from
 * that truss).  With keep = 0 every ktruss and ktruss_max call peels from
 * the supports, and what was kept is released; structures (the CSR, the
 * supports, triangle lists) are still kept within the memory bound.
 * Results are the same either way; a serving loop that must do each
 * request's work turns it off.  Errors: TC_EINVAL for a NULL graph.
 */
int tc_graph_set_result_cache(tc_graph* g, int32_t keep);

/*
 * Bounds the optional device memory the library may keep for this graph
 * beyond its CSR, edge arrays, supports and call scratch: the per-edge
 * triangle lists of the peel (24 bytes per triangle + 8 per edge), the
 * compacted adjacency of the latest ktruss (16 bytes per edge + 4 per
 * vertex) and the truss numbers of the latest ktruss_max (4 bytes per
 * edge), all of them together.  The triangle-list form of the peel is used
 * only when its lists fit.  bytes < 0 (the default): each structure may take
 * a share of the device's free memory at the call.  Results do not depend on
 * it; memory use and speed do.  A serving loop sets it to keep many resident
 * graphs within a device-memory budget.  Takes effect at the next call;
 * structures above a lowered bound are released then.
 */
int tc_graph_set_memory_limit(tc_graph* g, int64_t bytes);

/*
 * The k-truss as connected trusses (Section IV-A: "enumerating all
 * k-trusses"; the k-truss of ktruss() may fall apart into several connected
 * pieces).  Computes the k-truss (as ktruss(), sharing its cache), then the
 * connected components of the subgraph of its edges.  A component is
 * labelled by its smallest vertex id (original ids).
 *   edge_label_out:   m entries in canonical edge order (device or host):
 *                     the label of the edge's component, -1 for an edge
 *                     outside the k-truss; may be NULL only when m = 0;
 *   vertex_label_out: n entries (device or host, may be NULL): the label of
 *                     the vertex's component, -1 for a vertex with no
 *                     k-truss edge;
 *   count_out:        number of components (host).
 * Synchronises the stream.  Errors: TC_EINVAL (NULL graph, count_out or
 * edge_label_out, k < 2), TC_ENOMEM, TC_ECUDA, TC_ETIMEDOUT.
 */
int ktruss_components(tc_graph* g, int32_t k, int32_t* edge_label_out, int32_t* vertex_label_out,
                      int64_t* count_out, void* cuda_stream);

/*
 * Reads an edge list from a file (Section II's inputs): format 1 = the
 * Graph Challenge's tab-separated lines "u v [weight]", 2 = a Matrix Market
 * coordinate file ("%%MatrixMarket matrix coordinate ..." header, a
 * "rows cols entries" size line, then "i j [value]" lines), 0 = by the
 * file name (.mtx / .mm: Matrix Market, else tab-separated).  Ids in the
 * file are 1-based and are written 0-based; weights and values are ignored
 * (any listed pair is an edge); blank lines and comment lines ('%', and '#'
 * in tab-separated files) are skipped.  Entries are written in file order,
 * with nothing cleaned: pass the arrays to tc_build_csr.
 *   src, dst:  host int32 arrays of `capacity` entries, or both NULL to only
 *              count (call once with NULL to size the arrays);
 *   m_out:     entries in the file;
 *   n_out:     vertex count: the largest id in a tab-separated file, the
 *              declared size in a Matrix Market file.
 * Host code only (no device work).  Errors: TC_EINVAL (NULL path or
 * outputs, unreadable file, a malformed line — the message names it —, a
 * Matrix Market entry count other than the declared one, capacity smaller
 * than the entries), TC_ERANGE (an id of 0, above 2^31 - 1, or outside the
 * declared matrix size).
 */
int tc_read_edges(const char* path, int format, int32_t* src, int32_t* dst, int64_t capacity,
                  int64_t* m_out, int32_t* n_out);

/*
 * Serving (a request loop over device-resident graphs).  The paper times
 * single kernels; this runs them as a service: requests for the triangle
 * count or the k-truss size of one graph of a pool arrive over time and are
 * served by `slots` worker threads, each with its own CUDA stream, with
 * continuous batching: a free slot takes the oldest request that can run
 * now (its graph idle — a graph serves one call at a time — and resident,
 * or admissible within the device-memory budget after evicting
 * least-recently-used idle graphs), so requests that arrive while others
 * run overlap on the device.  Graphs are built on first use from the
 * caller's host edge lists (tc_build_csr rules) and get a memory bound of
 * optional_bytes_per_pair x input pairs (tc_graph_set_memory_limit); a
 * graph's first k-truss request computes its truss decomposition, which it
 * keeps, so later k-truss requests on it threshold the truss numbers.
 */
typedef struct {
    const int32_t* src;  /* host, m_in entries; must stay valid while the server lives */
    const int32_t* dst;
    int64_t m_in;
    int32_t n;
    int32_t pad;
} tc_graph_source;

#define TC_REQ_COUNT 0   /* result: the graph's triangle count */
#define TC_REQ_KTRUSS 1  /* result: edges in the graph's k-truss (k >= 2) */

typedef struct {
    int32_t graph;     /* index into the sources */
    int32_t kind;      /* TC_REQ_COUNT or TC_REQ_KTRUSS */
    int32_t k;
    int32_t pad;
    double arrival_s;  /* seconds after the run starts (open loop); non-decreasing */
} tc_request;

typedef struct {
    int64_t result;
    double start_s;    /* when a slot took the request (seconds after the run start) */
    double done_s;     /* when its result was on the host */
    int32_t status;    /* TC_* of the request */
    int32_t slot;
} tc_response;

typedef struct {
    int64_t builds, evictions, max_concurrent, peak_reserved_bytes, errors;
    int64_t violations;        /* test hook only: concurrent calls seen on one graph */
    int64_t reserved_bytes;    /* device bytes reserved for resident graphs now */
    int64_t resident_graphs;
} tc_server_stats;

typedef struct tc_server tc_server;

/* Creates a server on the current device (graphs are built later, on first
 * use).  budget_bytes: device memory for resident graphs.  slots: 1..256.
 * Errors: TC_EINVAL (NULL, bad sizes, a bad source), TC_ECUDA, TC_ENOMEM. */
int tc_server_create(const tc_graph_source* sources, int32_t num_graphs, int64_t budget_bytes,
                     int64_t optional_bytes_per_pair, int32_t slots, tc_server** out);

/* Serves num_reqs requests and returns when all are done.  open_loop = 1:
 * a request becomes available at its arrival_s; 0: all at once (closed
 * loop).  slots: how many of the server's slots serve this run (0 = all;
 * 1 = the plain loop, one request at a time in order, on the same resident
 * graphs).  out[i] receives request i's result, times, status and slot;
 * *wall_s (may be NULL) the run's duration.  Latency of request i =
 * out[i].done_s - reqs[i].arrival_s.  Graphs stay resident between runs.
 * Returns TC_OK, or TC_ECUDA if any request failed (its status says how),
 * TC_ERANGE / TC_EINVAL for a request naming no graph or malformed. */
int tc_server_run(tc_server* srv, const tc_request* reqs, int64_t num_reqs, int32_t open_loop,
                  int32_t slots, tc_response* out, double* wall_s);

/* Whether the server's graphs keep results between requests (keep != 0,
 * the default: a graph's first k-truss request computes and keeps its truss
 * decomposition, later ones threshold it).  keep = 0: every k-truss request
 * peels on the device (tc_graph_set_result_cache on each graph, now and on
 * those built later); the CSR, supports and structures within the memory
 * bound stay resident.  Call between runs.  Errors: TC_EINVAL for NULL. */
int tc_server_set_result_cache(tc_server* srv, int32_t keep);

/* Counters of the server's life so far (host struct).  Launches nothing. */
int tc_server_get_stats(const tc_server* srv, tc_server_stats* out);

/* Frees the server's graphs and streams.  NULL is a no-op. */
void tc_server_destroy(tc_server* srv);

/* Test hook: servers created while this is on run their scheduler with
 * sleeps in place of device work (no CUDA calls; results are
 * graph * 1000 + k), so the host logic can be tested without a GPU.
 * Returns the previous setting. */
int tc_debug_server_fake(int on);

/* Number of CUDA kernels the library has launched in this process (all
 * graphs, all threads); lets a caller count the launches of a region. */
int64_t tc_launch_count(void);

/*
 * Batches: many independent graphs in one pass.
 *
 * tc_batch_run cleans and builds all graphs of the batch as one graph (the
 * disjoint union, vertex ids offset per graph: a triangle or a k-truss never
 * spans two graphs, so the union's triangles and trusses are exactly the
 * graphs'), then computes per-graph triangle counts (Section III-A) and,
 * if k >= 2, per-graph k-truss sizes (Section III-B) with one launch per
 * phase over all graphs.  With use_graph = 1 the query phase (supports,
 * per-graph sums, the peel) is captured into one CUDA graph and launched
 * once.  The first batch with a given size/degree signature times the
 * masked-product kernels, and both peel forms at three grid sizes, on the
 * batch and keeps the fastest; later batches with that signature reuse the
 * choice.
 */
typedef struct {
    int64_t build_ns;          /* union build, CUDA events on the call's stream */
    int64_t query_ns;          /* supports + per-graph sums + peel */
    int64_t m;                 /* edges of all graphs after cleaning */
    int64_t triangles;         /* triangles of all graphs */
    int32_t intersect_form;    /* 1 = column kernel, 2 = edge-per-warp kernel,
                                  3 = edge-per-thread kernel, 4 = row kernel */
    int32_t peel_form;         /* 0 = no peel, 1 = triangle lists, 2 = intersections
                                  (or lists below the support bound with them) */
    int32_t tuned_from_cache;  /* 1 if the kernel choice came from the tuner's cache */
    int32_t captured;          /* 1 if the query ran as one CUDA graph launch */
    int32_t peel_blocks;       /* the tuner's cap on the peel's grid (0 = none) */
    int32_t light_degree;      /* column kernel: the tuner's degree bound of the
                                  columns that take a warp each (heavier ones take
                                  a block); 0 for the other kernels */
} tc_batch_stats_t;

typedef struct {
    int32_t num_graphs;          /* >= 1 */
    const int32_t* n;            /* host: vertices of each graph (each >= 1; sum < 2^31) */
    const int64_t* edge_off;     /* host: num_graphs + 1 offsets into src/dst, edge_off[0] = 0 */
    const int32_t* src;          /* edge_off[num_graphs] pairs, ids local to their graph */
    const int32_t* dst;          /* (device or host) */
    int32_t k;                   /* k-truss per graph (>= 2), or 0 for triangle counts only */
    int32_t use_graph;           /* 1: run the query phase as one captured CUDA graph */
    int64_t* triangles_out;      /* host: num_graphs triangle counts (required) */
    int64_t* edges_out;          /* host: num_graphs edge counts after cleaning, or NULL */
    int64_t* truss_edges_out;    /* host: num_graphs k-truss edge counts, or NULL */
    tc_batch_stats_t* stats_out; /* host, or NULL */
} tc_batch_desc;

/* Runs a batch.  Synchronises the stream (NULL: the library uses a private
 * stream).  Errors: TC_EINVAL (bad descriptor), TC_ERANGE (a local id outside
 * its graph), TC_EOVERFLOW, TC_ENOMEM, TC_ECUDA, TC_ETIMEDOUT. */
int tc_batch_run(const tc_batch_desc* d, void* cuda_stream);

/*
 * tc_sort_keys_static — sorts n uint64 keys ascending, in place, by their low
 * key_bits bits (an LSD radix sort, the library's own sort), WITHOUT
 * ALLOCATING: no cudaMalloc, no stream-ordered allocation, no allocating
 * library routine.  The paper has no counterpart; this entry point exists for
 * callers that cannot allocate device memory where they call it — code whose
 * device memory is owned by another allocator (e.g. a framework's caching
 * pool that holds the free memory), code with a fixed pre-planned memory
 * budget or a real-time deadline, code that must not enter the allocator.
 *
 * Scratch: one file-scope device array of TC_SORT_STATIC_SCRATCH_BYTES
 * (about 8.5 MiB), which every GPU that loads the library holds until the
 * process exits.  Limit: n <= TC_SORT_STATIC_MAX_KEYS (2^20); larger n
 * returns TC_EOVERFLOW without touching the keys.
 * keys: device memory of the caller, n entries (host pointers: TC_EINVAL).
 * key_bits: 1..64; bits above key_bits are ignored by the ordering (the
 * last digit pass masks them), and keys equal in their low key_bits bits
 * keep their input order (the sort is stable).
 * The first call on a device sets the array up (looks up its device address
 * and sets a kernel attribute) with that device current: make that first
 * call before any stream capture.  Every call shares the one array and the
 * array keeps the last call's contents (each call clears what must start at
 * zero): calls whose work overlaps on the GPU — on different streams or
 * threads without ordering between them — race and corrupt each other.
 * Synchronises the stream (to report a device-side wait that ran out:
 * TC_ETIMEDOUT).
 */
#define TC_SORT_STATIC_MAX_KEYS (1 << 20)
#define TC_SORT_STATIC_SCRATCH_BYTES ((size_t)8929536)
int tc_sort_keys_static(uint64_t* keys, int64_t n, int32_t key_bits, void* cuda_stream);

/* Releases a graph (NULL is a no-op).  Synchronises the device's work on
 * the graph's last stream first. */
void tc_graph_free(tc_graph* g);

/* Static description of a TC_* code. */
const char* tc_strerror(int code);

/* Description of the calling thread's most recent failed call ("" if none). */
const char* tc_last_error(void);

/*
 * Test hook for host-side fault injection: the nth device allocation made
 * by the library from now on (1 = the next one) fails as if the device were
 * out of memory; 0 disables.  Returns the previous setting.
 */
int64_t tc_debug_fail_alloc(int64_t nth);

/*
 * Test hook: which form of the peel ktruss / ktruss_max use.  0 = automatic
 * (per-edge triangle lists for every edge when they fit in free device
 * memory, else lists for only the edges whose support is below 8 with
 * intersections of live neighbour lists for the others when those fit, else
 * intersections alone), 1 = triangle lists (for every edge where 3T < 2^32,
 * else the bounded lists), 2 = always intersections, 3 = always the bounded
 * lists with intersections.  All forms give the same results.  Returns the
 * previous mode; other values leave it unchanged.
 */
int tc_debug_peel_mode(int mode);

/*
 * Test hook: which kernel tc_count / tc_edge_support (and the triangle-list
 * build of the peel) use.  0 = automatic (one thread per oriented edge
 * merging the two out-lists when the largest out-list has at most 16
 * entries; else the column kernel when the largest out-list fits its
 * shared-memory hash table; else one warp per oriented edge), 1 = the
 * column kernel (N+(v) hashed, the in-neighbours' out-lists above v
 * streamed against it) where the graph allows it, 2 = always one warp per
 * edge, 3 = always one thread per edge, 4 = the row kernel (N+(u) hashed,
 * its out-neighbours' out-lists streamed) where the graph allows it.  All
 * give the same results.  Returns the previous mode.
 */
int tc_debug_intersect_mode(int mode);

/*
 * Test hook: upper bound, in nanoseconds, on every device-side spin wait
 * (default 2e9).  A wait that runs out makes the call return TC_ETIMEDOUT.
 * Returns the previous value; values <= 0 leave it unchanged.
 */
int64_t tc_debug_spin_limit_ns(int64_t ns);

#ifdef __cplusplus
}
#endif

#endif /* TC_GB300_H */
