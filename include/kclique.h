/*
 * kclique.h -- C ABI of libkclique.so: exact k-clique counting on a low
 * out-degree orientation (the arb-count method of Shi, Dhulipala and Shun,
 * "Parallel Clique Counting and Peeling Algorithms", Section 3), on one
 * NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 *  - Pointers named d_* are device pointers on the current CUDA device;
 *    pointers named h_* are host pointers. The library never frees a
 *    caller's buffer.
 *  - All device work is enqueued on the caller's stream `stream` (0 = the
 *    legacy default stream). Entry points that return a host value
 *    synchronise that stream before returning.
 *  - Every entry point returns a kc_status. Nothing throws or aborts across
 *    the boundary; CUDA errors are reported as KC_ECUDA (the CUDA error string
 *    is available from kc_last_cuda_error()).
 *  - Counts are exact unsigned 64-bit integers. A count that does not fit is
 *    reported as KC_ERANGE, never wrapped.
 *  - Thread safety: distinct kc_dag handles may be used concurrently from
 *    different host threads and streams; one handle may be read (counted)
 *    concurrently, since counting never writes to it.
 */
#ifndef KCLIQUE_H
#define KCLIQUE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *kc_stream_t; /* a cudaStream_t */

typedef enum {
  KC_OK = 0,
  KC_EINVAL = 1,    /* bad argument, k out of range, or a malformed CSR */
  KC_ERANGE = 2,    /* a count does not fit in uint64 */
  KC_ENOMEM = 3,    /* a device allocation failed */
  KC_ETIMEDOUT = 4, /* the deadline passed or the cancel flag was raised */
  KC_ECUDA = 5,     /* a CUDA runtime error; see kc_last_cuda_error() */
  KC_ECAPACITY = 6  /* a root's out-neighbourhood exceeds KC_MAX_OUT_DEGREE */
} kc_status;

/* Largest k accepted (k = 1 .. KC_KMAX). */
#define KC_KMAX 32
/* Largest out-degree a root may have in the oriented graph. Under the degree
 * ordering every out-degree is at most sqrt(2m), so this bound is reached only
 * by graphs with m above ~1.3e8 that also hold a clique-like core of more than
 * 16384 vertices. */
#define KC_MAX_OUT_DEGREE 16384

/* Orientation methods (Section 3.1; Section 5, "Algorithm Implementations"). */
#define KC_ORIENT_DEGREE 0 /* rank by (degree, id), ascending */
#define KC_ORIENT_GP 1     /* Goodrich-Pszona rounds, Algorithm 3 with epsilon = 1 */
#define KC_ORIENT_BE 2     /* Barenboim-Elkin rounds (Section 3.1), epsilon = 1: remove every vertex of
                              induced degree < 3 * alpha~, alpha~ = 4 * the approximate densest
                              subgraph's density (removal rounds at degree <= 4 * density) */
/* Flags or-ed into `method`: */
#define KC_VALIDATE_SYMMETRY 0x100 /* also check that every arc u->v has v->u */
#define KC_CORE_BITS 0x200         /* always build the dense-core bit matrix (see kc_set_core_policy) */
#define KC_NO_CORE_BITS 0x400      /* never build it (default: built where it pays, see below) */

/*
 * Simple undirected graph in CSR form (Section 2, "Graph Storage").
 *   n        number of vertices (ids 0 .. n-1)
 *   nnz      number of directed arcs = 2m (each undirected edge twice)
 *   d_row_ptr device uint64[n+1], d_row_ptr[0] = 0, d_row_ptr[n] = nnz
 *   d_col    device uint32[nnz], row v = neighbours of v, strictly ascending,
 *            no self-loops (the paper assumes simple graphs, Section 2)
 * Borrowed: the library reads it during kc_orient only.
 */
typedef struct {
  uint32_t n;
  uint64_t nnz;
  const uint64_t *d_row_ptr;
  const uint32_t *d_col;
} kc_csr;

/* Opaque oriented graph (the DAG DG of Algorithm 1) with library-owned device
 * buffers: out-lists N+(v) (neighbours later in the total order), each sorted
 * in the total order itself (by rank, the order that decided the arc
 * directions), plus the root work list used by the counting kernels. */
typedef struct kc_dag kc_dag;

/*
 * kc_orient -- Orient(G) of Algorithm 1 (Section 3.1): rank the vertices by
 * the chosen total order and keep each edge as one arc from its lower to its
 * higher endpoint ("direct the graph in CSR format ... using prefix sum and
 * filter", end of Section 3.1).
 *   g       the input CSR (device arrays)
 *   method  KC_ORIENT_DEGREE, KC_ORIENT_GP or KC_ORIENT_BE, optionally | KC_VALIDATE_SYMMETRY
 *           and | KC_CORE_BITS or | KC_NO_CORE_BITS (not both)
 *   out     receives a new handle on success (*out untouched on error)
 * The CSR is validated first (ascending rows, no self-loops, ids < n,
 * row_ptr consistent; symmetry on request): a violation gives KC_EINVAL.
 * Synchronises `stream`. Free the handle with kc_dag_free.
 *
 * Dense core (a layout of the DAG; the paper has no counterpart). The build
 * of a root u's first-level induced subgraph (Section 3.4) reads the out-list
 * of every member of N+(u). The handle may also hold a bit matrix over a set
 * C of the highest-ranked vertices: every vertex whose ranking key is at least
 * a threshold, so that an out-neighbour of a vertex of C is in C. Bit (a, b)
 * is set iff C has the arc a -> b. The counting calls then take the row of a
 * member x of N+(u) from the matrix, one bit per later member of N+(u),
 * instead of scanning N+(x), where that reads less (kc_set_core_policy).
 * Counts are the same with and without it.
 * By default it is built when the largest out-degree is at least 128 and the
 * builds of all roots would read on average at least 16 out-list entries per
 * arc (the sum over arcs u -> x of d+(x)). Its size is at most
 * kc_set_core_policy's max_vertices, its matrix at most the size of the DAG's
 * arrays (64 MiB at least) and a quarter of the free device memory; if an
 * allocation for it fails, the handle has no core. With KC_CORE_BITS it is
 * always built (up to max_vertices) and a failed allocation gives KC_ENOMEM.
 * It costs |C|^2/8 bytes of device memory and one pass over the keys and the
 * core's arcs.
 */
kc_status kc_orient(const kc_csr *g, int method, kc_dag **out, kc_stream_t stream);

/*
 * Process-wide settings of the dense core (see kc_orient).
 *   max_vertices  largest core that kc_orient builds (default 131072 vertices,
 *                 a 2 GiB matrix); 0: none
 *   ratio         the counting calls take member x's row from the matrix when
 *                 d+(x) >= ratio * (members of N+(u) after x) (default 1;
 *                 0: always, for every member in the core); UINT32_MAX: the
 *                 counting calls do not use the matrix at all
 * Read by later kc_orient calls (max_vertices) and later counting calls
 * (ratio). Not synchronised with calls running on other threads.
 */
void kc_set_core_policy(uint32_t max_vertices, uint32_t ratio);

/* Number of vertices in the handle's dense core (0: it has none). */
uint32_t kc_dag_core_vertices(const kc_dag *d);

/* Release a handle (stream-ordered on the stream it was created on). NULL is a no-op. */
void kc_dag_free(kc_dag *d);

/* Vertex count n, arc count m (= undirected edges), largest out-degree. */
uint32_t kc_dag_n(const kc_dag *d);
uint64_t kc_dag_m(const kc_dag *d);
uint32_t kc_dag_max_out_degree(const kc_dag *d);

/*
 * Copy the oriented graph out (device to device): d_ptr uint64[n+1] and
 * d_col uint32[m], in the vertex ids of the input CSR, each out-list in
 * increasing rank (degree order: by (degree, id); Goodrich-Pszona: by
 * (round, induced degree at removal, id)). Either may be NULL.
 * Synchronises `stream`.
 */
kc_status kc_dag_export(const kc_dag *d, uint64_t *d_ptr, uint32_t *d_col, kc_stream_t stream);

/*
 * kc_count -- arb-count(G, k) of Algorithm 1: the number of k-cliques
 * (Section 2: k vertices with all k(k-1)/2 edges present).
 *   k        1 .. KC_KMAX (k = 1 gives n, k = 2 gives m)
 *   h_total  receives the count
 * Synchronises `stream`. KC_ERANGE if the count does not fit in uint64.
 */
kc_status kc_count(const kc_dag *d, int k, uint64_t *h_total, kc_stream_t stream);

/*
 * kc_count_per_vertex -- arb-count-v (Section 3.2, used by Algorithm 2):
 * d_out[v] = number of k-cliques that contain v, for every vertex v (so the
 * entries sum to k times the total).
 *   d_out    device uint64[n], caller-owned; overwritten
 *   h_total  optional (NULL allowed): receives the total count
 * Synchronises `stream`.
 */
kc_status kc_count_per_vertex(const kc_dag *d, int k, uint64_t *d_out, uint64_t *h_total,
                              kc_stream_t stream);

/*
 * kc_count_per_arc -- rooted counts used for sampled parity checks: for the
 * arc with index e in the exported out-lists (u -> v, e in
 * [ptr[u], ptr[u+1])), d_out[e] = number of k-cliques whose two lowest
 * vertices in the total order are u and v (the k-cliques found below that
 * arc by the recursion of Algorithm 1). k >= 2.
 *   d_out    device uint64[m], caller-owned; overwritten
 *   h_total  optional: receives the total count
 * Synchronises `stream`.
 */
kc_status kc_count_per_arc(const kc_dag *d, int k, uint64_t *d_out, uint64_t *h_total,
                           kc_stream_t stream);

/*
 * kc_count_budget -- kc_count (d_out NULL) or kc_count_per_vertex (d_out
 * device uint64[n]) with a time budget for the pass. (The paper has no
 * counterpart: a control for callers that serve requests.) The budget starts
 * when the pass starts on the GPU: a one-thread kernel enqueued on `stream`
 * just before the counting kernels takes the deadline from the device clock.
 * Past it the kernels take no new root, item or first-level sub-problem and
 * the call returns KC_ETIMEDOUT; the partial count is discarded and d_out is
 * left undefined. A sub-problem already started runs to its end, so a pass
 * can overrun its budget by one sub-problem.
 *   budget_us  1 .. 2^63 / 1000 microseconds
 *   h_total    receives the count when the pass finished in time
 * Synchronises `stream`. Other status codes as kc_count.
 */
kc_status kc_count_budget(const kc_dag *d, int k, uint64_t *d_out, uint64_t budget_us, uint64_t *h_total,
                          kc_stream_t stream);

/*
 * kc_count_roots -- rooted counts of a list of roots: d_out[i] = number of
 * k-cliques whose lowest vertex in the total order is d_roots[i], i.e. the
 * term that the top call of Algorithm 1 adds for that vertex (every clique is
 * found once, below its lowest vertex). Summed over all vertices this is
 * kc_count; over a subset of roots it is that subset's share, which serves
 * sampled checks on graphs too large to count whole and partitions of the
 * roots between independent passes.
 *   d_roots    device uint32[num_roots], distinct vertex ids < n; borrowed
 *   num_roots  may be 0
 *   d_out      device uint64[num_roots], caller-owned; overwritten
 *   h_total    optional (NULL allowed): the sum of d_out
 *   k          1 .. KC_KMAX (k = 1: 1 per root; k = 2: the root's out-degree)
 * The roots are copied to the host and ordered there by out-degree, then
 * counted by the same persistent kernels as kc_count. Synchronises `stream`.
 * KC_EINVAL for an id >= n or a repeated id; KC_ERANGE on uint64 overflow.
 */
kc_status kc_count_roots(const kc_dag *d, int k, const uint32_t *d_roots, uint32_t num_roots, uint64_t *d_out,
                         uint64_t *h_total, kc_stream_t stream);

/*
 * kc_count_noalloc -- the same total as kc_count, computed without allocating
 * any device memory. (The paper has no counterpart: this is an interface for
 * callers that cannot allocate.)
 *
 * Some callers cannot call cudaMalloc where they count: code under a fixed
 * memory budget or behind a custom allocator that owns the device memory (an
 * allocation by this library would fail or escape the owner's accounting), or
 * latency-critical paths that must not take allocator locks. kc_count
 * allocates a small work block (and, for very large out-neighbourhoods,
 * per-block matrices) on every call; this entry point takes that scratch from
 * one static device array of KC_NOALLOC_SCRATCH_BYTES instead, which every
 * GPU that loads the library holds until the process exits.
 *   d        a handle from kc_orient (created earlier, e.g. at set-up)
 *   k        1 .. KC_KMAX
 *   h_total  receives the count
 * Synchronises `stream`. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture. All calls share the one array and it keeps the last call's
 * contents (the entry point clears what must start at zero): calls that
 * overlap on the GPU, from different streams or threads, race and must be
 * serialised by the caller. Returns KC_ECAPACITY when one root's bit matrix
 * (largest out-degree about 8100 and up) does not fit the array; the other
 * status codes are those of kc_count (a CUDA error is recorded for
 * kc_last_cuda_error).
 */
#define KC_NOALLOC_SCRATCH_BYTES (8u << 20)
kc_status kc_count_noalloc(const kc_dag *d, int k, uint64_t *h_total, kc_stream_t stream);

/*
 * Batches of many small graphs (the paper counts one graph per call; this is
 * the many-graph form of the same arb-count pass, for workloads of thousands
 * of uneven graphs).
 *
 * A batch is one kc_dag oriented from the disjoint union of the graphs: graph
 * g owns the vertex ids [off[g], off[g+1]) of the union CSR (concatenate the
 * graphs' CSRs, shifting each graph's ids by off[g]) and has its own clique
 * size k[g]. Since no arc joins two graphs, the union's k-cliques rooted in
 * graph g are exactly graph g's k[g]-cliques, so all graphs are counted by one
 * pass of the persistent kernels, each root with its own graph's k.
 *   num_graphs        >= 1
 *   d_vertex_offsets  device uint64[num_graphs+1], off[0] = 0,
 *                     non-decreasing, off[num_graphs] = n of the union
 *   d_k               device uint8[num_graphs], each in [3, KC_KMAX]
 *                     (k = 1 and 2 are the graph's n and m)
 *   k_min             smallest value in d_k (roots with fewer than k_min-1
 *                     out-neighbours are skipped without being visited)
 * If arcs do join two graphs, total[g] counts the cliques whose lowest vertex
 * (in the total order of the orientation) lies in graph g.
 */
typedef struct {
  uint32_t num_graphs;
  const uint64_t *d_vertex_offsets;
  const uint8_t *d_k;
  uint8_t k_min;
} kc_batch;

/*
 * Tunables of a counting pass (0 in a field = the built-in default):
 *   light_max    warp/block split: roots with out-degree <= light_max are
 *                counted by one warp, larger ones by one 512-thread block
 *                (2 .. 64; default 64)
 *   compact_max  bitset width of the compacted sub-problems: candidate sets
 *                of at most this many vertices are renumbered into a 1- or
 *                2-word (64- or 128-bit) bit matrix (1 .. 128; default 128)
 *   chunk        work a warp takes per pull from the atomic work queue of
 *                the warp kernel: roots (out-degree order) or groups of 32
 *                vertex ids (id order) (default 1)
 *   light_order  order in which warps take the warp roots:
 *                KC_LIGHT_BY_DEGREE = decreasing out-degree (load balance),
 *                KC_LIGHT_BY_ID = increasing vertex id (locality: a batch's
 *                graphs are counted one id range at a time, so their
 *                out-lists stay in L2, but 32 consecutive ids go to one
 *                warp); 0 = by out-degree
 * Every setting gives the same counts; only the speed differs.
 */
#define KC_LIGHT_BY_DEGREE 1
#define KC_LIGHT_BY_ID 2
typedef struct {
  uint32_t light_max;
  uint32_t compact_max;
  uint32_t chunk;
  uint32_t light_order;
} kc_params;

/*
 * kc_count_batched -- the k[g]-clique count of every graph of a batch.
 *   d         kc_orient of the union CSR (see kc_batch)
 *   prm       tunables or NULL
 *   d_totals  device uint64[num_graphs], caller-owned, overwritten
 *   h_total   optional: receives the sum over all graphs
 * Allocates and frees its work space; synchronises `stream`. KC_EINVAL if
 * a d_k entry lies outside [3, KC_KMAX] (detected on the device).
 */
kc_status kc_count_batched(const kc_dag *d, const kc_batch *b, const kc_params *prm, uint64_t *d_totals,
                           uint64_t *h_total, kc_stream_t stream);

/*
 * A prepared batched pass for repeated, capturable launches: kc_plan_create
 * sizes the kernels for (d, b, prm), allocates the work block and any global
 * scratch, and keeps the pointers (d, b's arrays and d_totals must stay valid
 * while the plan lives). kc_plan_launch only enqueues work on `stream`: two
 * memsets (totals and work block) and the counting kernels, with no
 * allocation and no synchronisation, so it may be recorded into a CUDA graph
 * by stream capture and replayed. kc_plan_result copies the work block back,
 * synchronises `stream` and maps the device status of the last completed
 * launch to a kc_status (h_total, optional, receives the sum over graphs).
 * One plan's launches must not overlap on the GPU (they share its work
 * block); distinct plans are independent. kc_plan_free releases the plan's
 * buffers in the order of the stream it was created on: call it after the
 * last launch has completed (kc_plan_result synchronises), or after that
 * launch's stream has been made to wait on it.
 */
typedef struct kc_plan kc_plan;
kc_status kc_plan_create(const kc_dag *d, const kc_batch *b, const kc_params *prm, uint64_t *d_totals,
                         kc_plan **out, kc_stream_t stream);
kc_status kc_plan_launch(kc_plan *p, kc_stream_t stream);
kc_status kc_plan_result(kc_plan *p, uint64_t *h_total, kc_stream_t stream);
void kc_plan_free(kc_plan *p);

/*
 * kc_autotune_batched -- the tunables (light_order, light_max, compact_max, chunk) that
 * count the batch fastest on this device: times each candidate of a small
 * grid (two launches each, CUDA events, after one warm-up launch) and writes
 * the fastest to *out; *h_best_ms (optional) receives its time. d_totals is
 * used as the output of the trial passes. Synchronises `stream`.
 */
kc_status kc_autotune_batched(const kc_dag *d, const kc_batch *b, uint64_t *d_totals, kc_params *out,
                              float *h_best_ms, kc_stream_t stream);

/*
 * Serving: a request loop for count and per-vertex count requests on
 * device-resident oriented graphs (the paper counts one graph per call; this
 * is the many-request form of the same pass).
 *
 * kc_server_create starts a dispatcher thread with cfg->slots slots (one
 * CUDA stream each) on the current device. kc_server_submit queues a request
 * (a kc_dag that stays valid until the request is released, k in
 * [3, KC_KMAX], per_vertex 0 or 1, timeout_us the time budget from submission
 * or 0 for none) and returns at once. Requests are admitted
 * first come, first served, as soon as a slot is free and their device
 * footprint (the per-vertex output 8n bytes, the work block and the global
 * scratch of their largest roots) fits cfg->hbm_budget beside the requests in
 * flight; a request that does not fit waits, unless nothing else is
 * running (so a client holding per-vertex outputs cannot stall the queue). Admitted requests run concurrently on their slots' streams, each
 * with grids sized to its own work and capped at cfg->grid_share_pct percent
 * of the full persistent grid, so their kernels overlap on the GPU. The result of a
 * request does not depend on what else is in flight. A request whose time
 * budget runs out stops taking new roots (the kernels check the device clock,
 * mapped from the host clock when the server starts) and completes with
 * status KC_ETIMEDOUT; roots already taken finish first.
 *
 * kc_server_wait blocks until request id completes (timeout_ms < 0: no limit;
 * KC_ETIMEDOUT if it has not completed in time) and fills *out: out->status
 * is the request's own kc_status, out->total its count, and the times are
 * host steady-clock nanoseconds from submission. A count request is released
 * by a successful wait; a per-vertex request keeps its output (and its share
 * of the budget) until kc_server_release, after kc_server_fetch_per_vertex
 * has copied the n counts to dst (host or device memory; synchronises
 * `stream`). kc_server_destroy waits for the requests in flight and drops
 * the queued ones.
 */
typedef struct kc_server kc_server;
typedef struct {
  uint32_t slots;          /* requests in flight at most, 1 .. 64 */
  uint32_t grid_share_pct; /* grid cap per request, percent of the full persistent grid (0 = 100) */
  uint64_t hbm_budget;     /* bytes of request memory in flight */
} kc_server_config;
typedef struct {
  int status;          /* the request's kc_status */
  int slot;            /* slot it ran on */
  uint64_t total;      /* its count */
  uint64_t queue_ns;   /* submission to admission */
  uint64_t run_ns;     /* admission to completion */
  uint64_t latency_ns; /* submission to completion */
} kc_request_result;
typedef struct {
  uint64_t submitted, admitted, completed;
  uint64_t peak_in_flight; /* most requests on the GPU at once */
  uint64_t peak_bytes;     /* most request memory admitted at once */
  uint64_t bytes_in_use;   /* request memory held now */
  uint64_t queued;         /* requests waiting now */
} kc_server_stats;
kc_status kc_server_create(const kc_server_config *cfg, kc_server **out);
kc_status kc_server_submit(kc_server *s, const kc_dag *d, int k, int per_vertex, uint64_t timeout_us,
                           uint64_t *req_id);
kc_status kc_server_wait(kc_server *s, uint64_t req_id, int timeout_ms, kc_request_result *out);
kc_status kc_server_fetch_per_vertex(kc_server *s, uint64_t req_id, uint64_t *dst, kc_stream_t stream);
kc_status kc_server_release(kc_server *s, uint64_t req_id);
kc_status kc_server_get_stats(kc_server *s, kc_server_stats *out);
void kc_server_destroy(kc_server *s);

/*
 * kc_count_colorful -- approximate k-clique count by colorful sparsification
 * (Section 3.3, "Sampling"; estimator theorem in Appendix B): every vertex
 * takes a color in [0, colors) uniformly at random, only monochromatic edges
 * are kept, and the k-clique count C of that graph (oriented by `method`,
 * counted exactly by arb-count) gives the unbiased estimate C * colors^(k-1).
 *   g                the input CSR (validated as by kc_orient)
 *   k                1 .. KC_KMAX
 *   colors           c >= 1 (c = 1 keeps every edge: the exact count)
 *   seed             vertex v's color is the high 32 bits of
 *                    splitmix64(seed + (v + 1) * 0x9E3779B97F4A7C15)
 *                    (Steele, Lea and Flood, 2014) scaled to [0, c)
 *   h_sparse_count   receives C (exact)
 *   h_estimate       optional: receives C * c^(k-1) (double)
 * Synchronises `stream`.
 */
kc_status kc_count_colorful(const kc_csr *g, int k, uint32_t colors, uint64_t seed, int method,
                            uint64_t *h_sparse_count, double *h_estimate, kc_stream_t stream);

/*
 * kc_peel -- arb-peel (Algorithm 2, Section 4.1): exact k-clique peeling for
 * the k-clique densest subgraph, seeded by arb-count-v. Each round removes
 * every remaining vertex whose current k-clique count (in the graph induced
 * by the remaining vertices) is the minimum; Update counts the k-cliques
 * that the round removes (a clique with several vertices of the round is
 * counted at the lowest-ranked of them) and lowers the counts of the
 * remaining vertices. The result is the largest density (k-cliques per
 * vertex) among the graph itself and what remains after each round; the
 * paper proves it is at least 1/k of the k-clique densest subgraph's.
 *   g        the CSR d was oriented from (the undirected neighbour lists are
 *            read during the call)
 *   d        kc_orient(g, ...) (either method; the result does not depend
 *            on it)
 *   k        3 .. KC_KMAX
 *   d_round  device uint32[n], caller-owned: the round in which each vertex
 *            is removed (0-based)
 *   out      rounds: number of rounds; best_cliques / best_vertices: the best
 *            density as an exact fraction, reached by the vertices removed
 *            in rounds >= best_rounds (best_rounds = 0: the whole graph);
 *            total: k-cliques of the whole graph
 * Synchronises `stream` every round. KC_EINVAL if g and d differ in size;
 * KC_ECAPACITY if a vertex is removed while more than KC_MAX_OUT_DEGREE of
 * its neighbours remain (its candidate row exceeds the counting kernels'
 * root capacity).
 */
typedef struct {
  uint32_t rounds;
  uint32_t best_rounds;
  uint64_t best_cliques;
  uint64_t best_vertices;
  uint64_t total;
} kc_peel_result;
kc_status kc_peel(const kc_csr *g, const kc_dag *d, int k, uint32_t *d_round, kc_peel_result *out,
                  kc_stream_t stream);

/*
 * kc_peel_approx -- arb-approx-peel (Section 4.2): like kc_peel, but each
 * round removes every remaining vertex whose count is at most
 * floor(k (1 + eps) t / |S|) (t the k-cliques of the remaining set S,
 * computed exactly in integers), which takes O(log n) rounds for eps > 0 and
 * gives a 1/(k(1+eps))-approximation (Tsourakakis; Theorem of Section 4.2).
 *   eps_num / eps_den  eps as a fraction (eps_den > 0)
 * Other arguments and the result as for kc_peel.
 */
kc_status kc_peel_approx(const kc_csr *g, const kc_dag *d, int k, uint32_t eps_num, uint32_t eps_den,
                         uint32_t *d_round, kc_peel_result *out, kc_stream_t stream);

/*
 * Work statistics of an oriented graph, used for the bytes a counting pass
 * must move (computed exactly on the device):
 *   sum_out_sq     sum over roots u of d+(u)^2
 *   sum_arc_head   sum over arcs u->v of d+(v) (adjacency read to build the
 *                  first-level induced subgraphs of Section 3.4)
 *   triangles      number of 3-cliques
 *   max_out        largest out-degree
 *   core_vertices  vertices in the dense core (kc_orient), 0 if none
 *   build_scanned  out-list entries those builds scan under the current
 *                  dense-core rule (kc_set_core_policy); sum_arc_head without
 *                  a core
 *   build_lookups  dense-core bits they look up instead (one 64-bit word read
 *                  each); 0 without a core
 */
typedef struct {
  uint64_t sum_out_sq;
  uint64_t sum_arc_head;
  uint64_t triangles;
  uint32_t max_out;
  uint32_t core_vertices;
  uint64_t build_scanned;
  uint64_t build_lookups;
} kc_dag_stats;
kc_status kc_dag_get_stats(const kc_dag *d, kc_dag_stats *h_stats, kc_stream_t stream);

/*
 * kc_checked_sum -- the counting kernels' wrap-checked 64-bit reduction
 * (thread sums, then the block epilogue every counting kernel ends with: warp
 * butterfly, the warps' sums added in the block, one atomic per block)
 * applied to d_values
 * (device uint64[n]): *h_total = their sum, or KC_ERANGE if the sum does not
 * fit in uint64. (The paper has no counterpart: counts large enough to wrap
 * cannot be enumerated in test time, so this exercises the overflow path.)
 * Synchronises `stream`.
 */
kc_status kc_checked_sum(const uint64_t *d_values, uint64_t n, uint64_t *h_total, kc_stream_t stream);

/*
 * Measured rate of the counting kernels' unit of integer work on the current
 * device: one 64-bit AND followed by a population count (the bitset form of
 * the intersect of Algorithm 1). Used as the roofline peak of the counting
 * passes for k >= 5, which are bound by this work. Runs a short calibration
 * kernel (about 10 ms) on `stream` and synchronises it.
 *   h_rate  receives word operations per second
 */
kc_status kc_measure_word_op_rate(double *h_rate, kc_stream_t stream);

/* Number of CUDA kernels this library has launched in this process so far
 * (all entry points, all devices). For accounting in benchmarks. */
uint64_t kc_kernel_launches(void);

/*
 * Process-wide choice of how the counting kernels read the members'
 * out-lists when they build a block root's induced subgraph (the level-2
 * build of Section 3.4): enabled != 0 stages them through shared memory with
 * 1-D bulk copies (cp.async.bulk, two buffers per warp), enabled == 0 (the
 * default) reads them with ordinary loads, eight in flight per lane, which
 * measured faster on the GB300. Counts are identical either way; this is a
 * tunable for measurement. Applies to passes planned after the call.
 */
void kc_set_bulk_build(int enabled);

/*
 * Host-side fault injection for tests (the paper has no counterpart): after
 * `count` more successful stream-ordered device allocations, every further
 * one made by this library fails as an out-of-memory error, without calling
 * CUDA, so that the entry points' KC_ENOMEM paths (and the release of what
 * they had allocated) can be exercised without exhausting a GPU. count < 0
 * switches the injection off. Process-wide; for tests only.
 */
void kc_debug_fail_allocations_after(int64_t count);

/* Human-readable text for a status code (static storage). */
const char *kc_strerror(int status);
/* Text of the last CUDA error seen by this host thread (static per thread). */
const char *kc_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KCLIQUE_H */
