/*
 * CPU ORACLE for exact k-clique counting -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the slow, obviously correct reference that the CUDA path is
 * checked against. Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it; the library itself never does. It shares no code,
 * header, table or helper with the CUDA path.
 *
 * What it computes (Shi, Dhulipala, Shun, "Parallel Clique Counting and
 * Peeling Algorithms"):
 *   - a k-clique is a set of k vertices with all k(k-1)/2 edges present
 *     (Section 2, "Graph Notation");
 *   - the count is obtained by orienting the graph along a total order and
 *     running the recursion Rec-Count-Cliques of Algorithm 1 from every vertex,
 *     with sorted-list intersections for `intersect` (Section 3.2);
 *   - the per-vertex count of v is the number of k-cliques that contain v, the
 *     array C that seeds the peeling of Algorithm 2 (Section 3.2, "-v"
 *     variants; Section 4.1);
 *   - orderings: non-decreasing degree, the k-core (Matula-Beck) order, the
 *     original ids, and the Goodrich-Pszona rounds of Algorithm 3 with
 *     epsilon = 1 (Section 3.1, Section 5 "Algorithm Implementations").
 *
 * Counts are summed in unsigned 128-bit integers and reported as an overflow
 * error when they do not fit in 64 bits. Per-vertex counts check every add.
 *
 * Status codes returned by every routine: 0 ok, 1 invalid argument,
 * 2 overflow of uint64, 3 out of memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

enum { OR_OK = 0, OR_EINVAL = 1, OR_ERANGE = 2, OR_ENOMEM = 3 };

/* ------------------------------------------------------------ orderings */

typedef struct { uint64_t a, b, c; uint32_t v; } okey;

static int okey_cmp(const void *x, const void *y) {
  const okey *p = (const okey *)x, *q = (const okey *)y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  if (p->c != q->c) return p->c < q->c ? -1 : 1;
  if (p->v != q->v) return p->v < q->v ? -1 : 1;
  return 0;
}

/* Degree ordering: vertices by non-decreasing degree, ties by id.
 * rank[v] = position of v in that order (Section 5, degree ordering). */
int or_rank_degree(uint32_t n, const uint64_t *row_ptr, uint32_t *rank) {
  okey *keys = (okey *)malloc(sizeof(okey) * (n ? n : 1));
  if (!keys) return OR_ENOMEM;
  for (uint32_t v = 0; v < n; v++) {
    keys[v].a = row_ptr[v + 1] - row_ptr[v]; keys[v].b = 0; keys[v].c = 0; keys[v].v = v;
  }
  qsort(keys, n, sizeof(okey), okey_cmp);
  for (uint32_t i = 0; i < n; i++) rank[keys[i].v] = i;
  free(keys);
  return OR_OK;
}

/* Binary min-heap of 64-bit keys (the degeneracy order's priority queue). */
static void heap_push(uint64_t *h, size_t *len, uint64_t x) {
  size_t i = (*len)++;
  while (i > 0) {
    size_t p = (i - 1) / 2;
    if (h[p] <= x) break;
    h[i] = h[p];
    i = p;
  }
  h[i] = x;
}

static uint64_t heap_pop(uint64_t *h, size_t *len) {
  uint64_t top = h[0], x = h[--(*len)];
  size_t i = 0;
  for (;;) {
    size_t c = 2 * i + 1;
    if (c >= *len) break;
    if (c + 1 < *len && h[c + 1] < h[c]) c++;
    if (x <= h[c]) break;
    h[i] = h[c];
    i = c;
  }
  if (*len) h[i] = x;
  return top;
}

/* k-core (degeneracy) ordering, smallest-last as Matula and Beck define it:
 * repeatedly remove the vertex of minimum degree in the graph induced by the
 * vertices not yet removed, ties broken by the smaller id; rank = removal
 * position. The queue holds (degree << 32 | id) keys; a vertex whose degree
 * drops is pushed again with its new key, and popped keys that no longer
 * match a live vertex's degree are skipped. */
int or_rank_degeneracy(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, uint32_t *rank) {
  if (n == 0) return OR_OK;
  size_t cap = (size_t)n + (size_t)row_ptr[n] + 1, len = 0;
  uint32_t *deg = (uint32_t *)malloc(sizeof(uint32_t) * n);
  uint8_t *gone = (uint8_t *)calloc(n, 1);
  uint64_t *heap = (uint64_t *)malloc(sizeof(uint64_t) * cap);
  if (!deg || !gone || !heap) { free(deg); free(gone); free(heap); return OR_ENOMEM; }
  for (uint32_t v = 0; v < n; v++) {
    deg[v] = (uint32_t)(row_ptr[v + 1] - row_ptr[v]);
    heap_push(heap, &len, ((uint64_t)deg[v] << 32) | v);
  }
  uint32_t removed = 0;
  while (removed < n) {
    uint64_t key = heap_pop(heap, &len);
    uint32_t v = (uint32_t)key;
    if (gone[v] || (uint32_t)(key >> 32) != deg[v]) continue;  /* stale entry */
    gone[v] = 1;
    rank[v] = removed++;
    for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
      uint32_t u = col[e];
      if (!gone[u]) {
        deg[u]--;
        heap_push(heap, &len, ((uint64_t)deg[u] << 32) | u);
      }
    }
  }
  free(deg); free(gone); free(heap);
  return OR_OK;
}

/* Goodrich-Pszona orientation, Algorithm 3 with epsilon = 1. Reading taken:
 * each round removes ceil(n'/3) of the n' remaining vertices (the
 * epsilon/(2+epsilon) fraction applied to what remains, so the loop takes
 * O(log n) rounds as Section 3.1 states), namely those smallest by
 * (induced degree, id); within a round the appended vertices keep that order.
 * rank[v] = position in the final list L; round_out[v] and deg_out[v] (may be
 * NULL) receive the round in which v was removed and its induced degree then. */
int or_rank_gp(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, uint32_t *rank,
               uint32_t *round_out, uint32_t *deg_out) {
  uint32_t *deg = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  uint8_t *gone = (uint8_t *)calloc(n ? n : 1, 1);
  okey *keys = (okey *)malloc(sizeof(okey) * (n ? n : 1));
  if (!deg || !gone || !keys) { free(deg); free(gone); free(keys); return OR_ENOMEM; }
  for (uint32_t v = 0; v < n; v++) deg[v] = (uint32_t)(row_ptr[v + 1] - row_ptr[v]);
  uint32_t remaining = n, pos = 0, round = 0;
  while (remaining > 0) {
    uint32_t cnt = 0;
    for (uint32_t v = 0; v < n; v++)
      if (!gone[v]) { keys[cnt].a = deg[v]; keys[cnt].b = 0; keys[cnt].c = 0; keys[cnt].v = v; cnt++; }
    qsort(keys, cnt, sizeof(okey), okey_cmp);
    uint32_t take = (remaining + 2) / 3; /* ceil(n'/3), at least 1 */
    for (uint32_t i = 0; i < take; i++) {
      uint32_t v = keys[i].v;
      rank[v] = pos++;
      if (round_out) round_out[v] = round;
      if (deg_out) deg_out[v] = deg[v];
      gone[v] = 1;
    }
    for (uint32_t i = 0; i < take; i++) {
      uint32_t v = keys[i].v;
      for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; e++)
        if (!gone[col[e]]) deg[col[e]]--;
    }
    remaining -= take;
    round++;
  }
  free(deg); free(gone); free(keys);
  return OR_OK;
}

/* Direct the graph along a total order: keep arc u->v iff rank[u] < rank[v]
 * (out-neighbours are the neighbours higher in the order, Section 2). Each
 * out-list keeps the ascending-id order of the input row (a filter preserves
 * order, Section 2 "Parallel Primitives"). dag_col needs room for nnz/2.
 * Returns the number of arcs kept. */
int64_t or_direct(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *rank,
                  uint64_t *dag_ptr, uint32_t *dag_col) {
  uint64_t w = 0;
  for (uint32_t u = 0; u < n; u++) {
    dag_ptr[u] = w;
    for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; e++)
      if (rank[u] < rank[col[e]]) dag_col[w++] = col[e];
  }
  dag_ptr[n] = w;
  return (int64_t)w;
}

/* ------------------------------------------------------------- counting */

typedef struct {
  const uint64_t *ptr;
  const uint32_t *adj;
  uint32_t **buf;   /* buf[l]: room for the candidate set of level l */
  uint32_t *path;   /* vertices added so far (per-vertex mode) */
  int depth;
  uint64_t *pv;     /* per-vertex counts, or NULL */
  int ovf;
} rc_ctx;

/* |A ∩ B| into out (sorted merge of two ascending lists) */
static size_t intersect(const uint32_t *a, size_t na, const uint32_t *b, size_t nb, uint32_t *out) {
  size_t i = 0, j = 0, c = 0;
  while (i < na && j < nb) {
    if (a[i] < b[j]) i++;
    else if (a[i] > b[j]) j++;
    else { out[c++] = a[i]; i++; j++; }
  }
  return c;
}

static inline void pv_add(rc_ctx *cx, uint32_t v, uint64_t x) {
  uint64_t old = cx->pv[v];
  cx->pv[v] = old + x;
  if (cx->pv[v] < old) cx->ovf = 1;
}

/* Rec-Count-Cliques(DG, I, l) of Algorithm 1: if l = 1 the candidates each
 * complete a clique; otherwise add each v in I, intersect I with N+(v) and
 * recurse with l-1, summing the results. In per-vertex mode a completed
 * clique (path + one member of I) credits every path vertex and that member. */
static u128 rec_count(rc_ctx *cx, const uint32_t *I, size_t nI, int l) {
  if (l == 1) {
    if (cx->pv) {
      for (int p = 0; p < cx->depth; p++) pv_add(cx, cx->path[p], (uint64_t)nI);
      for (size_t i = 0; i < nI; i++) pv_add(cx, I[i], 1);
    }
    return (u128)nI;
  }
  u128 t = 0;
  uint32_t *next = cx->buf[l - 1];
  for (size_t i = 0; i < nI; i++) {
    uint32_t v = I[i];
    const uint32_t *nv = cx->adj + cx->ptr[v];
    size_t dv = (size_t)(cx->ptr[v + 1] - cx->ptr[v]);
    size_t c = intersect(I, nI, nv, dv, next);
    if (cx->pv) cx->path[cx->depth++] = v;
    t += rec_count(cx, next, c, l - 1);
    if (cx->pv) cx->depth--;
  }
  return t;
}

static int ctx_init(rc_ctx *cx, uint32_t n, const uint64_t *ptr, const uint32_t *adj, int k, uint64_t *pv) {
  uint64_t maxd = 0;
  for (uint32_t v = 0; v < n; v++) if (ptr[v + 1] - ptr[v] > maxd) maxd = ptr[v + 1] - ptr[v];
  cx->ptr = ptr; cx->adj = adj; cx->pv = pv; cx->ovf = 0; cx->depth = 0;
  cx->buf = (uint32_t **)calloc((size_t)k + 1, sizeof(uint32_t *));
  cx->path = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)k + 1));
  if (!cx->buf || !cx->path) return OR_ENOMEM;
  for (int l = 0; l <= k; l++) {
    cx->buf[l] = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(maxd + 1));
    if (!cx->buf[l]) return OR_ENOMEM;
  }
  return OR_OK;
}

static void ctx_free(rc_ctx *cx, int k) {
  if (cx->buf) for (int l = 0; l <= k; l++) free(cx->buf[l]);
  free(cx->buf); free(cx->path);
}

/* arb-count restricted to roots in [lo, hi): the top call of Algorithm 1 with
 * I = V adds each root v and recurses on N+(v) with k-1 vertices left; for
 * k = 1 every root is itself a clique. The 128-bit sum is returned as
 * (lo64, hi64); pv (NULL, or n entries, accumulated into) receives per-vertex
 * counts. */
int or_count(uint32_t n, const uint64_t *dag_ptr, const uint32_t *dag_col, int k,
             uint32_t lo, uint32_t hi, uint64_t *sum_lo, uint64_t *sum_hi, uint64_t *pv) {
  if (k < 1 || hi > n || lo > hi) return OR_EINVAL;
  rc_ctx cx;
  memset(&cx, 0, sizeof cx);
  if (ctx_init(&cx, n, dag_ptr, dag_col, k, pv)) { ctx_free(&cx, k); return OR_ENOMEM; }
  u128 t = 0;
  if (k == 1) {
    t = (u128)(hi - lo);
    if (pv) for (uint32_t v = lo; v < hi; v++) pv_add(&cx, v, 1);
  } else {
    for (uint32_t v = lo; v < hi; v++) {
      const uint32_t *nv = dag_col + dag_ptr[v];
      size_t dv = (size_t)(dag_ptr[v + 1] - dag_ptr[v]);
      if (pv) cx.path[cx.depth++] = v;
      t += rec_count(&cx, nv, dv, k - 1);
      if (pv) cx.depth--;
    }
  }
  int ovf = cx.ovf;
  ctx_free(&cx, k);
  *sum_lo = (uint64_t)t;
  *sum_hi = (uint64_t)(t >> 64);
  return ovf ? OR_ERANGE : OR_OK;
}

/* Number of k-cliques whose two lowest vertices in the order are the arc
 * u->v: Rec-Count-Cliques on N+(u) ∩ N+(v) with k-2 vertices left (k >= 3);
 * 1 for k = 2. The arc must exist. */
int or_count_arc(uint32_t n, const uint64_t *dag_ptr, const uint32_t *dag_col, int k,
                 uint32_t u, uint32_t v, uint64_t *sum_lo, uint64_t *sum_hi) {
  if (k < 2 || u >= n || v >= n) return OR_EINVAL;
  if (k == 2) { *sum_lo = 1; *sum_hi = 0; return OR_OK; }
  rc_ctx cx;
  memset(&cx, 0, sizeof cx);
  if (ctx_init(&cx, n, dag_ptr, dag_col, k, NULL)) { ctx_free(&cx, k); return OR_ENOMEM; }
  uint32_t *i2 = cx.buf[k];
  size_t s = intersect(dag_col + dag_ptr[u], (size_t)(dag_ptr[u + 1] - dag_ptr[u]),
                       dag_col + dag_ptr[v], (size_t)(dag_ptr[v + 1] - dag_ptr[v]), i2);
  u128 t = rec_count(&cx, i2, s, k - 2);
  ctx_free(&cx, k);
  *sum_lo = (uint64_t)t;
  *sum_hi = (uint64_t)(t >> 64);
  return OR_OK;
}

/* ---------------------------------------------------------- brute force */

/* Every k-subset of [0, n) in lexicographic order, counted when all pairs are
 * adjacent in the dense 0/1 matrix adj (row-major n x n). Definition of a
 * k-clique, nothing more; meant for n <= ~30. pv (NULL or n entries) gets the
 * number of k-cliques containing each vertex. */
int or_brute(uint32_t n, const uint8_t *adj, int k, uint64_t *total, uint64_t *pv) {
  if (k < 1 || (uint32_t)k > n) { *total = 0; if (pv) memset(pv, 0, sizeof(uint64_t) * n); return k < 1 ? OR_EINVAL : OR_OK; }
  uint32_t *s = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)k);
  if (!s) return OR_ENOMEM;
  if (pv) memset(pv, 0, sizeof(uint64_t) * n);
  for (int i = 0; i < k; i++) s[i] = (uint32_t)i;
  uint64_t cnt = 0;
  for (;;) {
    int ok = 1;
    for (int i = 0; i < k && ok; i++)
      for (int j = i + 1; j < k; j++)
        if (!adj[(size_t)s[i] * n + s[j]]) { ok = 0; break; }
    if (ok) { cnt++; if (pv) for (int i = 0; i < k; i++) pv[s[i]]++; }
    int i = k - 1;
    while (i >= 0 && s[i] == n - (uint32_t)(k - i)) i--;
    if (i < 0) break;
    s[i]++;
    for (int j = i + 1; j < k; j++) s[j] = s[j - 1] + 1;
  }
  free(s);
  *total = cnt;
  return OR_OK;
}
