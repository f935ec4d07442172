/*
 * Seeded synthetic graph generators: the input side shared by the CUDA path
 * and the CPU oracle. Nothing here counts cliques or orients a graph; this file
 * only draws edge lists and turns them into a simple undirected CSR.
 *
 * Determinism: all randomness comes from a counter-based splitmix64 stream
 * keyed by (seed, stream), and all floating point is made of IEEE basic
 * operations (+, -, *, /, frexp, ldexp) with contraction disabled at build
 * time, so the same seed gives the same graph on x86-64 and aarch64. The
 * logarithm and exponential are local series evaluations for that reason,
 * not libm calls.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- RNG ---- */
static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
  return mix64(mix64(seed + 0x9E3779B97F4A7C15ULL) ^ (stream * 0xD1B54A32D192ED03ULL + 0x632BE59BD9B4E019ULL));
}
/* splitmix64 output number `ctr` of the stream with state origin `key` */
static inline uint64_t rnd(uint64_t key, uint64_t ctr) {
  return mix64(key + (ctr + 1) * 0x9E3779B97F4A7C15ULL);
}
/* uniform in [0, bound) by the multiply-high method */
static inline uint64_t rnd_below(uint64_t key, uint64_t ctr, uint64_t bound) {
  return (uint64_t)(((u128)rnd(key, ctr) * (u128)bound) >> 64);
}
/* uniform double in (0, 1] with 53 random bits */
static inline double rnd_unit_open0(uint64_t key, uint64_t ctr) {
  return ((double)(rnd(key, ctr) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

/* -------------------------------------------- deterministic log / exp ---- */
static const double LN2 = 0.69314718055994530942;
/* natural log for x > 0: x = m 2^e, m in [sqrt(1/2), sqrt(2)), then
 * log m = 2 atanh(z), z = (m-1)/(m+1), summed as an odd power series. */
static double dlog(double x) {
  int e;
  double m = frexp(x, &e); /* m in [0.5, 1) */
  if (m < 0.70710678118654752440) { m = m * 2.0; e -= 1; }
  double z = (m - 1.0) / (m + 1.0);
  double z2 = z * z, term = z, sum = 0.0;
  for (int k = 1; k <= 41; k += 2) { sum = sum + term / (double)k; term = term * z2; }
  return 2.0 * sum + (double)e * LN2;
}
/* exp(y): y = q ln2 + r with |r| <= ln2/2, Taylor series for exp(r) */
static double dexp(double y) {
  double qf = floor(y / LN2 + 0.5);
  int q = (int)qf;
  double r = y - qf * LN2;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k <= 24; k++) { term = term * r / (double)k; sum = sum + term; }
  return ldexp(sum, q);
}

double gg_dlog(double x) { return dlog(x); }
double gg_dexp(double y) { return dexp(y); }

/* ------------------------------------------------------ Erdos-Renyi ---- */
/* G(n, p) by geometric skipping over the n(n-1)/2 pairs (i > j) in the order
 * (1,0), (2,0), (2,1), (3,0), ... Writes each sampled pair once. Returns the
 * pair count, or -(needed lower bound) if cap is too small. */
int64_t gg_er(uint32_t n, double p, uint64_t seed, uint32_t *eu, uint32_t *ev, int64_t cap) {
  if (n < 2 || p <= 0.0) return 0;
  uint64_t key = stream_key(seed, 1);
  int64_t cnt = 0;
  uint64_t ctr = 0;
  if (p >= 1.0) {
    for (uint64_t i = 1; i < n; i++)
      for (uint64_t j = 0; j < i; j++) {
        if (cnt < cap) { eu[cnt] = (uint32_t)i; ev[cnt] = (uint32_t)j; }
        cnt++;
      }
    return cnt <= cap ? cnt : -cnt;
  }
  double lq = dlog(1.0 - p);
  /* linear pair index t in [0, N); row i holds indices [i(i-1)/2, i(i+1)/2) */
  uint64_t N = (uint64_t)n * (uint64_t)(n - 1) / 2;
  uint64_t t = 0;
  uint64_t i = 1, row_lo = 0; /* row_lo = i(i-1)/2 */
  int first = 1;
  for (;;) {
    double u = rnd_unit_open0(key, ctr++);
    double sk = floor(dlog(u) / lq);
    if (sk >= (double)N) break;
    uint64_t skip = (uint64_t)sk;
    if (first) { t = skip; first = 0; }
    else { if (t + 1 + skip < t) break; t = t + 1 + skip; }
    if (t >= N) break;
    while (t >= row_lo + i) { row_lo += i; i++; }
    if (cnt < cap) { eu[cnt] = (uint32_t)i; ev[cnt] = (uint32_t)(t - row_lo); }
    cnt++;
  }
  return cnt <= cap ? cnt : -cnt;
}

/* ------------------------------------------------------------ R-MAT ---- */
/* nedges samples of the recursive matrix with quadrant probabilities
 * (a, b, c, 1-a-b-c), then the vertex ids are relabelled by a seeded
 * permutation when permute != 0. Self-loops and duplicates are kept here; the
 * CSR builder drops them. */
static void *rmat_worker(void *arg);
typedef struct {
  int scale; uint64_t lo, hi; uint64_t key; uint64_t ta, tab, tabc;
  const uint32_t *perm; uint32_t *eu, *ev;
} rmat_job;

static void *rmat_worker(void *arg) {
  rmat_job *jb = (rmat_job *)arg;
  for (uint64_t e = jb->lo; e < jb->hi; e++) {
    uint32_t u = 0, v = 0;
    for (int l = 0; l < jb->scale; l++) {
      uint64_t r = rnd(jb->key, e * 64 + (uint64_t)l) >> 11;
      uint32_t bu, bv;
      if (r < jb->ta) { bu = 0; bv = 0; }
      else if (r < jb->tab) { bu = 0; bv = 1; }
      else if (r < jb->tabc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u = (u << 1) | bu; v = (v << 1) | bv;
    }
    if (jb->perm) { u = jb->perm[u]; v = jb->perm[v]; }
    jb->eu[e] = u; jb->ev[e] = v;
  }
  return NULL;
}

/* seeded Fisher-Yates permutation of [0, n) */
void gg_permutation(uint32_t n, uint64_t seed, uint64_t stream, uint32_t *perm) {
  uint64_t key = stream_key(seed, stream);
  for (uint32_t i = 0; i < n; i++) perm[i] = i;
  for (uint64_t i = n; i > 1; i--) {
    uint64_t j = rnd_below(key, i, i);
    uint32_t tmp = perm[i - 1]; perm[i - 1] = perm[j]; perm[j] = tmp;
  }
}

static int clamp_threads(int nthreads) { return nthreads < 1 ? 1 : (nthreads > 256 ? 256 : nthreads); }

int gg_rmat(int scale, uint64_t nedges, double a, double b, double c, uint64_t seed,
            int permute, uint32_t *eu, uint32_t *ev, int nthreads) {
  if (scale < 1 || scale > 31) return -1;
  uint32_t n = 1u << scale;
  uint32_t *perm = NULL;
  if (permute) {
    perm = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    if (!perm) return -2;
    gg_permutation(n, seed, 3, perm);
  }
  const double two53 = 9007199254740992.0;
  rmat_job base;
  base.scale = scale; base.key = stream_key(seed, 2);
  base.ta = (uint64_t)(a * two53); base.tab = (uint64_t)((a + b) * two53);
  base.tabc = (uint64_t)((a + b + c) * two53);
  base.perm = perm; base.eu = eu; base.ev = ev;
  nthreads = clamp_threads(nthreads);
  pthread_t th[256]; rmat_job jobs[256];
  for (int t = 0; t < nthreads; t++) {
    jobs[t] = base;
    jobs[t].lo = nedges * (uint64_t)t / (uint64_t)nthreads;
    jobs[t].hi = nedges * (uint64_t)(t + 1) / (uint64_t)nthreads;
    pthread_create(&th[t], NULL, rmat_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
  free(perm);
  return 0;
}

/* -------------------------------------------------- Barabasi-Albert ---- */
/* Seed clique on m0+1 vertices, then every later vertex attaches m0 distinct
 * edges to targets drawn uniformly from the endpoint list of the edges so far
 * (degree-proportional). Returns the edge count; eu/ev need room for
 * m0(m0+1)/2 + (n-m0-1) m0 pairs (all of n's pairs when n <= m0+1). */
int64_t gg_ba(uint32_t n, uint32_t m0, uint64_t seed, uint32_t *eu, uint32_t *ev) {
  if (n == 0) return 0;
  if (m0 < 1) m0 = 1;
  uint64_t key = stream_key(seed, 4);
  uint32_t core = m0 + 1 < n ? m0 + 1 : n;
  int64_t cnt = 0;
  for (uint32_t i = 1; i < core; i++)
    for (uint32_t j = 0; j < i; j++) { eu[cnt] = i; ev[cnt] = j; cnt++; }
  if (core == n) return cnt;
  uint64_t cap_end = 2 * ((uint64_t)cnt + (uint64_t)(n - core) * m0);
  uint32_t *endp = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)cap_end);
  uint32_t *pick = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m0);
  if (!endp || !pick) { free(endp); free(pick); return -1; }
  uint64_t ne = 0;
  for (int64_t e = 0; e < cnt; e++) { endp[ne++] = eu[e]; endp[ne++] = ev[e]; }
  uint64_t ctr = 0;
  for (uint32_t v = core; v < n; v++) {
    uint32_t got = 0;
    while (got < m0) {
      uint32_t t = endp[rnd_below(key, ctr++, ne)];
      int dup = 0;
      for (uint32_t q = 0; q < got; q++) if (pick[q] == t) { dup = 1; break; }
      if (!dup) pick[got++] = t;
    }
    for (uint32_t q = 0; q < m0; q++) {
      eu[cnt] = v; ev[cnt] = pick[q]; cnt++;
      endp[ne++] = v; endp[ne++] = pick[q];
    }
  }
  free(endp); free(pick);
  return cnt;
}

/* ----------------------------------------------- Chung-Lu + planted ---- */
/* Expected-degree (Chung-Lu) graph: weights w_i = (i + i0)^(-1/(gamma-1))
 * scaled to mean `mean_deg`, each capped at sqrt(sum w); then npairs endpoint
 * pairs are drawn independently proportional to w (Vose alias table).
 * Returns 0, or a negative code on allocation failure. */
typedef struct {
  uint64_t lo, hi, key; uint32_t n; const double *prob; const uint32_t *alias;
  uint32_t *eu, *ev;
} cl_job;

static inline uint32_t alias_draw(const cl_job *jb, uint64_t ctr) {
  uint64_t r = rnd(jb->key, ctr);
  uint32_t col = (uint32_t)(((u128)r * (u128)jb->n) >> 64);
  double u = (double)(rnd(jb->key ^ 0x5555555555555555ULL, ctr) >> 11) * (1.0 / 9007199254740992.0);
  return u < jb->prob[col] ? col : jb->alias[col];
}
static void *cl_worker(void *arg) {
  cl_job *jb = (cl_job *)arg;
  for (uint64_t e = jb->lo; e < jb->hi; e++) {
    jb->eu[e] = alias_draw(jb, 2 * e);
    jb->ev[e] = alias_draw(jb, 2 * e + 1);
  }
  return NULL;
}

int gg_chung_lu(uint32_t n, double gamma, double mean_deg, double i0, uint64_t seed,
                uint64_t npairs, uint32_t *eu, uint32_t *ev, double *weights_out, int nthreads) {
  double *w = weights_out ? weights_out : (double *)malloc(sizeof(double) * (size_t)n);
  double *prob = (double *)malloc(sizeof(double) * (size_t)n);
  uint32_t *alias = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  uint32_t *small = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  uint32_t *large = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  if (!w || !prob || !alias || !small || !large) return -1;
  double expo = -1.0 / (gamma - 1.0), sum = 0.0;
  for (uint32_t i = 0; i < n; i++) { w[i] = dexp(expo * dlog((double)i + i0)); sum = sum + w[i]; }
  double scale = mean_deg * (double)n / sum;
  sum = 0.0;
  for (uint32_t i = 0; i < n; i++) { w[i] = w[i] * scale; sum = sum + w[i]; }
  double cap = sqrt(sum); /* sqrt is correctly rounded in IEEE 754 */
  sum = 0.0;
  for (uint32_t i = 0; i < n; i++) { if (w[i] > cap) w[i] = cap; sum = sum + w[i]; }
  /* Vose alias table over p_i = w_i / sum */
  uint32_t ns = 0, nl = 0;
  for (uint32_t i = 0; i < n; i++) {
    prob[i] = w[i] * (double)n / sum;
    if (prob[i] < 1.0) small[ns++] = i; else large[nl++] = i;
  }
  while (ns && nl) {
    uint32_t s = small[--ns], l = large[--nl];
    alias[s] = l;
    prob[l] = (prob[l] + prob[s]) - 1.0;
    if (prob[l] < 1.0) small[ns++] = l; else large[nl++] = l;
  }
  while (nl) { uint32_t l = large[--nl]; prob[l] = 1.0; alias[l] = l; }
  while (ns) { uint32_t s = small[--ns]; prob[s] = 1.0; alias[s] = s; }
  free(small); free(large);
  nthreads = clamp_threads(nthreads);
  pthread_t th[256]; cl_job jobs[256];
  for (int t = 0; t < nthreads; t++) {
    jobs[t].lo = npairs * (uint64_t)t / (uint64_t)nthreads;
    jobs[t].hi = npairs * (uint64_t)(t + 1) / (uint64_t)nthreads;
    jobs[t].key = stream_key(seed, 5); jobs[t].n = n; jobs[t].prob = prob; jobs[t].alias = alias;
    jobs[t].eu = eu; jobs[t].ev = ev;
    pthread_create(&th[t], NULL, cl_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
  free(prob); free(alias);
  if (!weights_out) free(w);
  return 0;
}

/* `count` cliques with sizes uniform in [smin, smax], each on a uniformly random
 * set of distinct vertices (rejection inside one clique). Writes the sizes to
 * sizes_out and the member lists, concatenated, to members_out (room for
 * count * smax). Returns the member total. */
int64_t gg_planted_sets(uint32_t n, uint32_t count, uint32_t smin, uint32_t smax, uint64_t seed,
                        uint32_t *sizes_out, uint32_t *members_out) {
  uint64_t key = stream_key(seed, 6);
  uint64_t ctr = 0;
  int64_t tot = 0;
  for (uint32_t c = 0; c < count; c++) {
    uint32_t s = smin + (uint32_t)rnd_below(key, ctr++, (uint64_t)(smax - smin + 1));
    if (s > n) s = n;
    sizes_out[c] = s;
    uint32_t *mem = members_out + tot;
    uint32_t got = 0;
    while (got < s) {
      uint32_t x = (uint32_t)rnd_below(key, ctr++, n);
      int dup = 0;
      for (uint32_t q = 0; q < got; q++) if (mem[q] == x) { dup = 1; break; }
      if (!dup) mem[got++] = x;
    }
    tot += s;
  }
  return tot;
}

/* ---------------------------------------------------------- CSR build ---- */
/* Symmetrise the pair list, drop self-loops, sort every row ascending and
 * drop duplicates. row_ptr has n+1 entries; col needs room for 2*ne entries.
 * Two stable counting sorts (by destination, then by source) give sorted rows
 * in O(n + ne). Returns nnz (the number of directed arcs kept), or -1. */
int64_t gg_csr(uint32_t n, uint64_t ne, const uint32_t *eu, const uint32_t *ev,
               uint64_t *row_ptr, uint32_t *col) {
  uint64_t na = 0;
  uint64_t *cnt = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
  if (!cnt) return -1;
  for (uint64_t e = 0; e < ne; e++) if (eu[e] != ev[e]) { cnt[eu[e]]++; cnt[ev[e]]++; na += 2; }
  uint32_t *src = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(na ? na : 1));
  uint32_t *dst = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(na ? na : 1));
  uint64_t *pos = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
  if (!src || !dst || !pos) { free(cnt); free(src); free(dst); free(pos); return -1; }
  /* pass 1: bucket by destination (cnt[x] = in-degree = out-degree, symmetric) */
  uint64_t acc = 0;
  for (uint32_t x = 0; x < n; x++) { pos[x] = acc; acc += cnt[x]; }
  for (uint64_t e = 0; e < ne; e++) {
    uint32_t a = eu[e], b = ev[e];
    if (a == b) continue;
    uint64_t p = pos[b]++; src[p] = a; dst[p] = b;
    p = pos[a]++; src[p] = b; dst[p] = a;
  }
  /* pass 2: stable bucket by source; rows come out sorted by destination */
  acc = 0;
  for (uint32_t x = 0; x < n; x++) { pos[x] = acc; acc += cnt[x]; }
  for (uint64_t i = 0; i < na; i++) { uint64_t p = pos[src[i]]++; col[p] = dst[i]; }
  free(src); free(dst);
  /* dedup in place, row by row */
  uint64_t w = 0, r0 = 0;
  for (uint32_t x = 0; x < n; x++) {
    uint64_t r1 = r0 + cnt[x];
    row_ptr[x] = w;
    for (uint64_t i = r0; i < r1; i++)
      if (i == r0 || col[i] != col[i - 1]) col[w++] = col[i];
    r0 = r1;
  }
  row_ptr[n] = w;
  free(cnt); free(pos);
  return (int64_t)w;
}
