// Counting kernels: arb-count and arb-count-v (Algorithm 1, Section 3.2)
// with the practical optimizations of Section 3.3, laid out for sm_103a.
//
// Work decomposition. Every k-clique is found exactly once, below its lowest
// vertex u in the total order (the root), as a (k-1)-clique of the DAG
// induced on N+(u). For each root the team (one warp for d+(u) <= 64, one
// block otherwise) builds that induced subgraph once -- "the induced subgraph
// on N_DG(v)" of Section 3.3 -- as a bit matrix: row i is the set of
// positions t in N+(u) with N+(u)[t] in N+(N+(u)[i]). Vertices are relabelled
// to their positions 0..d-1 in N+(u) (Section 3.3's relabelling to [0, O(alpha)]).
// The sub-problems below the root are split over lane groups: one item per
// arc u->x_i for k <= 4, one item per triangle u->x_i->x_j for k >= 5 (edge
// parallelism, Section 3.3). An item runs Rec-Count-Cliques on its candidate
// bitset: intersect = word-wise AND, |I| = population count, the base case
// l = 1 folded into the level above (l = 2: sum over x of |C & row_x|).
//
// Per-vertex counts (arb-count-v): a clique found at the l = 2 level with
// candidate set C as (x, y), y in C & row_x, credits x with |C & row_x| and
// y with |C & col_y| (col = transposed matrix), so no per-clique increment
// is made; vertices higher up get the totals of their sub-trees; the root
// gets the root total. Counts are flushed to global memory once per root.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kc_internal.cuh"

namespace kc {

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long add_ck(unsigned long long a, unsigned long long b, unsigned &ovf) {
  const unsigned long long s = a + b;
  ovf |= (s < a) ? ST_OVERFLOW : 0u;
  return s;
}

__device__ __forceinline__ void atomic_add_ck(unsigned long long *p, unsigned long long v, unsigned &ovf) {
  if (v == 0) return;
  const unsigned long long old = atomicAdd(p, v);
  ovf |= (old + v < old) ? ST_OVERFLOW : 0u;
}

// ---------------------------------------------------------- lane groups
template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (G == 32) return 0xffffffffu;
  else return ((1u << G) - 1u) << (lane_id() & ~(unsigned)(G - 1));
}

template <int G>
__device__ __forceinline__ unsigned gsum32(unsigned v, unsigned gm) {
  if constexpr (G == 1) return v;
  else return __reduce_add_sync(gm, v);
}

template <int G>
__device__ __forceinline__ unsigned long long gsum64(unsigned long long v, unsigned gm) {
  if constexpr (G == 1) return v;
#pragma unroll
  for (int o = G / 2; o; o >>= 1) v += __shfl_xor_sync(gm, v, o, G);
  return v;
}

// Next set bit of a group-distributed set (lane j of the group holds words
// r*G + j, r < NW); clears it and returns its position in x.
template <int G, int NW>
__device__ __forceinline__ bool next_bit(uint64_t (&T)[NW], unsigned gm, int j, int &x) {
#pragma unroll
  for (int r = 0; r < NW; ++r) {
    if constexpr (G == 1) {
      if (T[r]) {
        x = r * 64 + __ffsll((long long)T[r]) - 1;
        T[r] &= T[r] - 1;
        return true;
      }
    } else {
      unsigned bal = __ballot_sync(gm, T[r] != 0ull);
      if constexpr (G < 32) bal = (bal >> (lane_id() & ~(unsigned)(G - 1))) & ((1u << G) - 1u);
      if (bal) {
        const int jj = __ffs(bal) - 1;
        const uint64_t w = __shfl_sync(gm, T[r], jj, G);
        x = (r * G + jj) * 64 + __ffsll((long long)w) - 1;
        if (j == jj) T[r] &= T[r] - 1;
        return true;
      }
    }
  }
  return false;
}

// ------------------------------------------------------ per-root storage
struct RootView {
  uint32_t *L;               // N+(u): d ids, ascending
  uint64_t *rows;            // d x RS words
  uint64_t *colT;            // d x RS words (per-vertex only)
  unsigned long long *cnt;   // d per-vertex counters (per-vertex only)
  unsigned long long *asub;  // d per-arc sums (per-arc only)
  uint32_t *pre;             // d+1 pair prefix sums
  uint32_t d, RS;
};

// Same layout and sizes as root_bytes(cap, pv, pa) with RS = row_stride(cap).
__device__ __forceinline__ RootView carve(uint8_t *base, uint32_t cap, uint32_t RS, uint32_t d, bool pv, bool pa) {
  RootView v;
  size_t off = 0;
  v.L = (uint32_t *)(base + off);
  off += align16((size_t)cap * 4);
  v.rows = (uint64_t *)(base + off);
  off += align16((size_t)cap * RS * 8);
  v.colT = nullptr;
  v.cnt = nullptr;
  v.asub = nullptr;
  if (pv) {
    v.colT = (uint64_t *)(base + off);
    off += align16((size_t)cap * RS * 8);
    v.cnt = (unsigned long long *)(base + off);
    off += align16((size_t)cap * 8);
  }
  if (pa) {
    v.asub = (unsigned long long *)(base + off);
    off += align16((size_t)cap * 8);
  }
  v.pre = (uint32_t *)(base + off);
  v.d = d;
  v.RS = RS;
  return v;
}

// Build row i = {t : L[t] in N+(L[i])} (and its transpose) for rows i taken
// by warps warp, warp+nwarps, ...; lanes walk N+(L[i]) and binary-search L.
__device__ __forceinline__ void build_rows(const RootView &R, const uint64_t *__restrict__ ptr,
                                           const uint32_t *__restrict__ col, unsigned warp, unsigned nwarps,
                                           bool pv) {
  const unsigned lane = lane_id();
  const uint32_t d = R.d;
  if (d == 0) return;
  const uint32_t lo_id = R.L[0], hi_id = R.L[d - 1];
  for (uint32_t i = warp; i < d; i += nwarps) {
    const uint32_t x = R.L[i];
    const uint64_t b = ptr[x], e = ptr[x + 1];
    for (uint64_t p = b + lane; p < e; p += 32) {
      const uint32_t y = col[p];
      if (y < lo_id || y > hi_id) continue;
      uint32_t lo = 0, hi = d;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (R.L[mid] < y) lo = mid + 1; else hi = mid;
      }
      if (lo < d && R.L[lo] == y) {
        atomicOr((unsigned long long *)&R.rows[(size_t)i * R.RS + (lo >> 6)], 1ull << (lo & 63));
        if (pv) atomicOr((unsigned long long *)&R.colT[(size_t)lo * R.RS + (i >> 6)], 1ull << (i & 63));
      }
    }
  }
}

// --------------------------------------------------------------- leaves
// l = 2 below candidate set C: sum over x in C of |C & row_x|. With per-vertex
// counts the result is group-uniform and x, y are credited; otherwise each
// lane returns its partial sum.
template <int G, int NW, bool PV>
__device__ __forceinline__ unsigned long long leaf2(const uint64_t (&C)[NW], const RootView &R, unsigned gm, int j,
                                                    unsigned &ovf) {
  uint64_t T[NW];
#pragma unroll
  for (int r = 0; r < NW; ++r) T[r] = C[r];
  unsigned long long acc = 0;
  int x;
  while (next_bit<G, NW>(T, gm, j, x)) {
    const uint64_t *rx = R.rows + (size_t)x * R.RS + j;
    unsigned a = 0;
#pragma unroll
    for (int r = 0; r < NW; ++r) a += __popcll(C[r] & rx[r * G]);
    if (PV) {
      a = gsum32<G>(a, gm);
      if (j == 0 && a) atomic_add_ck(&R.cnt[x], a, ovf);
    }
    acc += a;
  }
  if (PV) {
#pragma unroll
    for (int r = 0; r < NW; ++r) T[r] = C[r];
    while (next_bit<G, NW>(T, gm, j, x)) {
      const uint64_t *cy = R.colT + (size_t)x * R.RS + j;
      unsigned b = 0;
#pragma unroll
      for (int r = 0; r < NW; ++r) b += __popcll(C[r] & cy[r * G]);
      b = gsum32<G>(b, gm);
      if (j == 0 && b) atomic_add_ck(&R.cnt[x], b, ovf);
    }
  }
  return acc;
}

// Rec-Count-Cliques with ell >= 2 vertices still to pick from C (Algorithm 1),
// as an explicit stack; prunes a branch whose candidate set has fewer than the
// vertices still needed (the cut-off of Section 5.1's discussion).
template <int G, int NW, bool PV>
__device__ unsigned long long dfs(const uint64_t (&C0)[NW], int ell, const RootView &R, unsigned gm, int j,
                                  unsigned &ovf) {
  if (ell == 2) return leaf2<G, NW, PV>(C0, R, gm, j, ovf);
  uint64_t Cs[kMaxFrames][NW], Ts[kMaxFrames][NW];
  unsigned long long subs[kMaxFrames];
  int xs[kMaxFrames];
  int top = 0;
#pragma unroll
  for (int r = 0; r < NW; ++r) Cs[0][r] = Ts[0][r] = C0[r];
  subs[0] = 0;
  unsigned long long ret = 0;
  for (;;) {
    const int l = ell - top;
    unsigned long long a = 0;
    bool done = false;
    uint64_t C[NW];
#pragma unroll
    for (int r = 0; r < NW; ++r) C[r] = Cs[top][r];
    if (l == 2) {
      a = leaf2<G, NW, PV>(C, R, gm, j, ovf);
      done = true;
    } else {
      uint64_t T[NW];
#pragma unroll
      for (int r = 0; r < NW; ++r) T[r] = Ts[top][r];
      int x;
      const bool has = next_bit<G, NW>(T, gm, j, x);
#pragma unroll
      for (int r = 0; r < NW; ++r) Ts[top][r] = T[r];
      if (!has) {
        a = subs[top];
        done = true;
      } else {
        const uint64_t *rx = R.rows + (size_t)x * R.RS + j;
        uint64_t Cn[NW];
        unsigned c = 0;
#pragma unroll
        for (int r = 0; r < NW; ++r) {
          Cn[r] = C[r] & rx[r * G];
          c += __popcll(Cn[r]);
        }
        c = gsum32<G>(c, gm);
        if (top + 1 >= kMaxFrames) ovf |= ST_CAPACITY;
        if ((int)c >= l - 1 && top + 1 < kMaxFrames) {
          xs[top] = x;
          ++top;
#pragma unroll
          for (int r = 0; r < NW; ++r) Cs[top][r] = Ts[top][r] = Cn[r];
          subs[top] = 0;
        }
      }
    }
    if (done) {
      if (top == 0) {
        ret = a;
        break;
      }
      --top;
      subs[top] = add_ck(subs[top], a, ovf);
      if (PV && j == 0) atomic_add_ck(&R.cnt[xs[top]], a, ovf);
    }
  }
  return ret;
}

// ------------------------------------------------------------ item loops
// Items of one root, taken by lane groups through the team counter `next`.
// k = 4: item i = arc u->x_i, candidates row_i, two vertices left.
// k >= 5: item t = triangle u->x_i->x_j (j the r-th bit of row_i with
// pre[i] + r = t), candidates row_i & row_j, k-3 vertices left.
// rsum receives this thread's share of the root total (lane partials, or the
// group-uniform value on the group's first lane).
template <int G, int NW, bool PV, bool PA>
__device__ void run_items(const RootView &R, int k, unsigned *next, uint32_t nitems, unsigned long long &rsum,
                          unsigned &ovf, unsigned *status) {
  const unsigned gm = group_mask<G>();
  const int j = (int)(lane_id() & (unsigned)(G - 1));
  for (;;) {
    unsigned t = 0;
    if (j == 0) t = atomicAdd(next, 1u);
    if constexpr (G > 1) t = __shfl_sync(gm, t, 0, G);
    if (t >= nitems) break;
    uint32_t i, jv = 0;
    uint64_t C[NW];
    if (k == 4) {
      i = t;
#pragma unroll
      for (int r = 0; r < NW; ++r) C[r] = R.rows[(size_t)i * R.RS + r * G + j];
    } else {
      uint32_t lo = 0, hi = R.d;  // last i with pre[i] <= t
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (R.pre[mid] <= t) lo = mid; else hi = mid - 1;
      }
      i = lo;
      if (i >= R.d) {
        if (j == 0) atomicOr(status, ST_CAPACITY);
        continue;
      }
      uint32_t rr = t - R.pre[i];
      int found = -1;
      for (uint32_t w = 0; w < R.RS; ++w) {
        uint64_t word = R.rows[(size_t)i * R.RS + w];
        const uint32_t c = (uint32_t)__popcll(word);
        if (rr < c) {
          for (; rr; --rr) word &= word - 1;
          found = (int)(w * 64 + __ffsll((long long)word) - 1);
          break;
        }
        rr -= c;
      }
      if (found < 0 || (uint32_t)found >= R.d) {
        if (j == 0) atomicOr(status, ST_CAPACITY);
        continue;
      }
      jv = (uint32_t)found;
#pragma unroll
      for (int r = 0; r < NW; ++r)
        C[r] = R.rows[(size_t)i * R.RS + r * G + j] & R.rows[(size_t)jv * R.RS + r * G + j];
    }
    const int ell = (k == 4) ? 2 : k - 3;
    unsigned pc = 0;
#pragma unroll
    for (int r = 0; r < NW; ++r) pc += __popcll(C[r]);
    pc = gsum32<G>(pc, gm);
    if ((int)pc < ell) continue;
    const unsigned long long s = dfs<G, NW, PV>(C, ell, R, gm, j, ovf);
    if (PV) {
      if (j == 0) {
        rsum = add_ck(rsum, s, ovf);
        atomic_add_ck(&R.cnt[i], s, ovf);
        if (k >= 5) atomic_add_ck(&R.cnt[jv], s, ovf);
        if (PA) atomic_add_ck(&R.asub[i], s, ovf);
      }
    } else {
      rsum = add_ck(rsum, s, ovf);
      if (PA) {
        const unsigned long long sg = gsum64<G>(s, gm);
        if (j == 0) atomic_add_ck(&R.asub[i], sg, ovf);
      }
    }
  }
}

// k = 3 at a root: |row_i| triangles on arc i; per vertex the middle vertex
// gets |row_i| and the top vertex t gets |col_t|.
template <bool PV, bool PA>
__device__ void triangles_at_root(const RootView &R, unsigned tid, unsigned nthreads, unsigned long long &rsum,
                                  unsigned &ovf) {
  for (uint32_t i = tid; i < R.d; i += nthreads) {
    unsigned c = 0, ct = 0;
    for (uint32_t w = 0; w < R.RS; ++w) {
      c += __popcll(R.rows[(size_t)i * R.RS + w]);
      if (PV) ct += __popcll(R.colT[(size_t)i * R.RS + w]);
    }
    rsum = add_ck(rsum, c, ovf);
    if (PV) R.cnt[i] += (unsigned long long)c + ct;
    if (PA) R.asub[i] = c;
  }
}

template <bool PV, bool PA>
__device__ void dispatch_items(const RootView &R, int k, unsigned *next, uint32_t nitems,
                               unsigned long long &rsum, unsigned &ovf, unsigned *status) {
  switch (R.RS) {
    case 1: run_items<1, 1, PV, PA>(R, k, next, nitems, rsum, ovf, status); break;
    case 2: run_items<2, 1, PV, PA>(R, k, next, nitems, rsum, ovf, status); break;
    case 4: run_items<4, 1, PV, PA>(R, k, next, nitems, rsum, ovf, status); break;
    case 8: run_items<8, 1, PV, PA>(R, k, next, nitems, rsum, ovf, status); break;
    case 16: run_items<16, 1, PV, PA>(R, k, next, nitems, rsum, ovf, status); break;
    case 32: run_items<32, 1, PV, PA>(R, k, next, nitems, rsum, ovf, status); break;
    case 64: run_items<32, 2, PV, PA>(R, k, next, nitems, rsum, ovf, status); break;
    case 128: run_items<32, 4, PV, PA>(R, k, next, nitems, rsum, ovf, status); break;
    case 256: run_items<32, 8, PV, PA>(R, k, next, nitems, rsum, ovf, status); break;
    default:
      if (lane_id() == 0) atomicOr(status, ST_CAPACITY);
  }
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------- block-level root
template <bool PV, bool PA>
__device__ void block_root(const CountArgs &a, uint32_t u, uint8_t *base, unsigned long long &tsum, unsigned &ovf,
                           unsigned long long *red, unsigned *s_next, unsigned *s_items) {
  const unsigned tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  const uint64_t b = a.ptr[u];
  const uint32_t d = (uint32_t)(a.ptr[u + 1] - b);
  const uint32_t RS = row_stride(d);
  const RootView R = carve(base, d, RS, d, PV, PA);
  for (uint32_t i = tid; i < d; i += kBlock) R.L[i] = a.col[b + i];
  for (size_t w = tid; w < (size_t)d * RS; w += kBlock) {
    R.rows[w] = 0;
    if (PV) R.colT[w] = 0;
  }
  for (uint32_t i = tid; i < d; i += kBlock) {
    if (PV) R.cnt[i] = 0;
    if (PA) R.asub[i] = 0;
  }
  __syncthreads();
  build_rows(R, a.ptr, a.col, warp, kWarps, PV);
  __syncthreads();
  unsigned long long rsum = 0;
  if (a.k == 3) {
    triangles_at_root<PV, PA>(R, tid, kBlock, rsum, ovf);
  } else {
    uint32_t nitems = d;
    if (a.k >= 5) {
      // pre[i] = sum_{i' < i} |row_i'|, by a block scan over per-thread chunks
      const uint32_t per = (d + kBlock - 1) / kBlock;
      const uint32_t c0 = tid * per, c1 = min(d, c0 + per);
      unsigned long long loc = 0;
      for (uint32_t i = c0; i < c1; ++i) {
        unsigned c = 0;
        for (uint32_t w = 0; w < RS; ++w) c += __popcll(R.rows[(size_t)i * RS + w]);
        R.pre[i] = c;  // temporarily the row count
        loc += c;
      }
      // exclusive scan of loc over the block
      unsigned long long x = loc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
      }
      if (lane == 31) red[warp] = x;
      __syncthreads();
      unsigned long long off = 0, all = 0;
      for (int w = 0; w < kWarps; ++w) {
        if (w < (int)warp) off += red[w];
        all += red[w];
      }
      off += x - loc;
      for (uint32_t i = c0; i < c1; ++i) {
        const uint32_t c = R.pre[i];
        R.pre[i] = (uint32_t)off;
        off += c;
      }
      if (tid == 0) {
        R.pre[d] = (uint32_t)all;
        *s_items = (uint32_t)all;
        if (all > 0xffffffffull) atomicOr(a.status, ST_CAPACITY);
      }
      __syncthreads();
      nitems = *s_items;
    }
    if (tid == 0) *s_next = 0;
    __syncthreads();
    dispatch_items<PV, PA>(R, a.k, s_next, nitems, rsum, ovf, a.status);
  }
  __syncthreads();
  if (PV) {
    unsigned long long r = warp_sum64(rsum);
    if (lane == 0) red[warp] = r;
    __syncthreads();
    if (tid == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < kWarps; ++w) t = add_ck(t, red[w], ovf);
      atomic_add_ck(&a.pv[u], t, ovf);
    }
    for (uint32_t i = tid; i < d; i += kBlock) atomic_add_ck(&a.pv[R.L[i]], R.cnt[i], ovf);
  }
  if (PA) {
    for (uint32_t i = tid; i < d; i += kBlock) a.pa[b + i] = R.asub[i];
  }
  tsum = add_ck(tsum, rsum, ovf);
  __syncthreads();
}

// -------------------------------------------------------- warp-level root
template <bool PV, bool PA>
__device__ void warp_root(const CountArgs &a, uint32_t u, const RootView &S, unsigned long long &tsum,
                          unsigned &ovf, unsigned *w_next) {
  const unsigned lane = lane_id();
  const uint64_t b = a.ptr[u];
  const uint32_t d = (uint32_t)(a.ptr[u + 1] - b);
  RootView R = S;
  R.d = d;
  R.RS = 1;
  for (uint32_t i = lane; i < kLightMax; i += 32) {
    if (i < d) R.L[i] = a.col[b + i];
    R.rows[i] = 0;
    if (PV) {
      R.colT[i] = 0;
      R.cnt[i] = 0;
    }
    if (PA) R.asub[i] = 0;
  }
  __syncwarp();
  build_rows(R, a.ptr, a.col, 0, 1, PV);
  __syncwarp();
  unsigned long long rsum = 0;
  if (a.k == 3) {
    triangles_at_root<PV, PA>(R, lane, 32, rsum, ovf);
  } else {
    uint32_t nitems = d;
    if (a.k >= 5) {
      // pre[i] = sum_{i' < i} |row_i'| over the 64 slots (rows past d are empty,
      // so pre[d] is the item total)
      const uint32_t c0 = lane < d ? (uint32_t)__popcll(R.rows[lane]) : 0u;
      const uint32_t c1 = lane + 32 < d ? (uint32_t)__popcll(R.rows[lane + 32]) : 0u;
      uint32_t z0 = c0, z1 = c1;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y0 = __shfl_up_sync(0xffffffffu, z0, o);
        const uint32_t y1 = __shfl_up_sync(0xffffffffu, z1, o);
        if (lane >= (unsigned)o) {
          z0 += y0;
          z1 += y1;
        }
      }
      const uint32_t tot0 = __shfl_sync(0xffffffffu, z0, 31);
      const uint32_t tot1 = __shfl_sync(0xffffffffu, z1, 31);
      R.pre[lane] = z0 - c0;
      R.pre[lane + 32] = tot0 + z1 - c1;
      if (lane == 0) R.pre[kLightMax] = tot0 + tot1;
      nitems = tot0 + tot1;
      __syncwarp();
    }
    if (lane == 0) *w_next = 0;
    __syncwarp();
    run_items<1, 1, PV, PA>(R, a.k, w_next, nitems, rsum, ovf, a.status);
  }
  __syncwarp();
  if (PV) {
    const unsigned long long t = warp_sum64(rsum);
    if (lane == 0) atomic_add_ck(&a.pv[u], t, ovf);
    for (uint32_t i = lane; i < d; i += 32) atomic_add_ck(&a.pv[R.L[i]], R.cnt[i], ovf);
  }
  if (PA) {
    for (uint32_t i = lane; i < d; i += 32) a.pa[b + i] = R.asub[i];
  }
  tsum = add_ck(tsum, rsum, ovf);
  __syncwarp();
}

// ---------------------------------------------------------------- kernel
// Persistent: roots are pulled from three atomic queues in order of
// decreasing out-degree (huge roots first, with their matrices in global
// scratch; then heavy roots, one block each; then light roots, one warp each).
template <bool PV, bool PA>
__global__ void __launch_bounds__(kBlock) count_kernel(CountArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ unsigned long long red[kWarps];
  __shared__ unsigned s_root, s_next, s_items, s_stop;
  __shared__ unsigned w_next[kWarps];
  const unsigned tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  unsigned ovf = 0;
  unsigned long long tsum = 0;

  // phase 1: huge roots
  if (blockIdx.x < a.scratch_blocks) {
    uint8_t *slab = (uint8_t *)a.scratch + (size_t)blockIdx.x * a.scratch_stride;
    for (;;) {
      if (tid == 0) {
        s_stop = 0;
        if (a.deadline_ns && globaltimer_ns() > a.deadline_ns) {
          atomicOr(a.status, ST_TIMEOUT);
          s_stop = 1;
        }
        s_root = s_stop ? 0xffffffffu : atomicAdd(&a.queue[0], 1u);
      }
      __syncthreads();
      const unsigned idx = s_root;
      __syncthreads();
      if (idx >= a.n_huge) break;
      block_root<PV, PA>(a, a.order[idx], slab, tsum, ovf, red, &s_next, &s_items);
    }
  }
  // phase 2: heavy roots
  for (;;) {
    if (tid == 0) {
      s_stop = 0;
      if (a.deadline_ns && globaltimer_ns() > a.deadline_ns) {
        atomicOr(a.status, ST_TIMEOUT);
        s_stop = 1;
      }
      s_root = s_stop ? 0xffffffffu : atomicAdd(&a.queue[1], 1u);
    }
    __syncthreads();
    const unsigned idx = s_root;
    __syncthreads();
    if (idx >= a.n_heavy_end - a.n_huge) break;
    block_root<PV, PA>(a, a.order[a.n_huge + idx], smem, tsum, ovf, red, &s_next, &s_items);
  }
  // phase 3: light roots, one warp each
  {
    const size_t slot = light_slot_bytes(PV, PA);
    const RootView S = carve(smem + (size_t)warp * slot, kLightMax, 1, 0, PV, PA);
    const uint32_t nlight = a.n_light_end - a.n_heavy_end;
    for (;;) {
      unsigned idx = 0;
      if (lane == 0) {
        if (a.deadline_ns && globaltimer_ns() > a.deadline_ns) {
          atomicOr(a.status, ST_TIMEOUT);
          idx = 0xffffffffu;
        } else {
          idx = atomicAdd(&a.queue[2], 1u);
        }
      }
      idx = __shfl_sync(0xffffffffu, idx, 0);
      if (idx >= nlight) break;
      warp_root<PV, PA>(a, a.order[a.n_heavy_end + idx], S, tsum, ovf, &w_next[warp]);
    }
  }
  // block reduction of the thread shares, one atomic per block
  __syncthreads();
  unsigned long long r = 0;
  {
    // overflow-checked warp reduction
    unsigned long long v = tsum;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, v, o);
      const unsigned long long s = v + y;
      ovf |= (s < v) ? ST_OVERFLOW : 0u;
      v = s;
    }
    r = v;
  }
  ovf = __reduce_or_sync(0xffffffffu, ovf);
  if (lane == 0) red[warp] = r;
  __syncthreads();
  if (tid == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kWarps; ++w) t = add_ck(t, red[w], ovf);
    atomic_add_ck(a.total, t, ovf);
  }
  if (lane == 0 && ovf) atomicOr(a.status, ovf);
}

cudaError_t set_count_smem(bool pv, bool pa, size_t smem) {
  cudaError_t e;
  if (pv && pa) e = cudaFuncSetAttribute(count_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else if (pv) e = cudaFuncSetAttribute(count_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else if (pa) e = cudaFuncSetAttribute(count_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else e = cudaFuncSetAttribute(count_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e;
}

int count_blocks_per_sm(bool pv, bool pa, size_t smem) {
  int nb = 0;
  if (pv && pa) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, count_kernel<true, true>, kBlock, smem);
  else if (pv) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, count_kernel<true, false>, kBlock, smem);
  else if (pa) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, count_kernel<false, true>, kBlock, smem);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, count_kernel<false, false>, kBlock, smem);
  return nb;
}

cudaError_t launch_count(const CountArgs &a, bool pv, bool pa, int grid, size_t smem, cudaStream_t s) {
  note_launch();
  if (pv && pa) count_kernel<true, true><<<grid, kBlock, smem, s>>>(a);
  else if (pv) count_kernel<true, false><<<grid, kBlock, smem, s>>>(a);
  else if (pa) count_kernel<false, true><<<grid, kBlock, smem, s>>>(a);
  else count_kernel<false, false><<<grid, kBlock, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace kc
