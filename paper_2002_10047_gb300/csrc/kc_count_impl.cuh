// Counting kernels: arb-count and arb-count-v (Algorithm 1, Section 3.2)
// with the practical optimizations of Section 3.3, laid out for sm_103a.
//
// Every k-clique is found exactly once, below its lowest vertex u in the total
// order (the root), as a (k-1)-clique of the DAG induced on N+(u). For each
// root the team (one warp when d+(u) <= 64, one block otherwise) builds that
// induced subgraph once -- "the induced subgraph on N_DG(v)" of Section 3.3 --
// as a bit matrix over positions 0..d-1 in N+(u) (the relabelling to
// [0, O(alpha)] of Section 3.3): row i holds N+(N+(u)[i]) within N+(u).
// Membership of an out-neighbour in N+(u) is found through an open-addressing
// hash table in shared memory.
//
// Below the root the work is split by arcs (edge parallelism, Section 3.3):
// the candidates of arc u->x_i are row_i = N+(u) ∩ N+(x_i). For k >= 5 a warp
// compacts that intersection (or, when it has more than 128 vertices, the
// intersection with one more vertex) to local ids 0..s-1: its own bit matrix
// of s <= 128 rows of one or two words. The warp's lanes then split the first
// level of that matrix and run Rec-Count-Cliques in registers: intersect =
// word-wise AND, |I| = population count, the base case l = 1 folded into the
// level above (l = 2: sum over x of |C & row_x|), and a branch is cut when
// its candidate set has fewer vertices than still needed.
//
// Per-vertex counts (arb-count-v): the cliques completed at the l = 2 level of
// candidate set C are the arcs x->y inside C; vertex v in C is in |C & sym_v|
// of them, sym_v = row_v | col_v being v's neighbours in either direction, and
// their number is half the sum of those credits -- one pass over C, no
// per-clique increment. Vertices higher on the path get the totals of their
// sub-trees and the root gets the root total. Counters are flushed to global memory once per
// root. Every addition is checked for uint64 wrap-around.
#pragma once
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

__device__ __forceinline__ unsigned long long warp_sum64_ck(unsigned long long v, unsigned &ovf) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, v, o);
    const unsigned long long s = v + y;
    ovf |= (s < v) ? ST_OVERFLOW : 0u;
    v = s;
  }
  return v;
}

__device__ __forceinline__ unsigned warp_incl_scan(unsigned v) {
  const unsigned lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= (unsigned)o) v += y;
  }
  return v;
}

// ------------------------------------------------------------ hash table
constexpr uint32_t kEmpty = 0xffffffffu;

__device__ __forceinline__ uint32_t hslot(uint32_t y, uint32_t mask) {
  const uint32_t h = y * 2654435761u;
  return (h ^ (h >> 15)) & mask;
}

// keys are distinct and the table has at least twice as many slots as keys
__device__ __forceinline__ void hinsert(uint32_t *hkey, uint16_t *hpos, uint32_t T, uint32_t y, uint32_t pos) {
  uint32_t s = hslot(y, T - 1);
  for (uint32_t probe = 0; probe < T; ++probe) {
    if (atomicCAS(&hkey[s], kEmpty, y) == kEmpty) {
      hpos[s] = (uint16_t)pos;
      return;
    }
    s = (s + 1) & (T - 1);
  }
}

__device__ __forceinline__ int hlookup(const uint32_t *hkey, const uint16_t *hpos, uint32_t T, uint32_t y) {
  uint32_t s = hslot(y, T - 1);
  for (uint32_t probe = 0; probe < T; ++probe) {
    const uint32_t k = hkey[s];
    if (k == y) return hpos[s];
    if (k == kEmpty) return -1;
    s = (s + 1) & (T - 1);
  }
  return -1;
}

// ---------------------------------------------------------- DFS engine
// A bit matrix as the DFS sees it: row x at rows + x*RS, W words in use.
struct MatView {
  const uint64_t *rows;
  const uint64_t *sym;         // rows | transposed rows (per-vertex only)
  unsigned long long *cnt;     // per-vertex counters (per-vertex only)
  uint32_t RS, W;
};

template <int G>
__device__ __forceinline__ unsigned gsum32(unsigned v) {
  if constexpr (G == 1) return v;
  else return __reduce_add_sync(0xffffffffu, v);
}

// Lane j of a G-lane group (G = 1 or 32) holds words r*G + j (r < NW) of a
// set; words at or past W read as zero (a one-word set always has W = 1).
template <int G, int NW>
__device__ __forceinline__ void load_row(const uint64_t *base, uint32_t W, int j, uint64_t (&out)[NW]) {
#pragma unroll
  for (int r = 0; r < NW; ++r) {
    const uint32_t w = (uint32_t)(r * G + j);
    out[r] = (NW == 1 || w < W) ? base[w] : 0ull;
  }
}

// Next set bit of a group-distributed set; clears it and returns its position.
template <int G, int NW>
__device__ __forceinline__ bool next_bit(uint64_t (&T)[NW], int j, int &x) {
#pragma unroll
  for (int r = 0; r < NW; ++r) {
    if constexpr (G == 1) {
      if (T[r]) {
        x = r * 64 + __ffsll((long long)T[r]) - 1;
        T[r] &= T[r] - 1;
        return true;
      }
    } else {
      const unsigned bal = __ballot_sync(0xffffffffu, T[r] != 0ull);
      if (bal) {
        const int jj = __ffs(bal) - 1;
        const uint64_t w = __shfl_sync(0xffffffffu, T[r], jj);
        x = (r * G + jj) * 64 + __ffsll((long long)w) - 1;
        if (j == jj) T[r] &= T[r] - 1;
        return true;
      }
    }
  }
  return false;
}

// l = 2 below candidate set C: the number of arcs x->y inside C, i.e. the sum
// over x in C of |C & row_x|; each lane returns its partial sum. With
// per-vertex counts every v in C is credited |C & sym_v| (the completed
// cliques through v) and the total is half their sum (group-uniform).
template <int G, int NW, bool PV>
__device__ __forceinline__ unsigned long long leaf2(const uint64_t (&C)[NW], const MatView &V, int j,
                                                    unsigned &ovf) {
  uint64_t T[NW];
#pragma unroll
  for (int r = 0; r < NW; ++r) T[r] = C[r];
  unsigned long long acc = 0;
  int x;
  if (!PV) {
    while (next_bit<G, NW>(T, j, x)) {
      uint64_t R[NW];
      load_row<G, NW>(V.rows + (size_t)x * V.RS, V.W, j, R);
      unsigned a = 0;
#pragma unroll
      for (int r = 0; r < NW; ++r) a += __popcll(C[r] & R[r]);
      acc += a;
    }
    return acc;
  }
  if (V.sym == nullptr) {
    ovf |= ST_CAPACITY;  // per-vertex credits need the symmetric rows
    return 0;
  }
  while (next_bit<G, NW>(T, j, x)) {
    uint64_t R[NW];
    load_row<G, NW>(V.sym + (size_t)x * V.RS, V.W, j, R);
    unsigned a = 0;
#pragma unroll
    for (int r = 0; r < NW; ++r) a += __popcll(C[r] & R[r]);
    a = gsum32<G>(a);
    if (j == 0 && a) atomic_add_ck(&V.cnt[x], a, ovf);
    acc += a;
  }
  return acc >> 1;
}

// Rec-Count-Cliques with ell >= 2 vertices still to pick from C, as an
// explicit stack; returns lane partials (group-uniform with per-vertex).
template <int G, int NW, bool PV>
__device__ unsigned long long dfs(const uint64_t (&C0)[NW], int ell, const MatView &V, int j, unsigned &ovf) {
  if (ell == 2) return leaf2<G, NW, PV>(C0, V, j, ovf);
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
      a = leaf2<G, NW, PV>(C, V, j, ovf);
      done = true;
    } else {
      uint64_t T[NW];
#pragma unroll
      for (int r = 0; r < NW; ++r) T[r] = Ts[top][r];
      int x;
      const bool has = next_bit<G, NW>(T, j, x);
#pragma unroll
      for (int r = 0; r < NW; ++r) Ts[top][r] = T[r];
      if (!has) {
        a = subs[top];
        done = true;
      } else {
        uint64_t R[NW], Cn[NW];
        load_row<G, NW>(V.rows + (size_t)x * V.RS, V.W, j, R);
        unsigned c = 0;
#pragma unroll
        for (int r = 0; r < NW; ++r) {
          Cn[r] = C[r] & R[r];
          c += __popcll(Cn[r]);
        }
        c = gsum32<G>(c);
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
      if (PV && j == 0) atomic_add_ck(&V.cnt[xs[top]], a, ovf);
    }
  }
  return ret;
}

// ----------------------------------------------------- warp item engines
struct Slot {
  uint64_t *mask;             // 32 mask words of the current candidate set (root positions)
  uint32_t *pfx;              // exclusive prefix of their population counts
  uint16_t *P;                // root positions of the compacted vertices
  uint64_t *S, *SN;           // compacted rows and their symmetric closure (s x NWc words)
  unsigned long long *cs;     // local per-vertex counters
};

__device__ __forceinline__ Slot carve_slot(uint8_t *base, bool pv) {
  const SlotLayout o = slot_layout(pv);
  Slot s;
  s.mask = (uint64_t *)(base + o.mask);
  s.pfx = (uint32_t *)(base + o.pfx);
  s.P = (uint16_t *)(base + o.P);
  s.S = (uint64_t *)(base + o.S);
  s.SN = pv ? (uint64_t *)(base + o.ST) : nullptr;
  s.cs = pv ? (unsigned long long *)(base + o.cs) : nullptr;
  return s;
}

// Count the cliques that take `picks` (>= 2) more vertices from a candidate set
// of s <= kCompactMax root positions whose words (W <= 32) lane w holds in
// mword. The set is compacted to local ids 0..s-1, its induced rows are
// extracted from the root matrix, and the lanes split the first pick.
// Per-vertex credits of the picked vertices go to the root counters rc.
// Returns the warp-uniform total.
template <bool PV>
__device__ unsigned long long compact_count(const MatView &M, uint64_t mword, uint32_t s, int picks, const Slot &sl,
                                            unsigned long long *rc, unsigned &ovf) {
  const unsigned lane = lane_id();
  const uint32_t W = M.W;
  const unsigned c = lane < W ? (unsigned)__popcll(mword) : 0u;
  const unsigned pfx = warp_incl_scan(c) - c;
  if (lane < W) {
    sl.mask[lane] = mword;
    sl.pfx[lane] = pfx;
    uint64_t bw = mword;
    unsigned r = pfx;
    while (bw) {
      if (r < (unsigned)kCompactMax) sl.P[r] = (uint16_t)(lane * 64 + __ffsll((long long)bw) - 1);
      ++r;
      bw &= bw - 1;
    }
  }
  const uint32_t NWc = s <= 64 ? 1u : 2u;
  for (uint32_t q = lane; q < s * NWc; q += 32) {
    sl.S[q] = 0;
    if (PV) sl.SN[q] = 0;
  }
  if (PV)
    for (uint32_t q = lane; q < s; q += 32) sl.cs[q] = 0;
  __syncwarp();
  // bit b of compacted row q <=> P[b] in N+(P[q]) within the set
  for (uint32_t q = lane; q < s; q += 32) {
    const uint64_t *src = M.rows + (size_t)sl.P[q] * M.RS;
    uint64_t o0 = 0, o1 = 0;
    for (uint32_t w = 0; w < W; ++w) {
      const uint64_t mk = sl.mask[w];
      uint64_t bits = src[w] & mk;
      while (bits) {
        const int bb = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        const uint32_t loc = sl.pfx[w] + (uint32_t)__popcll(mk & ((1ull << bb) - 1ull));
        if (loc < 64) o0 |= 1ull << loc;
        else o1 |= 1ull << (loc - 64);
        if (PV) {
          atomicOr((unsigned long long *)&sl.SN[loc * NWc + (q >> 6)], 1ull << (q & 63));
          atomicOr((unsigned long long *)&sl.SN[q * NWc + (loc >> 6)], 1ull << (loc & 63));
        }
      }
    }
    sl.S[q * NWc] = o0;
    if (NWc == 2) sl.S[q * NWc + 1] = o1;
  }
  __syncwarp();
  unsigned long long acc = 0;
  MatView V;
  V.rows = sl.S;
  V.sym = sl.SN;
  V.cnt = sl.cs;
  V.RS = NWc;
  V.W = NWc;
  for (uint32_t q = lane; q < s; q += 32) {
    unsigned long long sub = 0;
    if (NWc == 1) {
      uint64_t C[1] = {sl.S[q]};
      const int pc = __popcll(C[0]);
      if (picks == 2) sub = (unsigned long long)pc;
      else if (pc >= picks - 1) sub = dfs<1, 1, PV>(C, picks - 1, V, 0, ovf);
    } else {
      uint64_t C[2] = {sl.S[2 * q], sl.S[2 * q + 1]};
      const int pc = __popcll(C[0]) + __popcll(C[1]);
      if (picks == 2) sub = (unsigned long long)pc;
      else if (pc >= picks - 1) sub = dfs<1, 2, PV>(C, picks - 1, V, 0, ovf);
    }
    if (PV && picks > 2 && sub) atomic_add_ck(&sl.cs[q], sub, ovf);
    acc = add_ck(acc, sub, ovf);
  }
  if (PV && picks == 2) {
    // each arc q->y of the compacted subgraph is one clique: q and y both in it
    for (uint32_t y = lane; y < s; y += 32) {
      unsigned bcnt = (unsigned)__popcll(sl.SN[y * NWc]);
      if (NWc == 2) bcnt += (unsigned)__popcll(sl.SN[y * NWc + 1]);
      if (bcnt) atomic_add_ck(&sl.cs[y], bcnt, ovf);
    }
  }
  __syncwarp();
  if (PV)
    for (uint32_t q = lane; q < s; q += 32) atomic_add_ck(&rc[sl.P[q]], sl.cs[q], ovf);
  const unsigned long long tot = warp_sum64_ck(acc, ovf);
  __syncwarp();
  return tot;
}

// Position of the r-th set bit of the set whose words and exclusive prefix
// counts are in the slot (W <= 32 words).
__device__ __forceinline__ uint32_t slot_select(const Slot &sl, uint32_t W, uint32_t r) {
  uint32_t lo = 0, hi = W - 1;  // last word with pfx <= r
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (sl.pfx[mid] <= r) lo = mid; else hi = mid - 1;
  }
  uint64_t bb = sl.mask[lo];
  for (uint32_t q = r - sl.pfx[lo]; q; --q) bb &= bb - 1;
  return lo * 64 + (uint32_t)(__ffsll((long long)bb) - 1);
}

// Lanes split the first pick of the candidate set rowA & rowB (root
// positions, W <= NW <= 32 words) and each lane runs the DFS on the root's
// rows with NW-word sets in registers. Per-vertex credits go to the root
// counters of M. Returns the warp-uniform total.
template <int NW, bool PV>
__device__ unsigned long long split_count(const MatView &M, const uint64_t *rowA, const uint64_t *rowB, int picks,
                                          const Slot &sl, unsigned &ovf) {
  const unsigned lane = lane_id();
  const uint32_t W = M.W;
  const uint64_t mw = lane < W ? (rowA[lane] & (rowB ? rowB[lane] : ~0ull)) : 0ull;
  const unsigned c = (unsigned)__popcll(mw);
  const unsigned incl = warp_incl_scan(c);
  const uint32_t s = __shfl_sync(0xffffffffu, incl, 31);
  if (lane < W) {
    sl.mask[lane] = mw;
    sl.pfx[lane] = incl - c;
  }
  __syncwarp();
  unsigned long long acc = 0;
  for (uint32_t r = lane; r < s; r += 32) {
    const uint32_t x = slot_select(sl, W, r);
    const uint64_t *rx = M.rows + (size_t)x * M.RS;
    uint64_t C[NW];
    int pc = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      C[w] = (uint32_t)w < W ? (sl.mask[w] & rx[w]) : 0ull;
      pc += __popcll(C[w]);
    }
    unsigned long long sub = 0;
    if (picks == 2) sub = (unsigned long long)pc;
    else if (pc >= picks - 1) sub = dfs<1, NW, PV>(C, picks - 1, M, 0, ovf);
    if (PV && picks > 2 && sub) atomic_add_ck(&M.cnt[x], sub, ovf);
    acc = add_ck(acc, sub, ovf);
  }
  if (PV && picks == 2) {
    // each arc x->y inside the set is one clique: v is in |set & sym_v| of them
    for (uint32_t r = lane; r < s; r += 32) {
      const uint32_t y = slot_select(sl, W, r);
      const uint64_t *cy = M.sym + (size_t)y * M.RS;
      unsigned b = 0;
      for (uint32_t w = 0; w < W; ++w) b += (unsigned)__popcll(sl.mask[w] & cy[w]);
      if (b) atomic_add_ck(&M.cnt[y], b, ovf);
    }
  }
  __syncwarp();
  return warp_sum64_ck(acc, ovf);
}

// Lanes-over-words engine for a candidate set too large to compact: the warp
// is one 32-lane group, lane j holding words r*32 + j of the root's rows.
template <int NW, bool PV>
__device__ unsigned long long generic_count(const MatView &M, const uint64_t *rowA, const uint64_t *rowB, int picks,
                                            unsigned &ovf) {
  const int j = (int)lane_id();
  uint64_t C[NW];
#pragma unroll
  for (int r = 0; r < NW; ++r) {
    const uint32_t w = (uint32_t)(r * 32 + j);
    C[r] = w < M.W ? (rowA[w] & (rowB ? rowB[w] : ~0ull)) : 0ull;
  }
  unsigned long long s = dfs<32, NW, PV>(C, picks, M, j, ovf);
  if (!PV) s = warp_sum64_ck(s, ovf);
  return s;
}

template <bool PV>
__device__ unsigned long long generic_dispatch(const MatView &M, const uint64_t *rowA, const uint64_t *rowB,
                                               int picks, const Slot &sl, unsigned &ovf, unsigned *status) {
  if (M.W <= 2) return split_count<2, PV>(M, rowA, rowB, picks, sl, ovf);
  if (M.W <= 4) return split_count<4, PV>(M, rowA, rowB, picks, sl, ovf);
  if (M.W <= 8) return split_count<8, PV>(M, rowA, rowB, picks, sl, ovf);
  if (M.W <= 12) return split_count<12, PV>(M, rowA, rowB, picks, sl, ovf);
  const uint32_t nw = (M.W + 31u) / 32u;
  if (nw <= 1) return generic_count<1, PV>(M, rowA, rowB, picks, ovf);
  if (nw <= 2) return generic_count<2, PV>(M, rowA, rowB, picks, ovf);
  if (nw <= 4) return generic_count<4, PV>(M, rowA, rowB, picks, ovf);
  if (nw <= 8) return generic_count<8, PV>(M, rowA, rowB, picks, ovf);
  if (lane_id() == 0) atomicOr(status, ST_CAPACITY);
  return 0;
}

// k = 4 item of arc i: sum over q in row_i of |row_q & row_i| (lanes take the
// set bits of row_i by rank). Per vertex: q is in |sym_q & row_i| of them.
template <bool PV>
__device__ unsigned long long k4_item(const MatView &M, uint32_t i, uint32_t s, const Slot &sl, unsigned &ovf) {
  const unsigned lane = lane_id();
  const uint32_t W = M.W;
  const uint64_t *ri = M.rows + (size_t)i * M.RS;
  unsigned long long acc = 0;
  for (uint32_t w0 = 0; w0 < W; w0 += 32) {
    // chunks of 32 words (W > 32 only for roots in global scratch)
    const uint32_t wn = min(32u, W - w0);
    const uint64_t mword = lane < wn ? ri[w0 + lane] : 0ull;
    const unsigned c = (unsigned)__popcll(mword);
    const unsigned incl = warp_incl_scan(c);
    const unsigned cs = __shfl_sync(0xffffffffu, incl, 31);
    if (lane < wn) {
      sl.mask[lane] = mword;
      sl.pfx[lane] = incl - c;
    }
    __syncwarp();
    for (uint32_t r = lane; r < cs; r += 32) {
      uint32_t w = 0;
      while (w + 1 < wn && sl.pfx[w + 1] <= r) ++w;
      uint64_t bb = sl.mask[w];
      for (uint32_t q = r - sl.pfx[w]; q; --q) bb &= bb - 1;
      const uint32_t q = (w0 + w) * 64 + (uint32_t)(__ffsll((long long)bb) - 1);
      const uint64_t *rq = M.rows + (size_t)q * M.RS;
      unsigned x = 0, yv = 0;
      for (uint32_t z = 0; z < W; ++z) {
        x += (unsigned)__popcll(rq[z] & ri[z]);
        if (PV) yv += (unsigned)__popcll(M.sym[(size_t)q * M.RS + z] & ri[z]);
      }
      if (PV && yv) atomic_add_ck(&M.cnt[q], (unsigned long long)yv, ovf);
      acc += x;
    }
    __syncwarp();
  }
  (void)s;
  return warp_sum64_ck(acc, ovf);
}

// ------------------------------------------------------- block-level root
struct BlockShared {
  unsigned long long red[kRootWarps];
  unsigned root, next, items, pad;
};

template <bool PV, bool PA>
__device__ void block_root(const CountArgs &a, uint32_t u, uint8_t *base, uint8_t *slots, unsigned long long &tsum,
                           unsigned &ovf, BlockShared &sh) {
  const unsigned tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  const uint64_t b = a.ptr[u];
  const uint32_t d = (uint32_t)(a.ptr[u + 1] - b);
  const uint32_t W = words_of(d), T = hash_slots(d);
  const int k = a.k;
  const bool colT = PV && k >= 4;
  const RootLayout lay = root_layout(d, PV, PA, colT);
  uint32_t *L = (uint32_t *)(base + lay.L);
  uint64_t *rb = (uint64_t *)(base + lay.rb);
  uint32_t *rl = (uint32_t *)(base + lay.rl);
  uint32_t *hkey = (uint32_t *)(base + lay.hkey);
  uint16_t *hpos = (uint16_t *)(base + lay.hpos);
  uint64_t *rows = (uint64_t *)(base + lay.rows);
  uint64_t *sym = colT ? (uint64_t *)(base + lay.colT) : nullptr;
  unsigned long long *cnt = PV ? (unsigned long long *)(base + lay.cnt) : nullptr;
  unsigned long long *asub = PA ? (unsigned long long *)(base + lay.asub) : nullptr;
  uint32_t *pre = (uint32_t *)(base + lay.pre);
  const Slot sl = carve_slot(slots + (size_t)warp * slot_layout(PV).bytes, PV);

  for (uint32_t i = tid; i < d; i += kRootBlock) {
    const uint32_t x = a.col[b + i];
    const uint64_t xb = a.ptr[x];
    L[i] = x;
    rb[i] = xb;
    rl[i] = (uint32_t)(a.ptr[x + 1] - xb);
    if (PV) cnt[i] = 0;
    if (PA) asub[i] = 0;
  }
  for (uint32_t s = tid; s < T; s += kRootBlock) hkey[s] = kEmpty;
  for (size_t w = tid; w < (size_t)d * W; w += kRootBlock) {
    rows[w] = 0;
    if (colT) sym[w] = 0;
  }
  __syncthreads();
  for (uint32_t i = tid; i < d; i += kRootBlock) hinsert(hkey, hpos, T, L[i], i);
  __syncthreads();
  // the induced subgraph on N+(u): warp per row, lanes over N+(L[i]), four
  // loads in flight per lane
  for (uint32_t i = warp; i < d; i += kRootWarps) {
    const uint64_t xb = rb[i];
    const uint32_t len = rl[i];
    for (uint32_t e0 = lane; e0 < len; e0 += 128) {
      uint32_t y[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) y[q] = e0 + 32 * q < len ? a.col[xb + e0 + 32 * q] : kEmpty;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (y[q] == kEmpty) continue;
        const int t = hlookup(hkey, hpos, T, y[q]);
        if (t >= 0) {
          atomicOr((unsigned long long *)&rows[(size_t)i * W + (t >> 6)], 1ull << (t & 63));
          if (colT) {
            atomicOr((unsigned long long *)&sym[(size_t)t * W + (i >> 6)], 1ull << (i & 63));
            atomicOr((unsigned long long *)&sym[(size_t)i * W + (t >> 6)], 1ull << (t & 63));
          }
          if (PV && k == 3) atomicAdd(&cnt[t], 1ull);
        }
      }
    }
  }
  __syncthreads();
  MatView M;
  M.rows = rows;
  M.sym = sym;
  M.cnt = cnt;
  M.RS = W;
  M.W = W;
  unsigned long long rsum = 0;  // lane 0 of each warp holds its item totals
  if (k == 3) {
    for (uint32_t i = tid; i < d; i += kRootBlock) {
      unsigned c = 0;
      for (uint32_t w = 0; w < W; ++w) c += (unsigned)__popcll(rows[(size_t)i * W + w]);
      rsum = add_ck(rsum, c, ovf);
      if (PV) cnt[i] += c;  // cnt[i] already holds i's in-degree within N+(u)
      if (PA) asub[i] = c;
    }
  } else {
    const bool compactable = W <= (uint32_t)kCompactWords;
    uint32_t nitems = d;
    if (k >= 5) {
      // arcs whose candidate sets are too big to compact are split by their
      // next vertex; pre[] numbers those pair items
      const uint32_t per = (d + kRootBlock - 1) / kRootBlock;
      const uint32_t c0 = min(d, tid * per), c1 = min(d, c0 + per);
      unsigned loc = 0;
      for (uint32_t i = c0; i < c1; ++i) {
        unsigned c = 0;
        for (uint32_t w = 0; w < W; ++w) c += (unsigned)__popcll(rows[(size_t)i * W + w]);
        c = (k >= 6 && compactable && c > (unsigned)kCompactMax) ? c : 0u;
        pre[i] = c;
        loc += c;
      }
      const unsigned incl = warp_incl_scan(loc);
      if (lane == 31) sh.red[warp] = incl;
      __syncthreads();
      unsigned off = 0, all = 0;
      for (int w = 0; w < kRootWarps; ++w) {
        if (w < (int)warp) off += (unsigned)sh.red[w];
        all += (unsigned)sh.red[w];
      }
      off += incl - loc;
      for (uint32_t i = c0; i < c1; ++i) {
        const uint32_t c = pre[i];
        pre[i] = off;
        off += c;
      }
      if (tid == 0) {
        pre[d] = all;
        sh.items = d + all;
      }
      __syncthreads();
      nitems = sh.items;
    }
    if (tid == 0) sh.next = 0;
    __syncthreads();
    for (;;) {
      unsigned t = 0;
      if (lane == 0) t = atomicAdd(&sh.next, 1u);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t >= nitems) break;
      unsigned long long item = 0;
      uint32_t i, av = 0xffffffffu;
      if (t < d) {
        i = t;
        const uint64_t *ri = rows + (size_t)i * W;
        unsigned s = 0;
        for (uint32_t w = lane; w < W; w += 32) s += (unsigned)__popcll(ri[w]);
        s = __reduce_add_sync(0xffffffffu, s);
        if (k == 4) {
          if (s >= 2) item = k4_item<PV>(M, i, s, sl, ovf);
        } else if (s >= (unsigned)(k - 2)) {
          if (k == 5 || !compactable) {
            item = generic_dispatch<PV>(M, ri, nullptr, k - 2, sl, ovf, a.status);
          } else if (s <= (unsigned)kCompactMax) {
            item = compact_count<PV>(M, lane < W ? ri[lane] : 0ull, s, k - 2, sl, cnt, ovf);
          }  // else: split into pair items below
        }
      } else {
        // pair item: arc i (more than kCompactMax candidates) and its r-th candidate av
        const uint32_t tt = t - d;
        uint32_t lo = 0, hi = d;  // last i with pre[i] <= tt
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (pre[mid] <= tt) lo = mid; else hi = mid - 1;
        }
        i = lo;
        const uint64_t *ri = rows + (size_t)min(i, d - 1) * W;
        const uint64_t wv = (lane < W && i < d) ? ri[lane] : 0ull;
        const unsigned c = (unsigned)__popcll(wv);
        const unsigned incl = warp_incl_scan(c);
        const unsigned r = i < d ? tt - pre[i] : 0xffffffffu;
        const unsigned hit = __ballot_sync(0xffffffffu, lane < W && r < incl && r >= incl - c);
        if (hit) {
          const int wl = __ffs(hit) - 1;
          if ((int)lane == wl) {
            uint64_t bb = wv;
            for (unsigned q = r - (incl - c); q; --q) bb &= bb - 1;
            av = lane * 64 + (uint32_t)(__ffsll((long long)bb) - 1);
          }
          av = __shfl_sync(0xffffffffu, av, wl);
          const uint64_t *rv = rows + (size_t)av * W;
          const uint64_t mw = lane < W ? (ri[lane] & rv[lane]) : 0ull;
          const unsigned s0 = __reduce_add_sync(0xffffffffu, (unsigned)__popcll(mw));
          if (s0 >= (unsigned)(k - 3)) {
            if (s0 <= (unsigned)kCompactMax) item = compact_count<PV>(M, mw, s0, k - 3, sl, cnt, ovf);
            else item = generic_dispatch<PV>(M, ri, rv, k - 3, sl, ovf, a.status);
          }
        } else if (lane == 0) {
          atomicOr(a.status, ST_CAPACITY);
        }
      }
      if (lane == 0 && item) {
        rsum = add_ck(rsum, item, ovf);
        if (PV) {
          atomic_add_ck(&cnt[i], item, ovf);
          if (av != 0xffffffffu) atomic_add_ck(&cnt[av], item, ovf);
        }
        if (PA) atomic_add_ck(&asub[i], item, ovf);
      }
    }
  }
  __syncthreads();
  if (PV) {
    const unsigned long long r = warp_sum64_ck(rsum, ovf);
    if (lane == 0) sh.red[warp] = r;
    __syncthreads();
    if (tid == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < kRootWarps; ++w) t = add_ck(t, sh.red[w], ovf);
      atomic_add_ck(&a.pv[u], t, ovf);
    }
    for (uint32_t i = tid; i < d; i += kRootBlock) atomic_add_ck(&a.pv[L[i]], cnt[i], ovf);
  }
  if (PA)
    for (uint32_t i = tid; i < d; i += kRootBlock) a.pa[b + i] = asub[i];
  tsum = add_ck(tsum, rsum, ovf);
  __syncthreads();
}

__device__ __forceinline__ bool past_deadline(const CountArgs &a) {
  if (a.deadline_ns && globaltimer_ns() > a.deadline_ns) {
    atomicOr(a.status, ST_TIMEOUT);
    return true;
  }
  return false;
}

__device__ inline void finish_block(const CountArgs &a, unsigned long long tsum, unsigned ovf, unsigned long long *red,
                             int nwarps) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  __syncthreads();
  const unsigned long long r = warp_sum64_ck(tsum, ovf);
  ovf = __reduce_or_sync(0xffffffffu, ovf);
  if (lane == 0) red[warp] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < nwarps; ++w) t = add_ck(t, red[w], ovf);
    atomic_add_ck(a.total, t, ovf);
  }
  if (lane == 0 && ovf) atomicOr(a.status, ovf);
}

// Persistent block roots: first the ones whose matrices live in global
// scratch (largest out-degrees), then the shared-memory ones, all in order of
// decreasing out-degree.
template <bool PV, bool PA>
__global__ void __launch_bounds__(kRootBlock) count_block_kernel(CountArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ BlockShared sh;
  const unsigned tid = threadIdx.x;
  unsigned ovf = 0;
  unsigned long long tsum = 0;
  uint8_t *slots = smem;
  uint8_t *root_area = smem + (size_t)kRootWarps * slot_layout(PV).bytes;
  if (blockIdx.x < a.scratch_blocks) {
    uint8_t *slab = a.scratch + (size_t)blockIdx.x * a.scratch_stride;
    for (;;) {
      if (tid == 0) sh.root = past_deadline(a) ? 0xffffffffu : atomicAdd(&a.queue[0], 1u);
      __syncthreads();
      const unsigned idx = sh.root;
      __syncthreads();
      if (idx >= a.n_scratch) break;
      block_root<PV, PA>(a, a.order[idx], slab, slots, tsum, ovf, sh);
    }
  }
  for (;;) {
    if (tid == 0) sh.root = past_deadline(a) ? 0xffffffffu : atomicAdd(&a.queue[1], 1u);
    __syncthreads();
    const unsigned idx = sh.root;
    __syncthreads();
    if (idx >= a.n_big - a.n_scratch) break;
    block_root<PV, PA>(a, a.order[a.n_scratch + idx], root_area, slots, tsum, ovf, sh);
  }
  finish_block(a, tsum, ovf, sh.red, kRootWarps);
}

// ------------------------------------------------------- warp-level root
// Roots with d+ <= 64: one warp, rows of one word, items over lanes (arcs for
// k = 4, triangles u->x_i->x_j for k >= 5, each lane one item).
template <bool PV, bool PA>
__device__ void warp_root(const CountArgs &a, uint32_t u, uint8_t *slot, unsigned long long &tsum, unsigned &ovf,
                          unsigned *w_next) {
  const unsigned lane = lane_id();
  const LightLayout o = light_layout(PV, PA);
  uint32_t *L = (uint32_t *)(slot + o.L);
  uint64_t *rbeg = (uint64_t *)(slot + o.rb);
  uint32_t *hkey = (uint32_t *)(slot + o.hkey);
  uint16_t *hpos = (uint16_t *)(slot + o.hpos);
  uint64_t *rows = (uint64_t *)(slot + o.rows);
  uint64_t *sym = PV ? (uint64_t *)(slot + o.colT) : nullptr;
  unsigned long long *cnt = PV ? (unsigned long long *)(slot + o.cnt) : nullptr;
  unsigned long long *asub = PA ? (unsigned long long *)(slot + o.asub) : nullptr;
  uint32_t *pre = (uint32_t *)(slot + o.pre);
  uint32_t *epre = (uint32_t *)(slot + o.epre);
  const uint64_t b = a.ptr[u];
  const uint32_t d = (uint32_t)(a.ptr[u + 1] - b);
  const int k = a.k;
  for (uint32_t i = lane; i < (uint32_t)kLightMax; i += 32) {
    rows[i] = 0;
    if (PV) {
      sym[i] = 0;
      cnt[i] = 0;
    }
    if (PA) asub[i] = 0;
  }
  for (uint32_t s = lane; s < 128; s += 32) hkey[s] = kEmpty;
  // flattened adjacency of the rows: element e of the concatenation of N+(L[i])
  uint32_t e0 = 0, e1 = 0;
  if (lane < d) {
    const uint32_t x = a.col[b + lane];
    const uint64_t xb = a.ptr[x];
    L[lane] = x;
    rbeg[lane] = xb;
    e0 = (uint32_t)(a.ptr[x + 1] - xb);
  }
  if (lane + 32 < d) {
    const uint32_t x = a.col[b + lane + 32];
    const uint64_t xb = a.ptr[x];
    L[lane + 32] = x;
    rbeg[lane + 32] = xb;
    e1 = (uint32_t)(a.ptr[x + 1] - xb);
  }
  const unsigned z0 = warp_incl_scan(e0), z1 = warp_incl_scan(e1);
  const unsigned tot0 = __shfl_sync(0xffffffffu, z0, 31), tot1 = __shfl_sync(0xffffffffu, z1, 31);
  epre[lane] = z0 - e0;
  epre[lane + 32] = tot0 + z1 - e1;
  if (lane == 0) epre[kLightMax] = tot0 + tot1;
  __syncwarp();
  for (uint32_t i = lane; i < d; i += 32) hinsert(hkey, hpos, 128, L[i], i);
  __syncwarp();
  const uint32_t E = tot0 + tot1;
  for (uint32_t e00 = lane; e00 < E; e00 += 128) {
    uint32_t y[4], row[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t e = e00 + 32 * q;
      y[q] = kEmpty;
      row[q] = 0;
      if (e < E) {
        uint32_t lo = 0, hi = d - 1;  // last row with epre <= e
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (epre[mid] <= e) lo = mid; else hi = mid - 1;
        }
        row[q] = lo;
        y[q] = a.col[rbeg[lo] + (e - epre[lo])];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (y[q] == kEmpty) continue;
      const uint32_t i = row[q];
      const int t = hlookup(hkey, hpos, 128, y[q]);
      if (t >= 0) {
        atomicOr((unsigned long long *)&rows[i], 1ull << t);
        if (PV) {
          atomicOr((unsigned long long *)&sym[t], 1ull << i);
          atomicOr((unsigned long long *)&sym[i], 1ull << t);
        }
      }
    }
  }
  __syncwarp();
  MatView V;
  V.rows = rows;
  V.sym = sym;
  V.cnt = cnt;
  V.RS = 1;
  V.W = 1;
  unsigned long long rsum = 0;
  if (k == 3) {
    for (uint32_t i = lane; i < d; i += 32) {
      const unsigned c = (unsigned)__popcll(rows[i]);
      rsum = add_ck(rsum, c, ovf);
      if (PV) cnt[i] += (unsigned)__popcll(sym[i]);
      if (PA) asub[i] = c;
    }
  } else {
    uint32_t nitems = d;
    if (k >= 5) {
      const uint32_t c0 = lane < d ? (uint32_t)__popcll(rows[lane]) : 0u;
      const uint32_t c1 = lane + 32 < d ? (uint32_t)__popcll(rows[lane + 32]) : 0u;
      const unsigned y0 = warp_incl_scan(c0), y1 = warp_incl_scan(c1);
      const unsigned t0 = __shfl_sync(0xffffffffu, y0, 31), t1 = __shfl_sync(0xffffffffu, y1, 31);
      pre[lane] = y0 - c0;
      pre[lane + 32] = t0 + y1 - c1;
      if (lane == 0) pre[kLightMax] = t0 + t1;
      nitems = t0 + t1;
    }
    if (lane == 0) *w_next = 0;
    __syncwarp();
    for (;;) {
      const unsigned t = atomicAdd(w_next, 1u);
      if (t >= nitems) break;
      uint32_t i, jv = 0xffffffffu;
      uint64_t C[1];
      int ell;
      if (k == 4) {
        i = t;
        C[0] = rows[i];
        ell = 2;
      } else {
        uint32_t lo = 0, hi = d;  // last i with pre[i] <= t
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (pre[mid] <= t) lo = mid; else hi = mid - 1;
        }
        i = lo;
        if (i >= d) {
          atomicOr(a.status, ST_CAPACITY);
          continue;
        }
        uint64_t w = rows[i];
        for (uint32_t q = t - pre[i]; q; --q) w &= w - 1;
        if (!w) {
          atomicOr(a.status, ST_CAPACITY);
          continue;
        }
        jv = (uint32_t)(__ffsll((long long)w) - 1);
        C[0] = rows[i] & rows[jv];
        ell = k - 3;
      }
      if (__popcll(C[0]) < ell) continue;
      const unsigned long long s = dfs<1, 1, PV>(C, ell, V, 0, ovf);
      rsum = add_ck(rsum, s, ovf);
      if (PV) {
        atomic_add_ck(&cnt[i], s, ovf);
        if (jv != 0xffffffffu) atomic_add_ck(&cnt[jv], s, ovf);
      }
      if (PA) atomic_add_ck(&asub[i], s, ovf);
    }
  }
  __syncwarp();
  if (PV) {
    const unsigned long long t = warp_sum64_ck(rsum, ovf);
    if (lane == 0) atomic_add_ck(&a.pv[u], t, ovf);
    for (uint32_t i = lane; i < d; i += 32) atomic_add_ck(&a.pv[L[i]], cnt[i], ovf);
  }
  if (PA)
    for (uint32_t i = lane; i < d; i += 32) a.pa[b + i] = asub[i];
  tsum = add_ck(tsum, rsum, ovf);
  __syncwarp();
}

template <bool PV, bool PA>
__global__ void __launch_bounds__(kBlock) count_warp_kernel(CountArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ unsigned long long red[kWarps];
  __shared__ unsigned w_next[kWarps];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  unsigned ovf = 0;
  unsigned long long tsum = 0;
  uint8_t *slot = smem + (size_t)warp * light_layout(PV, PA).bytes;
  const uint32_t nlight = a.n_light_end - a.n_big;
  for (;;) {
    unsigned idx = 0;
    if (lane == 0) idx = past_deadline(a) ? 0xffffffffu : atomicAdd(&a.queue[2], 1u);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= nlight) break;
    warp_root<PV, PA>(a, a.order[a.n_big + idx], slot, tsum, ovf, &w_next[warp]);
  }
  finish_block(a, tsum, ovf, red, kWarps);
}


template <bool PV, bool PA>
cudaError_t occupancy_variant(size_t block_smem, int *block_per_sm, int *warp_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(count_block_kernel<PV, PA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)block_smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(block_per_sm, count_block_kernel<PV, PA>, kRootBlock,
                                                    block_smem);
  if (e != cudaSuccess) return e;
  const size_t wsm = (size_t)kWarps * light_layout(PV, PA).bytes;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(warp_per_sm, count_warp_kernel<PV, PA>, kBlock, wsm);
}

template <bool PV, bool PA>
cudaError_t launch_variant(const CountArgs &a, int block_grid, int warp_grid, size_t block_smem, cudaStream_t s) {
  if (a.n_big > 0 && block_grid > 0) {
    count_block_kernel<PV, PA><<<block_grid, kRootBlock, block_smem, s>>>(a);
    note_launch();
  }
  if (a.n_light_end > a.n_big && warp_grid > 0) {
    const size_t wsm = (size_t)kWarps * light_layout(PV, PA).bytes;
    count_warp_kernel<PV, PA><<<warp_grid, kBlock, wsm, s>>>(a);
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace kc
